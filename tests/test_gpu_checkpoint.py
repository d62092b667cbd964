"""GPU parity of the check-point quadrature (Sec. 3.1) against its FP64
oracle, the upsampling operator alone, and the sphere closed forms through
the GPU path.

Tolerance of the mixed path: the extrapolation sum_i e_i u(c_i) amplifies the
error of the check-point values by sum_i |e_i| (351 for the default nodes
t_i = (3 + i) h_c extrapolated to t = 0), and the mixed sums carry about
2e-7 relative error, so the bar is sum |e_i| x 3e-7.  The FP64 path keeps
1e-12."""
import numpy as np
import pytest

from oracle import checkpoint as CK
from synth import geometry as G
from tests._util import cuda, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    return P


@pytest.mark.parametrize("q,eta,ncomp", [(10, 2, 3), (10, 0, 3), (10, 3, 1), (4, 1, 2), (12, 3, 3)])
def test_upsample_matches_oracle(lib, q, eta, ncomp):
    import torch
    rng = np.random.default_rng(q * 10 + eta)
    npatch = 5
    coarse = rng.normal(size=(npatch * (q + 1) ** 2, ncomp))
    ref = CK.upsample(coarse, npatch, q, 1 << eta)
    t = torch.as_tensor(coarse, device="cuda")
    fine = lib.upsample_patches(t if ncomp > 1 else t[:, 0].contiguous(), npatch, q, eta)
    got = fine.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(coarse).max()


def _sphere(a=1.0, q=10, eta=2):
    cp, cn, cw, ch = G.cubed_sphere_patches(a, q, 1)
    fine = G.cubed_sphere_patches(a, q, 1 << eta)
    hc = float(np.sqrt(cw.sum() / cw.size))
    return (cp, cn), fine, hc


def mixed_tol(R, r, p):
    return 3e-7 * np.abs(CK.extrapolation_weights(R + r * np.arange(p + 1), 0.0)).sum()


@pytest.mark.parametrize("kernels", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_matches_oracle(lib, kernels, precision):
    (cp, cn), (fp, fn, fw, fh), hc = _sphere()
    rng = np.random.default_rng(7 + kernels)
    nc = cp.shape[0]
    f = rng.uniform(-1, 1, (nc, 3))
    phi = rng.uniform(-1, 1, (nc, 3))
    # targets: every third node on the surface and a few just inside
    idx = np.arange(0, nc, 3)
    depth = np.where(np.arange(idx.size) % 4 == 0, 0.3 * hc, 0.0)
    y, n = cp[idx], cn[idx]
    x = y - depth[:, None] * n
    R, r, p = 3 * hc, hc, 4
    tol = 1e-12 if precision == "fp64" else mixed_tol(R, r, p)
    ref = CK.checkpoint_eval(kernels, f, phi, 6, 10, 4, fp, fn, fw, x, y, n, R, r, p, 0.9)
    X, Y, N, FP, FN, FW, FH, F, PHI = cuda(x, y, n, fp, fn, fw, fh, f, phi)
    plan = lib.CheckpointPlan(6, FP, FN, FW, FH, X, Y, N, R, r, p, kernels=kernels,
                              precision=precision)
    u = plan(F if kernels & 1 else None, PHI if kernels & 2 else None, 0.9).cpu().numpy()
    assert rel_l2(u, ref) <= tol, rel_l2(u, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sphere_closed_forms_on_gpu(lib, precision):
    (cp, cn), (fp, fn, fw, fh), hc = _sphere(a=2.0)
    X, N, FP, FN, FW, FH = cuda(cp, cn, fp, fn, fw, fh)
    nc = cp.shape[0]
    fvec, cvec = np.array([0.3, -0.7, 0.45]), np.array([1.0, -2.0, 0.5])
    F, PHI = cuda(np.tile(fvec, (nc, 1)), np.tile(cvec, (nc, 1)))
    # quadrature error of the scheme (oracle pins: < 1e-6) plus the mixed bar
    tol = 1e-6 + (0.0 if precision == "fp64" else mixed_tol(3 * hc, hc, 4))
    sl = lib.CheckpointPlan(6, FP, FN, FW, FH, X, X, N, 3 * hc, hc, 4, kernels=1,
                            precision=precision)
    u = sl(F, None, 1.0).cpu().numpy()
    ref = 2 * 2.0 / 3 * fvec
    assert np.abs(u - ref).max() <= tol * np.abs(ref).max(), np.abs(u - ref).max()
    dl = lib.CheckpointPlan(6, FP, FN, FW, FH, X, X, N, 3 * hc, hc, 4, kernels=2,
                            precision=precision)
    u = dl(None, PHI).cpu().numpy()
    assert np.abs(u + cvec).max() <= tol * np.abs(cvec).max(), np.abs(u + cvec).max()


def test_vessel_wall_patches_and_edge_cases(lib):
    import torch
    q, eta = 10, 2
    cp, cn, cw, ch = G.cylinder_wall_patches(12.0, 30.0, 6, 4, q)
    fp, fn, fw, fh = G.cylinder_wall_fine(12.0, 30.0, 6, 4, q, 1 << eta)
    npatch = 24
    hc = float(np.sqrt(cw.sum() / cw.size))
    rng = np.random.default_rng(3)
    phi = rng.uniform(-1, 1, (cp.shape[0], 3))
    idx = np.arange(0, cp.shape[0], 11)
    y, n = cp[idx], cn[idx]
    x = y.copy()
    # the fluid is inside the vessel: check points toward the axis (normals point outward)
    ref = CK.checkpoint_eval(2, None, phi, npatch, q, 1 << eta, fp, fn, fw, x, y, n, 3 * hc, hc, 3)
    X, Y, N, FP, FN, FW, FH, PHI = cuda(x, y, n, fp, fn, fw, fh, phi)
    plan = lib.CheckpointPlan(npatch, FP, FN, FW, FH, X, Y, N, 3 * hc, hc, 3, kernels=2,
                              precision="fp64")
    u = plan(None, PHI)
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-12
    # accumulate adds; p = 0 is the value at the single check point
    u2 = plan(None, PHI, out=u.clone(), accumulate=True).cpu().numpy()
    assert np.allclose(u2, 2 * u.cpu().numpy(), rtol=1e-14, atol=0)
    ref0 = CK.checkpoint_eval(2, None, phi, npatch, q, 1 << eta, fp, fn, fw, x, y, n, 3 * hc, hc, 0)
    plan0 = lib.CheckpointPlan(npatch, FP, FN, FW, FH, X, Y, N, 3 * hc, hc, 0, kernels=2,
                               precision="fp64")
    assert rel_l2(plan0(None, PHI).cpu().numpy(), ref0) <= 1e-12
    # no targets: nothing to do
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    plan_e = lib.CheckpointPlan(npatch, FP, FN, FW, FH, empty, empty, empty, 3 * hc, hc, 3)
    assert plan_e(None, PHI).shape == (0, 3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bie_matvec_matches_oracle(lib, precision):
    (cp, cn), (fp, fn, fw, fh), hc = _sphere(a=1.4)
    cw = G.cubed_sphere_patches(1.4, 10, 1)[2]
    rng = np.random.default_rng(19)
    phi = rng.uniform(-1, 1, (cp.shape[0], 3))
    R, r, p = 3 * hc, hc, 4
    ref = CK.bie_matvec(phi, 6, 10, 4, cp, cn, cw, fp, fn, fw, R, r, p)
    X, N, W, FP, FN, FW, FH, PHI = cuda(cp, cn, cw, fp, fn, fw, fh, phi)
    plan = lib.BIEPlan(6, X, N, W, FP, FN, FW, FH, R, r, p, precision=precision)
    u = plan.matvec(PHI).cpu().numpy()
    tol = 1e-12 if precision == "fp64" else mixed_tol(R, r, p)
    assert rel_l2(u, ref) <= tol, rel_l2(u, ref)
    # the normal field: only the rank-completing term remains (closed form)
    un = plan.matvec(N).cpu().numpy()
    refn = 4 * np.pi * 1.4 ** 2 / 3 * cn
    assert np.abs(un - refn).max() <= 1e-4 * np.abs(refn).max()
