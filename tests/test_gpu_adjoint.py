"""GPU adjoint of the superposed layer potentials against the oracle's analytic
gradient and against central finite differences of the FP64 GPU forward.

Bars: FP64 form rel-L2 <= 1e-11, mixed form rel-L2 <= 1e-5 per gradient
against the oracle; finite differences (h = 1e-6) within 1e-4 of
max(|fd|, rms(grad)).  Nothing O(N^2) is stored by the backward."""
import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests._util import cuda, rel_l2

pytestmark = pytest.mark.gpu

KEYS = {"f": "grad_f", "phi": "grad_phi", "y": "grad_y", "n": "grad_n", "x": "grad_x"}


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    return P


def _case(ncell=6, box=30.0, p=12, seed=91, offset=True):
    rng = W.rng_for(seed)
    s = W.random_cells_in_box(rng, ncell, box, p)
    f, phi = W.densities(rng, s.n), W.densities(rng, s.n)
    trg = s.pts + (0.35 * s.nrm if offset else 0.0)
    g = W.densities(rng, trg.shape[0])
    return s, f, phi, trg, g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
@pytest.mark.parametrize("offset", [True, False])
def test_gradients_match_oracle(lib, precision, tol, offset):
    s, f, phi, trg, g = _case(offset=offset)
    ref = oracle.sldl_grad(s.pts, f, s.nrm, phi, s.w, trg, g, 0.9)
    Y, F, N, PH, Wt, H, X, G = cuda(s.pts, f, s.nrm, phi, s.w, s.h, trg, g)
    out = lib.sldl_grad(Y, F, N, PH, Wt, X, G, 0.9, h=H, precision=precision)
    for k, rk in KEYS.items():
        got = out[k].cpu().numpy()
        assert rel_l2(got, ref[rk]) <= tol, (k, rel_l2(got, ref[rk]))


def test_single_kernel_gradients(lib):
    s, f, phi, trg, g = _case(ncell=3, seed=92)
    Y, F, N, PH, Wt, H, X, G = cuda(s.pts, f, s.nrm, phi, s.w, s.h, trg, g)
    ref_sl = oracle.sldl_grad(s.pts, f, None, None, s.w, trg, g, 1.0)
    out = lib.sldl_grad(Y, F, None, None, Wt, X, G, 1.0, h=H, want=("f", "y", "x"))
    for k in ("f", "y", "x"):
        assert rel_l2(out[k].cpu().numpy(), ref_sl[KEYS[k]]) <= 1e-5
    ref_dl = oracle.sldl_grad(s.pts, None, s.nrm, phi, s.w, trg, g, 1.0)
    out = lib.sldl_grad(Y, None, N, PH, Wt, X, G, 1.0, h=H, want=("phi", "y", "n", "x"))
    for k in ("phi", "y", "n", "x"):
        assert rel_l2(out[k].cpu().numpy(), ref_dl[KEYS[k]]) <= 1e-5


def test_gradients_match_finite_differences(lib):
    import torch
    s, f, phi, trg, g = _case(ncell=3, seed=93)
    Y, F, N, PH, Wt, H, X, G = cuda(s.pts, f, s.nrm, phi, s.w, s.h, trg, g)
    grads = {p: lib.sldl_grad(Y, F, N, PH, Wt, X, G, 1.0, h=H, precision=p)
             for p in ("mixed", "fp64")}
    args = {"y": Y, "f": F, "n": N, "phi": PH, "x": X}
    rng = W.rng_for(5)
    hstep = 1e-6

    def loss(a):
        u = lib.sldl(a["y"], a["f"], a["n"], a["phi"], Wt, a["x"], 1.0, h=H, precision="fp64")
        return float(torch.sum(u * G))

    for name, t in args.items():
        # 64 sampled scalar coordinates per tensor
        for idx in rng.choice(t.numel(), 64, replace=False):
            i, k = divmod(int(idx), 3)
            vals = []
            for sgn in (1, -1):
                a2 = dict(args)
                a2[name] = t.clone()
                a2[name][i, k] += sgn * hstep
                vals.append(loss(a2))
            fd = (vals[0] - vals[1]) / (2 * hstep)
            for p, gr in grads.items():
                ref = gr[name]
                rms = float(torch.sqrt(torch.mean(ref ** 2)))
                assert abs(fd - float(ref[i, k])) <= 1e-4 * max(abs(fd), rms), (p, name, fd,
                                                                               float(ref[i, k]))


def test_autograd_function(lib):
    import torch
    s, f, phi, trg, g = _case(ncell=3, seed=94, offset=False)
    Y, F, N, PH, Wt, H, G = cuda(s.pts, f, s.nrm, phi, s.w, s.h, g)
    Y.requires_grad_(True)
    F.requires_grad_(True)
    N.requires_grad_(True)
    PH.requires_grad_(True)
    u = lib.StokesLayerFn.apply(Y, F, N, PH, Wt, Y, 1.0, H)  # targets are the sources
    torch.sum(u * G).backward()
    ref = oracle.sldl_grad(s.pts, f, s.nrm, phi, s.w, s.pts, g, 1.0)
    assert rel_l2(F.grad.cpu().numpy(), ref["grad_f"]) <= 1e-5
    assert rel_l2(PH.grad.cpu().numpy(), ref["grad_phi"]) <= 1e-5
    assert rel_l2(N.grad.cpu().numpy(), ref["grad_n"]) <= 1e-5
    # the shared position tensor receives the source and the target parts
    assert rel_l2(Y.grad.cpu().numpy(), ref["grad_y"] + ref["grad_x"]) <= 1e-5


def test_full_size_sampled(lib):
    """64 cells (34,816 points), targets = sources, sampled against the oracle."""
    wl, g = W.adjoint_workload()
    Y, F, N, PH, Wt, H, G = cuda(wl.src, wl.f, wl.nrm, wl.phi, wl.w, wl.h, g)
    rng = W.rng_for(95)
    js = np.sort(rng.choice(wl.src.shape[0], 200, replace=False))
    ref_src = oracle.sldl_grad(wl.src[js], wl.f[js], wl.nrm[js], wl.phi[js], wl.w[js], wl.trg, g,
                               1.0)
    ref_trg = oracle.sldl_grad(wl.src, wl.f, wl.nrm, wl.phi, wl.w, wl.trg[js], g[js], 1.0)
    for prec, tol in (("mixed", 1e-5), ("fp64", 1e-11)):
        out = lib.sldl_grad(Y, F, N, PH, Wt, None, G, 1.0, h=H, precision=prec)
        for k in ("f", "phi", "y", "n"):
            assert rel_l2(out[k].cpu().numpy()[js], ref_src[KEYS[k]]) <= tol, (prec, k)
        assert rel_l2(out["x"].cpu().numpy()[js], ref_trg["grad_x"]) <= tol, (prec, "x")


def test_dense_cluster_overflows_the_near_lists(lib):
    """Every pair near (spacing h larger than the cluster): each point has more near
    inputs than the per-point list holds, so the mixed form's FP64 pass rescans
    them with the FP32 pass's frame; a second cluster far away keeps far pairs in
    the same call.  Compared with the oracle's analytic gradient at 1e-7: the far
    pairs between the clusters carry FP32 rounding (2e-8 here), while a near pair
    missed or counted twice would move a point's gradient by about 1e-2."""
    rng = np.random.default_rng(95)
    m = 96
    a = rng.uniform(-0.5, 0.5, (m, 3))
    b = rng.uniform(-0.5, 0.5, (m, 3)) + np.array([20.0, 0.0, 0.0])
    pts = np.concatenate([a, b])
    n = pts.shape[0]
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    f, phi, g = (rng.uniform(-1, 1, (n, 3)) for _ in range(3))
    w = rng.uniform(0.01, 0.02, n)
    h = np.full(n, 3.0)  # alpha h = 3 > cluster diameter: all pairs inside a cluster are near
    trg = pts + 0.01 * rng.normal(size=(n, 3))
    ref = oracle.sldl_grad(pts, f, nrm, phi, w, trg, g, 1.0)
    Y, F, N, PH, Wt, H, X, G = cuda(pts, f, nrm, phi, w, h, trg, g)
    out = lib.sldl_grad(Y, F, N, PH, Wt, X, G, 1.0, h=H, precision="mixed")
    for k, rk in KEYS.items():
        got = out[k].cpu().numpy()
        assert rel_l2(got, ref[rk]) <= 1e-7, (k, rel_l2(got, ref[rk]))
