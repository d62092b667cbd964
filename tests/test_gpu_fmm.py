"""GPU far field of the FMM (stokes_fmm_far_eval, Sec. 3.1 "Far evaluation")
against the FMM oracle's far field on an adaptive octree of the near-field
workload's kind (cells and wall patches, leaves at several depths, non-empty
V, W and X lists), with the oracle's operators on both sides; and far field +
the GPU U-list sum against the direct sum."""
import numpy as np
import pytest

import oracle
from oracle import fmm as F
from synth import octree as O
from synth import workloads as W
from tests._util import cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    oracle.build()
    import paper_1909_11085_gb300 as P
    return P


@pytest.fixture(scope="module")
def case(lib):
    """The tree from the library's own builder (equal to the generator's, which
    the oracle reads)."""
    from paper_1909_11085_gb300 import ops
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    tn = ops.octree(wl.pts, 32)
    assert np.array_equal(tn["perm"], np.arange(wl.pts.shape[0]))
    assert np.array_equal(tn["ulist_idx"], wl.tree.ulist_idx)
    fl = O.far_lists(wl.tree)
    assert np.array_equal(tn["v_idx"], fl.v_idx) and np.array_equal(tn["w_idx"], fl.w_idx)
    t = ops.fmm_tree_arrays(**ops.fmm_tree_args(tn))
    t["ulist_ptr"], t["ulist_idx"] = tn["ulist_ptr"], tn["ulist_idx"]
    return wl, t


def _oracle_ops(wl, t, p, flux):
    S = F.cube_surface(p)
    by_depth = {}
    for d in range(2, t["max_depth"] + 1):
        r = wl.tree.root_size / (1 << d) / 2
        by_depth[d] = (F.pinv(F.upward_matrix(F.R_OUTER * r * S, F.R_INNER * r * S, wl.mu, flux)),
                       F.pinv(F.stokeslet_matrix(F.R_INNER * r * S, F.R_OUTER * r * S, wl.mu)))
    return by_depth


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("flux,kinds,m2l,precision,tol", [
    (True, "sldl", "dense", "fp64", 1e-10), (False, "sl", "dense", "fp64", 1e-10),
    (True, "sldl", "fft", "fp64", 1e-10), (True, "sldl", "dense", "mixed", 1e-5),
    (True, "sldl", "fft", "mixed", 1e-5)])
def test_far_field_matches_the_oracle(lib, case, flux, kinds, m2l, precision, tol):
    """Same operators on both sides; FP64 passes to rounding, the mixed form to
    FP32 accuracy (the FMM's own error here is 2e-3)."""
    import paper_1909_11085_gb300._abi as A
    from paper_1909_11085_gb300 import ops
    wl, t = case
    p = 4
    by_depth = _oracle_ops(wl, t, p, flux)
    U = np.stack([by_depth[d][0] for d in sorted(by_depth)])
    D = np.stack([by_depth[d][1] for d in sorted(by_depth)])
    plan = ops.FmmFarPlan(t, p=p, mu=wl.mu, flux=flux, uc2e=U, dc2e=D, m2l=m2l,
                          precision=precision)
    pts, f, phi, nrm, w = cuda(wl.pts, wl.f, wl.phi, wl.nrm, wl.w)
    if kinds == "sl":
        phi = nrm = None
    L = A.lib()
    c0 = L.stokes_launch_count()
    far = plan(pts, f, phi, nrm, w).cpu().numpy()
    launches = L.stokes_launch_count() - c0
    ref = F.fmm_adaptive(wl.tree, wl.pts, wl.f, None if kinds == "sl" else wl.phi, wl.nrm, wl.w,
                         p, wl.mu, flux, ops=by_depth, near=False)
    assert _rel(far, ref) <= tol, _rel(far, ref)
    fft, mixed = m2l == "fft", precision == "mixed"
    # set-up + the passes; Fourier space adds 3 per depth; mixed adds the
    # packing and operator-splitting passes and, with spectra, their rounding,
    # and (the CTA-blocked form) the octant table, the first-child scan, the
    # parent list and the work items of the L2T (counts, their scan, the
    # list), and with spectra the table of each parent's neighbours and the
    # table of the tensor-core operand B
    assert launches == (1 + 2 + 4 * (t["max_depth"] - 1) - 1 + 3 * fft * (t["max_depth"] - 1)
                        + mixed * (2 + fft * 3 + 6))
    # accumulate
    import torch
    base = torch.full((wl.pts.shape[0], 3), 0.5, dtype=torch.float64, device="cuda")
    acc = plan(pts, f, phi, nrm, w, out=base.clone(), accumulate=True).cpu().numpy()
    np.testing.assert_allclose(acc, 0.5 + far, rtol=0, atol=1e-14 if precision == "fp64" else 1e-9)


def test_far_plus_near_is_the_fmm(lib, case):
    """With the library's own operators, far field + FP64 U-list sum on the
    GPU approximates the direct sum as the oracle's FMM does (p = 4)."""
    from paper_1909_11085_gb300 import ops
    wl, t = case
    p = 4
    plan = ops.FmmFarPlan(t, p=p, mu=wl.mu, flux=True)
    pts, f, phi, nrm, w = cuda(wl.pts, wl.f, wl.phi, wl.nrm, wl.w)
    far = plan(pts, f, phi, nrm, w)
    near = ops.P2PPlan(wl.pts.shape[0], t["leaf_ptr"], t["ulist_ptr"], t["ulist_idx"], 3, "fp64")
    u = near(pts, f, phi, nrm, w, None, wl.mu, out=far.clone(), accumulate=True).cpu().numpy()
    direct = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    ref = F.fmm_adaptive(wl.tree, wl.pts, wl.f, wl.phi, wl.nrm, wl.w, p, wl.mu, True)
    assert _rel(u, ref) <= 1e-9, _rel(u, ref)
    assert _rel(u, direct) <= 5e-3


def test_fmm_plan_from_unsorted_points(lib):
    """FmmPlan on shuffled points: the caller puts positions and densities in
    the plan's leaf order (perm) and gets the FMM velocity in that order; equal
    to the oracle's FMM on the same tree and within the p = 4 FMM error of the
    direct sum."""
    from paper_1909_11085_gb300 import ops
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    rng = np.random.default_rng(21)
    sh = rng.permutation(wl.pts.shape[0])
    cols = [a[sh] for a in (wl.pts, wl.f, wl.phi, wl.nrm, wl.w)]
    plan = ops.FmmPlan(cols[0], max_leaf=32, p=4, mu=wl.mu, near_precision="fp64")
    leaf = [c[plan.perm] for c in cols]
    u = plan(*cuda(*leaf)).cpu().numpy()
    ref = F.fmm_adaptive(wl.tree, wl.pts, wl.f, wl.phi, wl.nrm, wl.w, 4, wl.mu, True)
    # the workload's points are in leaf order; the plan's leaf order is the same tree's
    np.testing.assert_array_equal(leaf[0], wl.pts)
    assert _rel(u, ref) <= 1e-9, _rel(u, ref)
    direct = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    assert _rel(u, direct) <= 5e-3


@pytest.fixture(scope="module")
def deep(lib):
    """A tree six deep (12 cells and 6 wall patches, <= 16 points per leaf,
    7,254 points): M2M and L2L chains of four translations, W and X lists at
    several depths, and the oracle's far field with the same operators."""
    from paper_1909_11085_gb300 import ops
    wl = W.p2p_workload(ncell=12, radius=10.0, n_wall_patch=6, max_leaf=16)
    tn = ops.octree(wl.pts, 16)
    assert np.array_equal(tn["perm"], np.arange(wl.pts.shape[0]))
    t = ops.fmm_tree_arrays(**ops.fmm_tree_args(tn))
    assert t["max_depth"] == 6 and tn["w_idx"].size > 0 and tn["x_idx"].size > 0
    by_depth = _oracle_ops(wl, t, 4, True)
    ref = F.fmm_adaptive(wl.tree, wl.pts, wl.f, wl.phi, wl.nrm, wl.w, 4, wl.mu, True,
                         ops=by_depth, near=False)
    return wl, t, by_depth, ref


@pytest.mark.parametrize("m2l,precision,tol", [("fft", "fp64", 1e-10), ("fft", "mixed", 1e-5),
                                               ("dense", "mixed", 1e-5)])
def test_far_field_six_deep_tree(lib, deep, m2l, precision, tol):
    """Depth >= 5 on the device: the far field of the six-deep tree against the
    oracle's, same operators on both sides; the mixed form's per-pass events
    (stokes_fmm_set_pass_events) cover every launch but the set-up.""" 
    import ctypes
    import torch
    import paper_1909_11085_gb300._abi as A
    from paper_1909_11085_gb300 import ops
    wl, t, by_depth, ref = deep
    U = np.stack([by_depth[d][0] for d in sorted(by_depth)])
    D = np.stack([by_depth[d][1] for d in sorted(by_depth)])
    plan = ops.FmmFarPlan(t, p=4, mu=wl.mu, flux=True, uc2e=U, dc2e=D, m2l=m2l,
                          precision=precision)
    pts, f, phi, nrm, w = cuda(wl.pts, wl.f, wl.phi, wl.nrm, wl.w)
    L = A.lib()
    cap = 256
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(cap)]
    for e in evs:
        e.record()
    handles = (ctypes.c_void_p * cap)(*[e.cuda_event for e in evs])
    names = (ctypes.c_char_p * (cap // 2))()
    count = ctypes.c_int32(0)
    A.check(L.stokes_fmm_set_pass_events(handles, cap, names, ctypes.byref(count)))
    try:
        c0 = L.stokes_launch_count()
        far = plan(pts, f, phi, nrm, w).cpu().numpy()
        launches = L.stokes_launch_count() - c0
    finally:
        A.check(L.stokes_fmm_set_pass_events(None, 0, None, None))
    A.check(L.stokes_device_status(A.ptr(plan.ws), plan.ws.numel()))
    assert _rel(far, ref) <= tol, _rel(far, ref)
    if precision == "mixed":
        # the set-up kernel is not hooked; the work items (counts, scan, list)
        # are timed as one entry
        assert count.value == launches - 3
        got = {names[k].decode() for k in range(count.value)}
        assert {"s2m", "uc2e", "dchk", "dc2e", "l2t"} <= got
        assert ({"ufft", "kmulp", "ifft"} <= got) == (m2l == "fft")
        ms = [evs[2 * k].elapsed_time(evs[2 * k + 1]) for k in range(count.value)]
        assert min(ms) >= 0.0
    else:
        assert count.value == 0
