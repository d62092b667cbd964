"""The GPU far field's passes (paper_1909_11085_gb300/csrc/fmm_passes.cuh),
built for the host by tests/fmm_harness with every index checked, against the
FMM oracle's far field (Sec. 3.1, "Far evaluation") on an adaptive octree of
the near-field workload's kind; and the host set-up of the tree arrays and
operators.  No GPU is needed: the per-output functions and the pass sequence
are the ones the kernels run."""
import numpy as np
import pytest

import oracle
from oracle import fmm as F
from paper_1909_11085_gb300 import ops
from synth import octree as O
from synth import workloads as W
from tests import fmm_harness as H


@pytest.fixture(scope="module")
def case():
    oracle.build()
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    fl = O.far_lists(wl.tree)
    t = ops.fmm_tree_arrays(fl.depth, fl.anchor, fl.parent, fl.leaf, wl.tree.leaf_ptr, fl.v_ptr,
                            fl.v_idx, fl.w_ptr, fl.w_idx, fl.x_ptr, fl.x_idx, wl.tree.root_lo,
                            wl.tree.root_size)
    return wl, fl, t


def oracle_operators(wl, t, p, flux, rcond=1e-13):
    """The oracle's own pseudo-inverses per depth, as a dict and as the stacked
    arrays the passes take."""
    S = F.cube_surface(p)
    by_depth = {}
    for d in range(2, t["max_depth"] + 1):
        r = wl.tree.root_size / (1 << d) / 2
        by_depth[d] = (F.pinv(F.upward_matrix(F.R_OUTER * r * S, F.R_INNER * r * S, wl.mu, flux),
                              rcond),
                       F.pinv(F.stokeslet_matrix(F.R_INNER * r * S, F.R_OUTER * r * S, wl.mu),
                              rcond))
    U = np.stack([by_depth[d][0] for d in sorted(by_depth)])
    D = np.stack([by_depth[d][1] for d in sorted(by_depth)])
    return by_depth, U, D


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_tree_arrays(case):
    """Children are the boxes [child_ptr[b], child_ptr[b+1]) and have parent b;
    leaf_box inverts box_leaf; depth_ptr brackets each depth."""
    wl, fl, t = case
    M = t["depth"].size
    for b in range(M):
        kids = np.nonzero(t["parent"] == b)[0]
        assert list(range(t["child_ptr"][b], t["child_ptr"][b + 1])) == list(kids)
    assert np.all(t["box_leaf"][t["leaf_box"]] == np.arange(t["leaf_box"].size))
    for d in range(t["max_depth"] + 1):
        lo, hi = t["depth_ptr"][d], t["depth_ptr"][d + 1]
        assert np.all(t["depth"][lo:hi] == d)
    assert t["depth_ptr"][-1] == M and t["max_depth"] >= 3
    # colleague[b][(dx+1) 9 + (dy+1) 3 + (dz+1)]: the same-depth box at anchor + d
    where = {(int(t["depth"][b]),) + tuple(int(v) for v in t["anchor"][b]): b for b in range(M)}
    for b in range(M):
        a = t["anchor"][b]
        for o, (dx, dy, dz) in enumerate(np.ndindex(3, 3, 3)):
            want = where.get((int(t["depth"][b]), a[0] + dx - 1, a[1] + dy - 1, a[2] + dz - 1), -1)
            assert t["colleague"][b, o] == want


def test_tree_arrays_reject_a_box_order_the_passes_cannot_use(case):
    wl, fl, t = case
    args = [fl.depth, fl.anchor, fl.parent, fl.leaf, wl.tree.leaf_ptr, fl.v_ptr, fl.v_idx,
            fl.w_ptr, fl.w_idx, fl.x_ptr, fl.x_idx, wl.tree.root_lo, wl.tree.root_size]
    bad = list(args)
    bad[2] = fl.parent.copy()
    i = int(np.nonzero(fl.depth == 2)[0][0])
    j = int(np.nonzero(fl.depth == 3)[0][-1])
    bad[2][j] = fl.parent[i]  # a depth-3 box whose parent is at depth 1
    with pytest.raises(ValueError):
        ops.fmm_tree_arrays(*bad)
    bad = list(args)
    bad[3] = fl.leaf.copy()
    bad[3][bad[3] >= 0] = 0  # every leaf numbered 0
    with pytest.raises(ValueError):
        ops.fmm_tree_arrays(*bad)
    bad = list(args)
    bad[6] = fl.v_idx.copy()
    bad[6][0] = fl.depth.size  # a V entry past the last box
    with pytest.raises(ValueError):
        ops.fmm_tree_arrays(*bad)


@pytest.mark.parametrize("flux,kinds,m2l", [(True, "sldl", "dense"), (False, "sl", "dense"),
                                            (True, "dl", "dense"), (True, "sldl", "fft"),
                                            (False, "sl", "fft"), (True, "sldl", "fft-vlist")])
def test_host_passes_match_the_oracle_far_field(case, flux, kinds, m2l):
    """Same operators on both sides: the passes reproduce the oracle's far
    field (upward, V/W/X lists, downward, L2T) up to rounding, with M2L dense
    or in Fourier space (the library's kernel spectra; products blocked by
    parent through the colleague table, or summed per box over its V-list);
    the Stokeslet-only upward density (flux off) serves the single layer
    alone."""
    wl, fl, t = case
    p = 4
    by_depth, U, D = oracle_operators(wl, t, p, flux)
    f = wl.f if "sl" in kinds else None
    phi = wl.phi if kinds in ("sldl", "dl") else None
    spec = ops.fmm_m2l_spectra(p, wl.mu, flux) if m2l.startswith("fft") else None
    blocked = m2l != "fft-vlist"
    far, npass = H.far_eval(wl.pts, f, phi, wl.nrm, wl.w, t, p, U, D, wl.mu, flux, spec=spec,
                            blocked=blocked)
    ref = F.fmm_adaptive(wl.tree, wl.pts, f, phi, wl.nrm, wl.w, p, wl.mu, flux, ops=by_depth,
                         near=False)
    # the deepest depth has no M2M; Fourier-space M2L adds 3 passes per depth
    assert npass == 2 + (4 + 3 * (spec is not None)) * (t["max_depth"] - 1) - 1
    assert _rel(far, ref) <= 1e-10, _rel(far, ref)
    # accumulate adds to what out holds
    base = np.full_like(far, 0.25)
    acc, _ = H.far_eval(wl.pts, f, phi, wl.nrm, wl.w, t, p, U, D, wl.mu, flux, out=base.copy(),
                        accumulate=True, spec=spec, blocked=blocked)
    np.testing.assert_allclose(acc, base + far, rtol=0, atol=1e-15)


def test_library_operators_give_the_same_fmm(case):
    """With the library's operators (one-sided Jacobi pseudo-inverses; the
    downward one scaled by r from half-width 1) the far field stays within
    1e-10 of the oracle's at p = 4, and far field + U-list sum approximates
    the direct sum as the oracle's FMM does."""
    wl, fl, t = case
    p = 4
    U, D = ops.fmm_operators(p, t["root_size"], t["max_depth"], wl.mu, True)
    far, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, p, U, D, wl.mu, True)
    ref = F.fmm_adaptive(wl.tree, wl.pts, wl.f, wl.phi, wl.nrm, wl.w, p, wl.mu, True, near=False)
    assert _rel(far, ref) <= 1e-10, _rel(far, ref)
    near = oracle.p2p(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.tree.leaf_ptr, wl.tree.ulist_ptr,
                      wl.tree.ulist_idx, 3, wl.mu)
    direct = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    assert _rel(far + near, direct) <= 5e-3


def test_shallow_tree_has_no_far_field():
    """A tree of depth < 2 (every leaf touches every other): zero, or out unchanged."""
    oracle.build()
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (300, 3))
    tree = O.build_octree(pts, max_leaf=64)
    fl = O.far_lists(tree)
    assert int(fl.depth.max()) <= 1
    t = ops.fmm_tree_arrays(fl.depth, fl.anchor, fl.parent, fl.leaf, tree.leaf_ptr, fl.v_ptr,
                            fl.v_idx, fl.w_ptr, fl.w_idx, fl.x_ptr, fl.x_idx, tree.root_lo,
                            tree.root_size)
    sp = pts[tree.perm]
    f = rng.normal(size=(300, 3))
    w = np.full(300, 1.0 / 300)
    far, npass = H.far_eval(sp, f, None, None, w, t, 4, np.zeros((0, 1)), np.zeros((0, 1)))
    assert npass == 2 and np.all(far == 0.0)
    acc, _ = H.far_eval(sp, f, None, None, w, t, 4, np.zeros((0, 1)), np.zeros((0, 1)),
                        out=np.ones((300, 3)), accumulate=True)
    assert np.all(acc == 1.0)


@pytest.mark.parametrize("m2l,flux", [("dense", True), ("fft", True), ("fft", False)])
def test_mixed_passes_stay_within_fp32_of_the_oracle(case, m2l, flux):
    """The mixed form (FP32 evaluations on local coordinates, check-to-equivalent
    products in double-FP32 arithmetic) reproduces the oracle's far field at
    p = 4 to FP32 accuracy, far below the FMM's truncation error there (2e-3)."""
    wl, fl, t = case
    p = 4
    by_depth, U, D = oracle_operators(wl, t, p, flux)
    spec = ops.fmm_m2l_spectra(p, wl.mu, flux) if m2l == "fft" else None
    phi = wl.phi if flux else None  # without sources: the single layer alone
    far, npass = H.far_eval(wl.pts, wl.f, phi, wl.nrm, wl.w, t, p, U, D, wl.mu, flux,
                            spec=spec, mixed=True)
    ref = F.fmm_adaptive(wl.tree, wl.pts, wl.f, phi, wl.nrm, wl.w, p, wl.mu, flux,
                         ops=by_depth, near=False)
    # + the packing and operator-splitting passes, and the spectra's rounding with
    # Fourier-space M2L
    assert npass == 4 + (4 + 3 * (m2l == "fft")) * (t["max_depth"] - 1) - 1 + (m2l == "fft")
    assert _rel(far, ref) <= 1e-5, _rel(far, ref)


def test_mixed_at_p6_with_operators_cut_at_fp32_resolution(case):
    """At p = 6 the mixed form takes operators cut at rcond = 1e-7: it then
    stays within 1e-5 of the FP64 passes on the same operators, and far field +
    U-list sum approximates the direct sum as well as the FP64 form (4e-5)."""
    wl, fl, t = case
    p = 6
    _, U, D = oracle_operators(wl, t, p, True, rcond=1e-7)
    spec = ops.fmm_m2l_spectra(p, wl.mu, True)
    f64, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, p, U, D, wl.mu, True, spec=spec)
    f32, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, p, U, D, wl.mu, True, spec=spec,
                        mixed=True)
    assert _rel(f32, f64) <= 1e-5, _rel(f32, f64)
    near = oracle.p2p(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.tree.leaf_ptr, wl.tree.ulist_ptr,
                      wl.tree.ulist_idx, 3, wl.mu)
    direct = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    e64, e32 = _rel(f64 + near, direct), _rel(f32 + near, direct)
    assert e64 <= 1e-4 and e32 <= 1.05 * e64, (e64, e32)


def test_plan_set_up_on_the_host(case):
    """FmmFarPlan's set-up is host logic: operator shapes are checked against
    p and flux, the forms are validated, the mixed form at p >= 6 takes
    operators cut at 1e-7, and the workspace query sizes every buffer of the
    chosen form (FP32 points and spectra for the mixed Fourier-space form)."""
    import torch
    wl, fl, t = case
    cpu = torch.device("cpu")
    D = t["max_depth"] - 1
    ns = 4 ** 3 - 2 ** 3
    good = (np.zeros((D, 4 * ns, 3 * ns)), np.zeros((D, 3 * ns, 3 * ns)))
    with pytest.raises(ValueError):
        ops.FmmFarPlan(t, p=4, uc2e=np.zeros((D, 3 * ns, 3 * ns)), dc2e=good[1], device=cpu)
    with pytest.raises(ValueError):
        ops.FmmFarPlan(t, p=4, uc2e=good[0], dc2e=good[1], m2l="fast", device=cpu)
    with pytest.raises(ValueError):
        ops.FmmFarPlan(t, p=4, uc2e=good[0], dc2e=good[1], precision="fp16", device=cpu)
    sizes = {}
    for m2l in ("dense", "fft"):
        for prec in ("fp64", "mixed"):
            plan = ops.FmmFarPlan(t, p=4, uc2e=good[0], dc2e=good[1], m2l=m2l, precision=prec,
                                  device=cpu)
            sizes[m2l, prec] = plan.ws.numel()
    M, n, nf = t["depth"].size, int(t["leaf_ptr"][-1]), 4 * 16 * 5
    assert sizes["dense", "fp64"] >= 8 * M * (3 + 4 + 3) * ns
    assert sizes["fft", "fp64"] - sizes["dense", "fp64"] >= 8 * M * (2 * nf * 7 + 3 * ns)
    nops = D * (4 * ns + 3 * ns) * 3 * ns  # both operators, as FP32 pairs
    assert sizes["dense", "mixed"] >= 4 * 12 * n + 4 * M * (3 + 4 + 3) * ns + 8 * nops
    assert sizes["fft", "mixed"] - sizes["dense", "mixed"] >= 4 * (343 * nf * 24 + M * 2 * nf * 7)
    # the cut-off the mixed form takes at p = 6 (operators computed by the library)
    seen = []
    real = ops.fmm_operators
    try:
        ops.fmm_operators = lambda *a: (seen.append(a[5]), real(*a))[1]  # a[5]: rcond
        # the same boxes declared two deep: one depth of operators to compute
        small = {**t, "max_depth": 2, "depth_ptr": np.concatenate(
            [t["depth_ptr"][:3], [t["depth"].size]]).astype(np.int32)}
        ops.FmmFarPlan(small, p=6, precision="mixed", device=cpu)
        ops.FmmFarPlan(small, p=4, precision="mixed", device=cpu)
    finally:
        ops.fmm_operators = real
    assert seen == [1e-7, 1e-13]


def test_deep_tree_far_plus_near_is_the_fmm():
    """A tree six deep (M2M and L2L chains of four translations, W and X lists
    at several depths) where the U-list sum alone misses 93% of the velocity:
    far field (Fourier-space M2L, FP64 and mixed) + the oracle's U-list sum
    approximate the direct sum within the p = 4 FMM's error, and the mixed
    form stays within FP32 accuracy of the FP64 one."""
    oracle.build()
    wl = W.p2p_workload(ncell=12, radius=10.0, n_wall_patch=6, max_leaf=16)
    fl = O.far_lists(wl.tree)
    t = ops.fmm_tree_arrays(fl.depth, fl.anchor, fl.parent, fl.leaf, wl.tree.leaf_ptr, fl.v_ptr,
                            fl.v_idx, fl.w_ptr, fl.w_idx, fl.x_ptr, fl.x_idx, wl.tree.root_lo,
                            wl.tree.root_size)
    assert t["max_depth"] == 6 and fl.w_idx.size > 0 and fl.x_idx.size > 0
    U, D = ops.fmm_operators(4, t["root_size"], t["max_depth"], wl.mu, True)
    spec = ops.fmm_m2l_spectra(4, wl.mu, True)
    f64, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, 4, U, D, wl.mu, True, spec=spec)
    f32, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, 4, U, D, wl.mu, True, spec=spec,
                        mixed=True)
    near = oracle.p2p(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.tree.leaf_ptr, wl.tree.ulist_ptr,
                      wl.tree.ulist_idx, 3, wl.mu)
    direct = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    assert _rel(near, direct) >= 0.5
    assert _rel(f64 + near, direct) <= 3e-3
    assert _rel(f32, f64) <= 1e-5


def test_scaled_upward_operators(case):
    """upward="scaled" derives every depth's upward operator from one
    pseudo-inverse: it reproduces the check velocities at every depth as the
    per-depth operator does (A_r uc2e_r = the same projector), and the FMM it
    gives stays within the truncation error of the per-depth one."""
    wl, fl, t = case
    p = 4
    Us, Ds = ops.fmm_operators(p, t["root_size"], t["max_depth"], wl.mu, True, upward="scaled")
    Up, Dp = ops.fmm_operators(p, t["root_size"], t["max_depth"], wl.mu, True)
    np.testing.assert_array_equal(Ds, Dp)
    S = F.cube_surface(p)
    rng = np.random.default_rng(4)
    for i, d in enumerate(range(2, t["max_depth"] + 1)):
        r = t["root_size"] / (1 << d) / 2
        A = F.upward_matrix(F.R_OUTER * r * S, F.R_INNER * r * S, wl.mu, True)
        chk = A @ rng.normal(size=A.shape[1])  # a check velocity in the range
        assert _rel(A @ (Us[i] @ chk), chk) <= 1e-8
        assert _rel(A @ (Up[i] @ chk), chk) <= 1e-8
    spec = ops.fmm_m2l_spectra(p, wl.mu, True)
    fs, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, p, Us, Ds, wl.mu, True, spec=spec)
    fp, _ = H.far_eval(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t, p, Up, Dp, wl.mu, True, spec=spec)
    near = oracle.p2p(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.tree.leaf_ptr, wl.tree.ulist_ptr,
                      wl.tree.ulist_idx, 3, wl.mu)
    direct = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    es, ep = _rel(fs + near, direct), _rel(fp + near, direct)
    assert _rel(fs, fp) <= ep and es <= 1.2 * ep, (_rel(fs, fp), es, ep)


def test_double_fp32_row_product_carries_the_cancellation():
    """The mixed form's check-to-equivalent row product (operator entry split
    into an FP32 pair, exact FMA products, two-sum accumulation) meets the
    double-FP32 bound |error| <= 2 u |a.x| + 4 n u^2 sum |a_j x_j| (u = 2^-24):
    sums cancelling by a factor k come out to ~u + n u^2 k relative (1e-7 at
    k = 3e4, a few 1e-6 at k = 1e7), where a plain FP32 dot product loses every
    digit beyond k ~ 1e7."""
    rng = np.random.default_rng(17)
    u = 2.0 ** -24
    for cancel in (1e2, 1e5, 1e8):
        for _ in range(20):
            n = 456
            x = rng.normal(size=n).astype(np.float32)
            xd = x.astype(np.float64)
            a = rng.normal(size=n) * cancel
            a -= (a @ xd) / (xd @ xd) * xd  # remove most of a's projection on x
            a += rng.normal() * xd / (xd @ xd)
            exact = float(np.sum(a.astype(np.longdouble) * xd.astype(np.longdouble)))
            mag = float(np.sum(np.abs(a * xd)))
            got = H.row_df(a, x)
            assert abs(got - exact) <= 2 * u * abs(exact) + 4 * n * u * u * mag, (cancel, got, exact)
    plain = float(np.dot(a.astype(np.float32), x))
    assert abs(plain - exact) > abs(exact)  # at the strongest cancellation
