"""Pins of the kernel-independent FMM oracle (the far field of Sec. 3.1, "Far
evaluation") against what the mathematics fixes: with no far field (a tree of
depth 1) it is the direct sum; a leaf's upward equivalent density reproduces the
leaf's field away from it; the error against the direct sum falls with the
surface order; and the double layer's far field needs the point-source part of
the equivalent density (Stokeslets carry no flux)."""
import numpy as np
import pytest

import oracle
from oracle import fmm as F


@pytest.fixture(scope="module")
def cloud():
    oracle.build()
    rng = np.random.default_rng(5)
    n = 800
    pts = rng.uniform(0, 1, (n, 3))
    f, phi = rng.uniform(-1, 1, (n, 3)), rng.uniform(-1, 1, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    w = rng.uniform(0.5, 1.5, n) / n
    return pts, f, phi, nrm, w


def _rel(u, r):
    return np.linalg.norm(u - r) / np.linalg.norm(r)


def test_without_far_field_it_is_the_direct_sum(cloud):
    pts, f, phi, nrm, w = cloud
    ref = oracle.sldl(pts, f, nrm, phi, w, pts, 0.8)
    u = F.fmm(pts, f, phi, nrm, w, depth=1, p=4, mu=0.8)
    assert _rel(u, ref) <= 1e-13


def test_leaf_equivalent_density_reproduces_its_far_field(cloud):
    pts, f, phi, nrm, w = cloud
    sel = np.all(pts < 0.25, axis=1)  # one box of half-width 0.125 about (0.125,)*3
    c, r = np.full(3, 0.125), 0.125
    rng = np.random.default_rng(6)
    d = rng.normal(size=(50, 3))
    # at 2 to 6 box widths from the centre, as interaction-list boxes are
    far = c + 4 * r * (d / np.linalg.norm(d, axis=1)[:, None]) * rng.uniform(1.0, 3.0, (50, 1))
    ref = oracle.sldl(pts[sel], f[sel], nrm[sel], phi[sel], w[sel], far, 1.0)
    err = {}
    for p in (4, 6):
        S = F.cube_surface(p)
        chk = oracle.sldl(pts[sel], f[sel], nrm[sel], phi[sel], w[sel], c + F.R_OUTER * r * S, 1.0)
        e = F.pinv(F.upward_matrix(F.R_OUTER * r * S, F.R_INNER * r * S, 1.0, True)) @ chk.reshape(-1)
        got = (F.upward_matrix(far, c + F.R_INNER * r * S, 1.0, True) @ e).reshape(-1, 3)
        err[p] = _rel(got, ref)
    assert err[6] <= 1e-3 and err[6] <= err[4] / 5, err


def test_error_falls_with_surface_order(cloud):
    pts, f, phi, nrm, w = cloud
    ref = oracle.sldl(pts, f, nrm, phi, w, pts, 1.0)
    e4 = _rel(F.fmm(pts, f, phi, nrm, w, depth=3, p=4), ref)
    e6 = _rel(F.fmm(pts, f, phi, nrm, w, depth=3, p=6), ref)
    assert e4 <= 1e-2 and e6 <= 5e-4 and e6 <= e4 / 10, (e4, e6)


def test_double_layer_far_field_needs_the_source_term(cloud):
    pts, f, phi, nrm, w = cloud
    ref = oracle.sldl(pts, np.zeros_like(f), nrm, phi, w, pts, 1.0)
    with_flux = _rel(F.fmm(pts, None, phi, nrm, w, depth=3, p=4, flux=True), ref)
    stokeslets = _rel(F.fmm(pts, None, phi, nrm, w, depth=3, p=4, flux=False), ref)
    assert with_flux <= 1e-2 and stokeslets >= 10 * with_flux, (with_flux, stokeslets)


def test_adaptive_tree_matches_the_direct_sum():
    """On an adaptive octree of the near-field workload's kind (cells and wall
    patches, leaves at several depths) the W and X lists carry real interactions,
    and the far field still falls with the surface order against the direct sum."""
    from synth import workloads as W
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    ref = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts, wl.mu)
    st = {}
    e4 = _rel(F.fmm_adaptive(wl.tree, wl.pts, wl.f, wl.phi, wl.nrm, wl.w, 4, wl.mu, stats=st), ref)
    e5 = _rel(F.fmm_adaptive(wl.tree, wl.pts, wl.f, wl.phi, wl.nrm, wl.w, 5, wl.mu), ref)
    assert st["w"] > 0 and st["x"] > 0 and st["v"] > 0 and len(set(wl.tree.leaf_depth)) > 1
    assert e4 <= 5e-3 and e5 <= e4 / 2, (e4, e5)


def test_generated_far_lists_match_their_definitions():
    """The interaction lists the input generator hands to both paths (as it hands
    the U-lists) equal the oracle's, which follow the definitions box by box."""
    from synth import octree as O
    from synth import workloads as W
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    fl = O.far_lists(wl.tree)
    st = {}
    F.fmm_adaptive(wl.tree, wl.pts[:0], None, None, None, np.zeros(0), 2, stats=st, lists_only=True)
    key = lambda n: (int(fl.depth[n]),) + tuple(int(v) for v in fl.anchor[n])
    for name, ptr, idx in (("V", fl.v_ptr, fl.v_idx), ("W", fl.w_ptr, fl.w_idx), ("X", fl.x_ptr, fl.x_idx)):
        ref = st["lists"][name]
        got = {key(n): sorted(key(int(a)) for a in idx[ptr[n]:ptr[n + 1]]) for n in range(fl.depth.size)}
        for nd, lst in ref.items():
            assert sorted(lst) == got[nd], (name, nd)
        assert sum(len(v) for v in got.values()) == sum(len(v) for v in ref.values()), name


@pytest.mark.parametrize("p", [4, 6])
def test_m2l_is_a_circular_convolution_on_the_surface_lattice(p):
    """The upward equivalent and downward check surfaces of two boxes share one
    radius (1.05 r), so their points are the boundary of one p^3 lattice of
    spacing 2 (1.05 r) / (p - 1), shifted by the boxes' offset o; the kernel
    then depends on the lattice index difference alone, K(delta (i - j) - o).
    Zero-padding to a (2p)^3 grid turns the M2L translation into a circular
    convolution whose FFT form equals the dense translation up to rounding,
    for any o (no lattice alignment of o is needed)."""
    rng = np.random.default_rng(p)
    r = 0.37
    a = F.R_INNER * r
    delta = 2 * a / (p - 1)
    S = F.cube_surface(p)
    idx = np.rint((S + 1) * (p - 1) / 2).astype(int)
    np.testing.assert_allclose(-a + delta * idx, a * S, atol=1e-15)
    g = 2 * p
    m = np.stack(np.meshgrid(*(np.arange(g),) * 3, indexing="ij"), -1).reshape(-1, 3)
    m = np.where(m >= p, m - g, m)  # index differences -(p-1)..p-1, circular storage
    e = rng.normal(size=(S.shape[0], 4))
    E = np.zeros((g, g, g, 4))
    E[idx[:, 0], idx[:, 1], idx[:, 2]] = e
    Ef = np.fft.fftn(E, axes=(0, 1, 2))
    for o in [(2, 0, 0), (3, -2, 1), (-2, 3, 3), (-3, -3, 2)]:
        oc = np.asarray(o, float) * 2 * r
        dense = F.upward_matrix(a * S, oc + a * S, 1.0, True) @ e.reshape(-1)
        K = F.upward_matrix(delta * m, oc[None, :], 1.0, True).reshape(g, g, g, 3, 4)
        Uf = np.einsum("xyzij,xyzj->xyzi", np.fft.fftn(K, axes=(0, 1, 2)), Ef)
        U = np.real(np.fft.ifftn(Uf, axes=(0, 1, 2)))
        conv = U[idx[:, 0], idx[:, 1], idx[:, 2]].reshape(-1)
        assert _rel(conv, dense) <= 1e-13


@pytest.mark.parametrize("p,rcond,ratio", [(4, 1e-13, 0.2), (6, 1e-13, 1.0), (6, 1e-7, 0.2)])
def test_m2l_inputs_rounded_to_fp32_stay_below_the_truncation_error(p, rcond, ratio):
    """The precision reading for a single-precision M2L: the upward equivalent
    densities stay within a few times the check velocities they reproduce (no
    large cancelling coefficients), so rounding them and the translation to
    FP32 changes the field a V-list pair carries into the target box by less
    than the FMM's own truncation error at that order: a fifth of it at p = 4;
    at p = 6 up to the error itself with the pseudo-inverses cut at 1e-13, and
    a fifth of it when they are cut at 1e-7 (FP32's resolution)."""
    oracle.build()
    rng = np.random.default_rng(40 + p)
    S = F.cube_surface(p)
    r = 0.1
    uc2e = F.pinv(F.upward_matrix(F.R_OUTER * r * S, F.R_INNER * r * S, 1.0, True), rcond)
    dc2e = F.pinv(F.stokeslet_matrix(F.R_INNER * r * S, F.R_OUTER * r * S, 1.0), rcond)
    o = np.array([3.0, 1.0, -2.0]) * 2 * r
    M = F.upward_matrix(o + F.R_INNER * r * S, F.R_INNER * r * S, 1.0, True)
    for _ in range(3):
        y = rng.uniform(-r, r, (60, 3))
        f, phi = rng.normal(size=(60, 3)), rng.normal(size=(60, 3))
        n = rng.normal(size=(60, 3))
        n /= np.linalg.norm(n, axis=1)[:, None]
        w = np.full(60, 0.01)
        chk = oracle.sldl(y, f, n, phi, w, F.R_OUTER * r * S, 1.0).reshape(-1)
        up = uc2e @ chk
        assert np.abs(up).max() <= 10 * np.abs(chk).max()
        x = o + rng.uniform(-r, r, (40, 3))
        L2T = F.stokeslet_matrix(x, o + F.R_OUTER * r * S, 1.0)
        u64 = L2T @ (dc2e @ (M @ up))
        u32 = L2T @ (dc2e @ (M.astype(np.float32) @ up.astype(np.float32)).astype(np.float64))
        true = oracle.sldl(y, f, n, phi, w, x, 1.0).reshape(-1)
        trunc = _rel(u64, true)
        assert _rel(u32, u64) <= ratio * trunc, (_rel(u32, u64), trunc)


def test_check_to_equivalent_products_need_fp64():
    """Why the mixed far field keeps the check-to-equivalent products in FP64:
    the operators' entries reach 1e3 (p = 4) to 6e7 (p = 6), so the same
    products in FP32 move the field a V-list pair carries by 1e-3 at p = 4
    (about the whole FMM's error there) and by more than the field itself at
    p = 6, against 1e-5 or less for the FP32 M2L inputs."""
    oracle.build()
    rng = np.random.default_rng(77)
    change = {}
    for p in (4, 6):
        S = F.cube_surface(p)
        r = 0.1
        uc2e = F.pinv(F.upward_matrix(F.R_OUTER * r * S, F.R_INNER * r * S, 1.0, True))
        dc2e = F.pinv(F.stokeslet_matrix(F.R_INNER * r * S, F.R_OUTER * r * S, 1.0))
        o = np.array([3.0, 1.0, -2.0]) * 2 * r
        M = F.upward_matrix(o + F.R_INNER * r * S, F.R_INNER * r * S, 1.0, True)
        y = rng.uniform(-r, r, (60, 3))
        f, phi = rng.normal(size=(60, 3)), rng.normal(size=(60, 3))
        n = rng.normal(size=(60, 3))
        n /= np.linalg.norm(n, axis=1)[:, None]
        chk = oracle.sldl(y, f, n, phi, np.full(60, 0.01), F.R_OUTER * r * S, 1.0).reshape(-1)
        L2T = F.stokeslet_matrix(o + rng.uniform(-r, r, (40, 3)), o + F.R_OUTER * r * S, 1.0)

        def field(dt):
            up = (uc2e.astype(dt) @ chk.astype(dt)).astype(np.float64)
            dn = (dc2e.astype(dt) @ (M @ up).astype(dt)).astype(np.float64)
            return L2T @ dn
        change[p] = _rel(field(np.float32), field(np.float64))
    assert 3e-4 <= change[4] <= 1e-2, change
    assert change[6] >= 1.0, change
