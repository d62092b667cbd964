"""Host-side FMM operators of the library (surface points and check-to-equivalent
pseudo-inverses, FP64 Jacobi SVD) against the FMM oracle's own numpy version:
the same surface, the Penrose conditions of the pseudo-inverse, and the same far
field from the equivalent densities they give.  No GPU is needed."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import fmm as F
from paper_1909_11085_gb300 import _abi as A
from paper_1909_11085_gb300 import build as B


@pytest.fixture(scope="module")
def L():
    B.build()
    oracle.build()
    return A.lib()


def _surface(L, p):
    c = ctypes.c_int32(0)
    assert L.stokes_fmm_surface(p, None, ctypes.byref(c)) == 0
    pts = np.zeros((c.value, 3))
    assert L.stokes_fmm_surface(p, pts.ctypes.data, None) == 0
    return pts


def _c2e(L, p, r, mu, upward, flux):
    ns = p ** 3 - (p - 2) ** 3
    out = np.zeros(((4 if (upward and flux) else 3) * ns, 3 * ns))
    assert L.stokes_fmm_check_to_equiv(p, r, mu, int(upward), int(flux), 1e-13, out.ctypes.data) == 0
    return out


@pytest.mark.parametrize("p", [3, 4, 6])
def test_surface_matches_the_oracle(L, p):
    np.testing.assert_allclose(_surface(L, p), F.cube_surface(p), rtol=0, atol=1e-15)


@pytest.mark.parametrize("upward,flux", [(True, True), (True, False), (False, False)])
def test_check_to_equivalent(L, upward, flux):
    p, r, mu = 4, 0.37, 0.8
    S = F.cube_surface(p)
    chk, eqv = ((F.R_OUTER, F.R_INNER) if upward else (F.R_INNER, F.R_OUTER))
    K = (F.upward_matrix(chk * r * S, eqv * r * S, mu, flux) if upward
         else F.stokeslet_matrix(chk * r * S, eqv * r * S, mu))
    X = _c2e(L, p, r, mu, upward, flux)
    # Penrose conditions of the (truncated) pseudo-inverse
    assert np.linalg.norm(K @ X @ K - K) <= 1e-9 * np.linalg.norm(K)
    assert np.linalg.norm(X @ K @ X - X) <= 1e-6 * np.linalg.norm(X)
    assert np.allclose(X @ K, (X @ K).T, rtol=0, atol=1e-6) and np.allclose(K @ X, (K @ X).T, rtol=0, atol=1e-6)
    # the field of sources inside (upward) or outside (downward) the box, fitted on
    # the check points, is reproduced where the expansion is used
    rng = np.random.default_rng(7)
    if upward:
        ys = rng.uniform(-r, r, (20, 3))
        far = rng.normal(size=(40, 3))
        far = 4 * r * far / np.linalg.norm(far, axis=1)[:, None] * rng.uniform(1, 2, (40, 1))
    else:
        ys = rng.normal(size=(20, 3))
        ys = 4 * r * ys / np.linalg.norm(ys, axis=1)[:, None] * rng.uniform(1, 2, (20, 1))
        far = rng.uniform(-r, r, (40, 3))
    fs = rng.uniform(-1, 1, (20, 3))
    src = lambda x: (F.stokeslet_matrix(x, ys, mu) @ fs.reshape(-1))
    e_lib, e_np = X @ src(chk * r * S), F.pinv(K) @ src(chk * r * S)
    Kf = (F.upward_matrix(far, eqv * r * S, mu, flux) if upward else F.stokeslet_matrix(far, eqv * r * S, mu))
    ref = src(far)
    err_lib = np.linalg.norm(Kf @ e_lib - ref) / np.linalg.norm(ref)
    err_np = np.linalg.norm(Kf @ e_np - ref) / np.linalg.norm(ref)
    assert err_lib <= 1e-3 and err_lib <= 2 * err_np + 1e-12, (err_lib, err_np)


def test_rejects_bad_arguments(L):
    out = np.zeros(1)
    assert L.stokes_fmm_check_to_equiv(1, 1.0, 1.0, 1, 1, 1e-13, out.ctypes.data) != 0
    assert L.stokes_fmm_check_to_equiv(4, -1.0, 1.0, 1, 1, 1e-13, out.ctypes.data) != 0
    assert L.stokes_fmm_check_to_equiv(4, 1.0, 1.0, 1, 1, 1e-13, None) != 0


@pytest.mark.parametrize("ncomp", [3, 4])
def test_translation_matrices_match_the_oracle(L, ncomp):
    """M2L between two boxes of one level (an offset of the interaction list)
    and M2M from a child to its parent, built from placed surfaces."""
    p, r, mu = 4, 0.25, 1.3
    S = F.cube_surface(p)
    for x, y in [(F.R_INNER * r * S, np.array([2.0, -3.0, 1.0]) * 2 * r + F.R_INNER * r * S),
                 (F.R_OUTER * 2 * r * S, np.array([0.5, -0.5, 0.5]) * 2 * r + F.R_INNER * r * S)]:
        out = np.zeros((3 * x.shape[0], ncomp * y.shape[0]))
        assert L.stokes_fmm_kernel_matrix(np.ascontiguousarray(x).ctypes.data, x.shape[0],
                                          np.ascontiguousarray(y).ctypes.data, y.shape[0], mu,
                                          ncomp, out.ctypes.data) == 0
        ref = F.upward_matrix(x, y, mu, ncomp == 4)
        np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-16 * np.abs(ref).max())


@pytest.mark.parametrize("p,flux", [(4, True), (3, False)])
def test_m2l_spectra_are_the_dft_of_the_lattice_kernel(L, p, flux):
    """The library's M2L kernel spectra are numpy's FFT of the kernel
    K(delta m - 2 o) tabulated on the zero-padded (2p)^3 lattice of index
    differences (half spectrum along z), at half-width 1; neighbouring offsets
    (never in a V-list) are zero."""
    mu, G = 0.7, 2 * p
    nc = 4 if flux else 3
    spec = np.zeros((343, G, G, p + 1, 3, nc, 2))
    assert L.stokes_fmm_m2l_spectra(p, mu, int(flux), spec.ctypes.data) == 0
    m = np.stack(np.meshgrid(*(np.arange(G),) * 3, indexing="ij"), -1).reshape(-1, 3)
    m = np.where(m >= p, m - G, m)
    delta = 2 * F.R_INNER / (p - 1)
    for o in [(2, 0, 0), (3, -2, 1), (-3, -3, 3), (0, 0, -2)]:
        K = F.upward_matrix(delta * m, 2.0 * np.array(o, float)[None, :], mu, flux)
        Kf = np.fft.fftn(K.reshape(G, G, G, 3, nc), axes=(0, 1, 2))[:, :, :p + 1]
        oi = (o[0] + 3) * 49 + (o[1] + 3) * 7 + (o[2] + 3)
        got = spec[oi, ..., 0] + 1j * spec[oi, ..., 1]
        assert np.abs(got - Kf).max() <= 1e-14 * np.abs(Kf).max()
    for o in [(0, 0, 0), (1, -1, 0), (-1, 1, 1)]:
        assert not spec[(o[0] + 3) * 49 + (o[1] + 3) * 7 + (o[2] + 3)].any()
    assert L.stokes_fmm_m2l_spectra(1, mu, 1, spec.ctypes.data) != 0
    assert L.stokes_fmm_m2l_spectra(p, -1.0, 1, spec.ctypes.data) != 0


def test_library_derives_the_tree_arrays():
    """stokes_fmm_tree_complete (through fmm_tree_arrays): depth ranges, child
    ranges, leaf boxes and the same-depth neighbours equal a brute-force search
    over the anchors of a generator tree; a misordered tree is rejected."""
    import numpy as np
    from paper_1909_11085_gb300 import ops
    from synth import octree as O
    from synth import workloads as W
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    fl = O.far_lists(wl.tree)
    t = ops.fmm_tree_arrays(fl.depth, fl.anchor, fl.parent, fl.leaf, wl.tree.leaf_ptr, fl.v_ptr,
                            fl.v_idx, fl.w_ptr, fl.w_idx, fl.x_ptr, fl.x_idx, wl.tree.root_lo,
                            wl.tree.root_size)
    dep, anc, par = np.asarray(fl.depth), np.asarray(fl.anchor), np.asarray(fl.parent)
    M = dep.size
    assert list(t["depth_ptr"]) == [int(np.searchsorted(dep, d)) for d in range(t["max_depth"] + 2)]
    for b in range(M):
        kids = np.nonzero(par == b)[0]
        assert t["child_ptr"][b + 1] - t["child_ptr"][b] == kids.size
        if kids.size:
            assert t["child_ptr"][b] == kids[0]
        for o in range(27):
            dv = np.array([o // 9 - 1, (o // 3) % 3 - 1, o % 3 - 1])
            hit = np.nonzero((dep == dep[b]) & np.all(anc == anc[b] + dv, axis=1))[0]
            assert t["colleague"][b, o] == (hit[0] if hit.size else -1)
    leaf = np.asarray(fl.leaf)
    assert np.array_equal(leaf[t["leaf_box"]], np.arange(t["leaf_box"].size))
    bad_depth = dep.copy()
    bad_depth[1] = 3
    with pytest.raises(ValueError):
        ops.fmm_tree_arrays(bad_depth, fl.anchor, fl.parent, fl.leaf, wl.tree.leaf_ptr, fl.v_ptr,
                            fl.v_idx, fl.w_ptr, fl.w_idx, fl.x_ptr, fl.x_idx, wl.tree.root_lo,
                            wl.tree.root_size)


def test_library_operators_per_depth():
    """stokes_fmm_operators: every depth's operators equal the single-depth
    pseudo-inverses of stokes_fmm_check_to_equiv at that half-width (per-depth
    upward form), and the Stokeslet-only ones scale exactly with r."""
    import ctypes
    import numpy as np
    from paper_1909_11085_gb300 import _abi as A
    from paper_1909_11085_gb300 import ops
    p, root, md, mu = 4, 40.0, 4, 0.8
    U, D = ops.fmm_operators(p, root, md, mu, True)
    ns = p ** 3 - (p - 2) ** 3
    for i, d in enumerate(range(2, md + 1)):
        r = root / (1 << d) / 2
        u1 = np.zeros((4 * ns, 3 * ns))
        d1 = np.zeros((3 * ns, 3 * ns))
        A.check(A.lib().stokes_fmm_check_to_equiv(p, r, mu, 1, 1, 1e-13, u1.ctypes.data))
        A.check(A.lib().stokes_fmm_check_to_equiv(p, r, mu, 0, 0, 1e-13, d1.ctypes.data))
        np.testing.assert_allclose(U[i], u1, rtol=0, atol=1e-9 * np.abs(u1).max())
        np.testing.assert_allclose(D[i], d1, rtol=0, atol=1e-9 * np.abs(d1).max())
