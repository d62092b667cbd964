"""Pins of the check-point quadrature oracle (Sec. 3.1, "Singular and
near-singular integral quadrature") against what the mathematics fixes:
polynomial exactness of the upsampling and the extrapolation, and closed
forms on a sphere for targets on and just inside the surface (uniform
single layer: 2 a f / (3 mu); constant double layer: the interior limit -c;
rigid-motion double layer: -(a + w x x))."""
import numpy as np
import pytest

from oracle import checkpoint as CK
from synth import geometry as G

Q, M, P_EXT = 10, 4, 4


def test_interpolation_exact_for_degree_q():
    rng = np.random.default_rng(1)
    c = rng.normal(size=Q + 1)
    poly = np.polynomial.Polynomial(c)
    t = rng.uniform(-1, 1, 50)
    Mx = CK.interp_matrix(Q, t)
    np.testing.assert_allclose(Mx @ poly(CK.cc_nodes(Q)), poly(t), rtol=0, atol=1e-12 * np.abs(c).sum())
    assert np.allclose(Mx.sum(1), 1.0)  # constants are reproduced
    # at the nodes the interpolant is the data
    np.testing.assert_array_equal(CK.interp_matrix(Q, CK.cc_nodes(Q)), np.eye(Q + 1))


def test_upsampling_of_a_tensor_polynomial_is_exact():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(Q + 1, Q + 1))
    pval = lambda u, v: np.polynomial.polynomial.polyval2d(u, v, A)
    x = CK.cc_nodes(Q)
    U, V = np.meshgrid(x, x, indexing="ij")
    coarse = np.stack([pval(U, V).ravel(), np.ones(U.size), U.ravel()], axis=1)
    coarse = np.tile(coarse, (2, 1))  # two patches
    fine = CK.upsample(coarse, 2, Q, M)
    us, vs, _ = G._patch_grid_nodes(Q, M)
    ref = []
    for _ in range(2):
        for s in range(M * M):
            Uf, Vf = np.meshgrid(us[s], vs[s], indexing="ij")
            ref.append(np.stack([pval(Uf, Vf).ravel(), np.ones(Uf.size), Uf.ravel()], axis=1))
    ref = np.concatenate(ref)
    np.testing.assert_allclose(fine, ref, rtol=0, atol=1e-11 * np.abs(A).sum())


def test_extrapolation_weights_exact_for_degree_p():
    tn = 0.3 + 0.1 * np.arange(P_EXT + 1)
    for t in (0.0, 0.05, -0.02, 0.31):
        e = CK.extrapolation_weights(tn, t)
        for k in range(P_EXT + 1):
            assert abs(e @ tn ** k - t ** k) <= 1e-12 * max(1.0, abs(t) ** k)


@pytest.fixture(scope="module")
def sphere():
    a = 1.3
    cp, cn, cw, ch = G.cubed_sphere_patches(a, Q, 1)
    fp, fn, fw, fh = G.cubed_sphere_patches(a, Q, M)
    hc = float(np.sqrt(cw.sum() / cw.size))
    return a, (cp, cn, cw), (fp, fn, fw), hc


def _targets(cp, cn, depth):
    idx = np.arange(0, cp.shape[0], 5)
    y, n = cp[idx], cn[idx]
    return y - depth * n, y, n


@pytest.mark.parametrize("depth_frac", [0.0, 0.4, 1.5])
def test_sphere_uniform_single_layer(sphere, depth_frac):
    a, (cp, cn, cw), (fp, fn, fw), hc = sphere
    mu = 0.8
    x, y, n = _targets(cp, cn, depth_frac * hc)
    fvec = np.array([0.3, -0.7, 0.45])
    f = np.tile(fvec, (cp.shape[0], 1))
    u = CK.checkpoint_eval(1, f, None, 6, Q, M, fp, fn, fw, x, y, n, 3 * hc, hc, P_EXT, mu)
    ref = 2 * a / (3 * mu) * fvec
    assert np.abs(u - ref).max() <= 1e-6 * np.abs(ref).max(), np.abs(u - ref).max()


@pytest.mark.parametrize("depth_frac", [0.0, 0.4, 1.5])
def test_sphere_constant_double_layer_interior_limit(sphere, depth_frac):
    a, (cp, cn, cw), (fp, fn, fw), hc = sphere
    x, y, n = _targets(cp, cn, depth_frac * hc)
    cvec = np.array([1.0, -2.0, 0.5])
    phi = np.tile(cvec, (cp.shape[0], 1))
    u = CK.checkpoint_eval(2, None, phi, 6, Q, M, fp, fn, fw, x, y, n, 3 * hc, hc, P_EXT)
    assert np.abs(u + cvec).max() <= 1e-6 * np.abs(cvec).max(), np.abs(u + cvec).max()


def test_sphere_rigid_motion_double_layer(sphere):
    """a + w x y is not a polynomial on a gnomonic patch, so upsampling it from
    the 11 x 11 nodes costs about 6e-5; with the density sampled exactly on the
    fine nodes, check points and extrapolation alone reproduce the closed form."""
    import oracle
    a, (cp, cn, cw), (fp, fn, fw), hc = sphere
    x, y, n = _targets(cp, cn, 0.0)
    av, om = np.array([0.2, 0.1, -0.3]), np.array([0.5, -0.4, 0.25])
    ref = -(av + np.cross(om, x))
    u = CK.checkpoint_eval(2, None, av + np.cross(om, cp), 6, Q, M, fp, fn, fw, x, y, n, 3 * hc,
                           hc, P_EXT)
    assert np.abs(u - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(u - ref).max()
    c = CK.check_points(y, n, 3 * hc, hc, P_EXT).reshape(-1, 3)
    uc = oracle.dl(fp, fn, av + np.cross(om, fp), fw, c).reshape(y.shape[0], P_EXT + 1, 3)
    e = CK.extrapolation_weights(3 * hc + hc * np.arange(P_EXT + 1), 0.0)
    ue = np.einsum("q,tqc->tc", e, uc)
    assert np.abs(ue - ref).max() <= 1e-6 * np.abs(ref).max(), np.abs(ue - ref).max()


def test_refinement_reduces_the_error(sphere):
    """The same constant-density problem with 4 instead of 16 sub-patches is
    much less accurate at the same check points (the fine rule resolves them)."""
    a, (cp, cn, cw), (fp, fn, fw), hc = sphere
    f2 = G.cubed_sphere_patches(a, Q, 2)
    x, y, n = _targets(cp, cn, 0.0)
    phi = np.tile([1.0, 0.0, 0.0], (cp.shape[0], 1))
    e4 = np.abs(CK.checkpoint_eval(2, None, phi, 6, Q, M, fp, fn, fw, x, y, n, 2 * hc, hc, P_EXT)[:, 0] + 1).max()
    e2 = np.abs(CK.checkpoint_eval(2, None, phi, 6, Q, 2, f2[0], f2[1], f2[2], x, y, n, 2 * hc, hc,
                                   P_EXT)[:, 0] + 1).max()
    assert e4 < e2 / 50, (e2, e4)


def test_null_space_term_closed_forms(sphere):
    """N on a sphere of radius a: N n = (4 pi a^2 / 3) n, N[a0 + w x y] = (4 pi a^3 / 3) n x w."""
    a, (cp, cn, cw), _, hc = sphere
    np.testing.assert_allclose(CK.null_space_term(cn, cn, cw, cn), 4 * np.pi * a * a / 3 * cn,
                               rtol=0, atol=1e-5)
    a0, om = np.array([0.2, -0.1, 0.4]), np.array([0.5, -0.4, 0.25])
    got = CK.null_space_term(a0 + np.cross(om, cp), cn, cw, cn)
    np.testing.assert_allclose(got, 4 * np.pi * a ** 3 / 3 * np.cross(cn, om), rtol=0, atol=1e-5)


def test_bie_operator_null_vector_and_rigid_motion(sphere):
    """The fluid-side limit of the double layer annihilates the normal field and
    maps a + w x y to -(a + w x x) (Lorentz reciprocity), so the operator gives
    N n for phi = n and -(a + w x x) + N[a + w x y] for a rigid motion."""
    a, (cp, cn, cw), (fp, fn, fw), hc = sphere
    u = CK.bie_matvec(cn, 6, Q, M, cp, cn, cw, fp, fn, fw, 3 * hc, hc, P_EXT)
    ref = 4 * np.pi * a * a / 3 * cn
    assert np.abs(u - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(u - ref).max()
    a0, om = np.array([0.2, -0.1, 0.4]), np.array([0.5, -0.4, 0.25])
    u = CK.bie_matvec(a0 + np.cross(om, cp), 6, Q, M, cp, cn, cw, fp, fn, fw, 3 * hc, hc, P_EXT)
    ref = -(a0 + np.cross(om, cp)) + 4 * np.pi * a ** 3 / 3 * np.cross(cn, om)
    assert np.abs(u - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(u - ref).max()
