"""Pins of the FP64 CPU oracle to facts that do not come from the oracle itself.

Each test targets a plausible slip in the oracle: a dropped term, a wrong
sign, constant or power, a transposed operand, a misplaced weight or a wrong
restriction of the near-field sum.
  * hand values of both kernels (tests/golden/hand_values.txt);
  * the single layer of a uniformly loaded sphere (Stokes drag: (2a/(3mu)) F
    inside, the Stokeslet-plus-degenerate-quadrupole field outside);
  * the double-layer identity for constant density on a closed surface
    (-c inside, -c/2 on the surface, 0 outside) and its rigid-motion form;
  * symmetry of the Stokeslet, translation/rotation invariance, linearity;
  * the near-field (U-list) sum against the direct sum over the same sources.
"""
import os

import numpy as np
import pytest

import oracle
from synth import geometry as G
from synth.octree import build_octree
from synth.workloads import random_cells_in_box, rng_for, interior_targets

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_values.txt")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_hand_values():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for r in rows:
        kind, mu = r[0], float(r[1])
        d, n, dens = (np.array(r[2 + 3 * k:5 + 3 * k], float) for k in range(3))
        w, exp = float(r[11]), np.array(r[12:15], float) / (8 * np.pi)
        y = np.zeros((1, 3))
        x = d[None]
        if kind == "sl":
            u = oracle.sl(y, dens[None], [w], x, mu)
        else:
            u = oracle.dl(y, n[None], dens[None], [w], x)
        np.testing.assert_allclose(u[0], exp, rtol=1e-14, atol=1e-16)


def _sphere_sl_exact(x, a, mu, F):
    r = np.linalg.norm(x)
    if r <= a:
        return 2 * a / (3 * mu) * F
    I, xx = np.eye(3), np.outer(x, x)
    return (a * a / (2 * mu)) * ((I / r + xx / r ** 3) + (a * a / 3) * (I / r ** 3 - 3 * xx / r ** 5)) @ F


@pytest.mark.parametrize("a,mu", [(1.0, 1.0), (2.3, 0.7)])
def test_sphere_single_layer_closed_form(a, mu):
    rng = rng_for(7)
    F = rng.uniform(-1, 1, 3)
    X, n, w = G.sphere_surface(32, a)
    dirs = rng.normal(size=(12, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    radii = np.array([0.0, 0.2, 0.4, 0.5, 0.55, 0.6, 1.5, 1.8, 2.5, 4.0, 8.0, 20.0]) * a
    trg = dirs * radii[:, None]
    u = oracle.sl(X, np.tile(F, (X.shape[0], 1)), w, trg, mu)
    for i in range(trg.shape[0]):
        ue = _sphere_sl_exact(trg[i], a, mu, F)
        assert np.linalg.norm(u[i] - ue) <= 1e-10 * np.linalg.norm(F) * a / mu, (i, u[i], ue)


def test_sphere_single_layer_converges_spectrally():
    F = np.array([0.3, -0.2, 0.5])
    x = np.array([[0.0, 0.0, 0.8]])
    errs = []
    for p in (8, 16, 24, 32):
        X, n, w = G.sphere_surface(p, 1.0)
        u = oracle.sl(X, np.tile(F, (X.shape[0], 1)), w, x, 1.0)
        errs.append(np.linalg.norm(u[0] - _sphere_sl_exact(x[0], 1.0, 1.0, F)))
    # geometric decrease by more than 10x per 8 orders at distance 0.2 from the surface
    for k in range(3):
        assert errs[k + 1] < 0.1 * errs[k]
    assert errs[3] < 1e-6


def _cell(p, seed=3):
    rng = rng_for(seed)
    return random_cells_in_box(rng, 1, 12.0, p)


def test_double_layer_identity_constant_density():
    """Constant c on a closed surface: D[c] = -c inside, 0 outside.

    On a sphere the rule is spectrally exact at these distances; on a
    biconcave cell the interior ring (about 1 um from the surface) converges
    geometrically in the order p.
    """
    c = np.array([0.4, -1.1, 0.7])
    X, n, w = G.sphere_surface(24, 1.3)
    t = np.array([[0, 0, 0], [0.3, 0.2, -0.4], [3, 1, 0], [0, -4, 1.0]])
    u = oracle.dl(X, n, np.tile(c, (X.shape[0], 1)), w, t)
    np.testing.assert_allclose(u[:2], -np.tile(c, (2, 1)), atol=1e-13)
    np.testing.assert_allclose(u[2:], 0.0, atol=1e-14)
    errs = []
    for p in (16, 24, 32, 48):
        s = _cell(p)
        inside = interior_targets(s, 8)
        dirs = rng_for(5).normal(size=(8, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        outside = s.centres[0] + dirs * 9.0
        u = oracle.dl(s.pts, s.nrm, np.tile(c, (s.n, 1)), s.w, np.concatenate([inside, outside]))
        errs.append(np.abs(u[:8] + c).max())
        np.testing.assert_allclose(u[8:], 0.0, atol=1e-6)
    for k in range(3):
        assert errs[k + 1] < 0.05 * errs[k]
    assert errs[3] < 1e-9


def test_double_layer_identity_on_surface_converges():
    """On the surface (punctured rule) D[c] -> -c/2; low-order but decreasing in p."""
    c = np.array([1.0, 0.5, -0.25])
    errs = []
    for p in (16, 24, 32):
        X, n, w = G.sphere_surface(p, 1.0)
        u = oracle.dl(X, n, np.tile(c, (X.shape[0], 1)), w, X)
        errs.append(np.sqrt(np.mean(np.sum((u + c / 2) ** 2, 1))) / np.linalg.norm(c))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05


def test_double_layer_rigid_motion():
    """phi = a + omega x y gives D[phi](x) = -(a + omega x x) inside, 0 outside."""
    a = np.array([0.3, -0.4, 0.2])
    om = np.array([0.5, 0.1, -0.7])
    s = _cell(48, seed=4)
    phi = a + np.cross(om, s.pts)
    inside = interior_targets(s, 8)
    outside = s.centres[0] + np.array([[0, 0, 7.0], [8, 1, 0], [-3, -7, 2]])
    u = oracle.dl(s.pts, s.nrm, phi, s.w, np.concatenate([inside, outside]))
    np.testing.assert_allclose(u[:8], -(a + np.cross(om, inside)), atol=1e-8)
    np.testing.assert_allclose(u[8:], 0.0, atol=1e-8)


def _random_cloud(n, seed):
    rng = rng_for(seed)
    return rng.uniform(-2, 2, (n, 3)), rng


def test_single_layer_symmetry():
    """The Stokeslet is symmetric: <g, S f> = <f, S g> with unit weights."""
    y, rng = _random_cloud(60, 11)
    f, g = rng.uniform(-1, 1, (60, 3)), rng.uniform(-1, 1, (60, 3))
    w = np.ones(60)
    lhs = np.sum(g * oracle.sl(y, f, w, y, 1.3))
    rhs = np.sum(f * oracle.sl(y, g, w, y, 1.3))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_self_pair_and_coincident_points_skip():
    y = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.0, 0, 0]])
    f = np.array([[1.0, 2, 3], [1.0, 1, 1], [0.5, 0.5, 0.5]])
    u = oracle.sl(y, f, np.ones(3), y, 1.0)
    # point 1 sees point 0 only (point 2 is coincident): (1,2,3)/1 + (-1,0,0)*(-1)
    np.testing.assert_allclose(u[1] * 8 * np.pi, [2.0, 2.0, 3.0], rtol=1e-15)
    assert np.all(np.isfinite(u))


def test_translation_rotation_linearity():
    y, rng = _random_cloud(50, 12)
    x = rng.uniform(-3, 3, (20, 3))
    f, phi = rng.uniform(-1, 1, (50, 3)), rng.uniform(-1, 1, (50, 3))
    n = rng.normal(size=(50, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    w = rng.uniform(0.5, 1.5, 50)
    base = oracle.sldl(y, f, n, phi, w, x, 0.9)
    sh = np.array([10.0, -7.0, 3.0])
    np.testing.assert_allclose(oracle.sldl(y + sh, f, n, phi, w, x + sh, 0.9), base,
                               rtol=1e-12, atol=1e-12 * np.abs(base).max())
    Q = G.random_rotation(rng)
    rot = oracle.sldl(y @ Q.T, f @ Q.T, n @ Q.T, phi @ Q.T, w, x @ Q.T, 0.9)
    np.testing.assert_allclose(rot, base @ Q.T, rtol=1e-12, atol=1e-12 * np.abs(base).max())
    two = oracle.sldl(y, 2 * f, n, -3 * phi, w, x, 0.9)
    ref = 2 * oracle.sl(y, f, w, x, 0.9) - 3 * oracle.dl(y, n, phi, w, x)
    np.testing.assert_allclose(two, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _small_tree_case(seed=21, ncell=6, leaf=64):
    rng = rng_for(seed)
    s = random_cells_in_box(rng, ncell, 22.0, 8)
    tree = build_octree(s.pts, leaf)
    P = tree.perm
    f, phi = rng.uniform(-1, 1, (s.n, 3)), rng.uniform(-1, 1, (s.n, 3))
    return s.pts[P], s.nrm[P], s.w[P], f, phi, tree


def test_p2p_restriction_matches_direct_sum_over_ulist():
    pts, nrm, w, f, phi, tree = _small_tree_case()
    assert tree.nleaf > 8
    u = oracle.p2p(pts, f, phi, nrm, w, tree.leaf_ptr, tree.ulist_ptr, tree.ulist_idx, 3, 1.1)
    rng = rng_for(1)
    for b in rng.choice(tree.nleaf, 6, replace=False):
        src = np.concatenate([np.arange(tree.leaf_ptr[a], tree.leaf_ptr[a + 1])
                              for a in tree.ulist_idx[tree.ulist_ptr[b]:tree.ulist_ptr[b + 1]]])
        tg = np.arange(tree.leaf_ptr[b], tree.leaf_ptr[b + 1])
        ref = oracle.sldl(pts[src], f[src], nrm[src], phi[src], w[src], pts[tg], 1.1)
        np.testing.assert_allclose(u[tg], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    # kernel selection: SL only and DL only add up to both
    usl = oracle.p2p(pts, f, phi, nrm, w, tree.leaf_ptr, tree.ulist_ptr, tree.ulist_idx, 1, 1.1)
    udl = oracle.p2p(pts, f, phi, nrm, w, tree.leaf_ptr, tree.ulist_ptr, tree.ulist_idx, 2, 1.1)
    np.testing.assert_allclose(usl + udl, u, rtol=1e-12, atol=1e-12 * np.abs(u).max())


def test_p2p_single_leaf_and_full_lists_equal_direct():
    pts, nrm, w, f, phi, tree = _small_tree_case(seed=22, ncell=3)
    n = pts.shape[0]
    direct = oracle.sldl(pts, f, nrm, phi, w, pts, 1.0)
    one = oracle.p2p(pts, f, phi, nrm, w, np.array([0, n]), np.array([0, 1]), np.array([0]), 3)
    np.testing.assert_allclose(one, direct, rtol=1e-13, atol=1e-13 * np.abs(direct).max())
    L = tree.nleaf
    full_ptr = np.arange(L + 1) * L
    full_idx = np.tile(np.arange(L), L)
    allu = oracle.p2p(pts, f, phi, nrm, w, tree.leaf_ptr, full_ptr, full_idx, 3)
    np.testing.assert_allclose(allu, direct, rtol=1e-12, atol=1e-12 * np.abs(direct).max())


def test_batched_is_sl_on_cells_plus_dl_on_wall():
    rng = rng_for(31)
    s = random_cells_in_box(rng, 2, 16.0, 8)
    wp, wn, ww, wh = G.cylinder_wall_patches(9.0, 10.0, 4, 1, q=4)
    pts = np.concatenate([s.pts, wp, s.pts + 50.0])
    nrm = np.concatenate([s.nrm, wn, s.nrm])
    w = np.concatenate([s.w, ww, s.w])
    n = pts.shape[0]
    f, phi = rng.uniform(-1, 1, (n, 3)), rng.uniform(-1, 1, (n, 3))
    ptr = np.array([0, s.n + wp.shape[0], n])
    ncl = np.array([s.n, s.n])
    u = oracle.batched(pts, f, phi, nrm, w, ptr, ncl, 1.0)
    a, b, c = s.n, s.n + wp.shape[0], n
    ref0 = oracle.sl(pts[:a], f[:a], w[:a], pts[:b], 1.0) + \
        oracle.dl(pts[a:b], nrm[a:b], phi[a:b], w[a:b], pts[:b])
    ref1 = oracle.sl(pts[b:], f[b:], w[b:], pts[b:], 1.0)
    np.testing.assert_allclose(u[:b], ref0, rtol=1e-13, atol=1e-13 * np.abs(ref0).max())
    np.testing.assert_allclose(u[b:], ref1, rtol=1e-13, atol=1e-13 * np.abs(ref1).max())
