"""GPU near-zone search (Sec. 3.2) against the brute-force oracle on small
surfaces, and against the closed-form closest point (radial projection) on the
320-patch vessel wall with many targets."""
import numpy as np
import pytest

from oracle import nearzone as NZ
from synth import geometry as G
from tests._util import cuda

pytestmark = pytest.mark.gpu
Q = 10


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    return P


def _compare(lib, nodes, npatch, x, d_eps):
    ref_p, ref_uv, ref_y, ref_n, ref_d = NZ.near_patch_search(nodes, npatch, Q, x, d_eps)
    N, X = cuda(nodes, x)
    p, uv, y, n, d = (t.cpu().numpy() for t in lib.near_patch_search(N, npatch, X, d_eps, Q))
    np.testing.assert_array_equal(p >= 0, ref_p >= 0)
    hit = ref_p >= 0
    np.testing.assert_allclose(d[hit], ref_d[hit], rtol=0, atol=1e-9)
    np.testing.assert_allclose(y[hit], ref_y[hit], rtol=0, atol=1e-8)
    np.testing.assert_allclose(n[hit], ref_n[hit], rtol=0, atol=1e-7)
    # the patch is unique away from patch edges; where two tie, both are valid
    same = p[hit] == ref_p[hit]
    assert same.mean() > 0.9
    assert (d[~hit] == -1).all() and (p[~hit] == -1).all()


def test_wall_matches_oracle(lib):
    Rw, Lw, nth, nz = 6.0, 8.0, 6, 2
    cp, cn, cw, ch = G.cylinder_wall_patches(Rw, Lw, nth, nz, Q)
    rng = np.random.default_rng(8)
    th = rng.uniform(0, 2 * np.pi, 16)
    rho = Rw + rng.uniform(-1.5, 0.6, 16)
    z = rng.uniform(0.5, Lw - 0.5, 16)
    x = np.stack([rho * np.cos(th), rho * np.sin(th), z], axis=1)
    _compare(lib, cp, nth * nz, x, 1.0)


def test_sphere_matches_oracle(lib):
    a = 1.2
    cp, cn, cw, ch = G.cubed_sphere_patches(a, Q, 1)
    rng = np.random.default_rng(9)
    d = rng.normal(size=(16, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    x = d * (a + rng.uniform(-0.4, 0.4, 16))[:, None]
    _compare(lib, cp, 6, x, 0.3)


def test_vessel_wall_radial_projection_and_edges(lib):
    import torch
    from synth import workloads as W
    c = W.checkpoint_wall_workload()
    R, L = 50.0, 74.0
    rng = np.random.default_rng(10)
    m = 20000
    th = rng.uniform(0, 2 * np.pi, m)
    z = rng.uniform(0.3, L - 0.3, m)
    delta = rng.uniform(0.0, 3.0, m)
    x = np.stack([(R - delta) * np.cos(th), (R - delta) * np.sin(th), z], axis=1)
    N, X = cuda(c.pts, x)
    p, uv, y, n, d = (t.cpu().numpy() for t in lib.near_patch_search(N, c.npatch, X, 2.0, Q))
    near = delta <= 2.0 - 1e-9
    assert (p[near] >= 0).all() and (p[delta > 2.0 + 1e-9] == -1).all()
    yref = np.stack([R * np.cos(th), R * np.sin(th), z], axis=1)
    np.testing.assert_allclose(d[near], delta[near], atol=1e-7)
    np.testing.assert_allclose(y[near], yref[near], atol=1e-7)
    np.testing.assert_allclose(n[near], np.stack([np.cos(th), np.sin(th), 0 * th], 1)[near],
                               atol=1e-6)
    # no targets; no surface
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    assert lib.near_patch_search(N, c.npatch, e, 2.0, Q)[0].numel() == 0
    p0 = lib.near_patch_search(N[:0], 0, X[:5], 2.0, Q)[0].cpu().numpy()
    assert (p0 == -1).all()


def test_targets_on_nodes_and_edges(lib):
    """A target on a node is its own closest point at distance 0, also for
    d_eps = 0; on a node shared by neighbouring patches the lower patch index
    wins (Sec. 3.2 step e, ties to the lower index); targets outside the grid
    of patch boxes get none."""
    Rw, Lw, nth, nz = 6.0, 8.0, 6, 2
    cp, cn, cw, ch = G.cylinder_wall_patches(Rw, Lw, nth, nz, Q)
    npatch = nth * nz
    n1 = Q + 1
    nodes = cp.reshape(npatch, n1 * n1, 3)
    rng = np.random.default_rng(12)
    pick = rng.choice(npatch * n1 * n1, 40, replace=False)
    x = cp[pick]
    far = np.array([[100.0, 0.0, 0.0], [0.0, 0.0, -50.0], [0.0, 0.0, 4.0]])  # the last: the axis
    N, X = cuda(cp, np.concatenate([x, far]))
    for d_eps in (0.0, 0.5):
        p, uv, y, n, d = (t.cpu().numpy() for t in lib.near_patch_search(N, npatch, X, d_eps, Q))
        np.testing.assert_array_equal(d[:40], 0.0)
        np.testing.assert_array_equal(y[:40], x)
        # lowest patch that holds the point as a node
        for i, j in enumerate(pick):
            owners = [q for q in range(npatch) if np.any(np.all(nodes[q] == cp[j], axis=1))]
            assert p[i] == min(owners), (i, p[i], owners)
        assert (p[40:] == -1).all() and (d[40:] == -1.0).all()
        np.testing.assert_allclose(np.linalg.norm(n[:40], axis=1), 1.0, atol=1e-12)
