"""Checks of the synthetic input generators (no GPU, no oracle)."""
import numpy as np
from scipy.spatial import cKDTree

from synth import geometry as G
from synth import workloads as W


def _min_nonzero_distance(p):
    d, _ = cKDTree(p).query(p, k=2)
    d = d[:, 1]
    return d[d > 0].min()


def test_wall_patches_share_edges_exactly():
    P, N, Wt, H = G.cylinder_wall_patches(20.0, 30.0, 16, 4)
    assert _min_nonzero_distance(P) > 0.05
    assert abs(Wt.sum() - 2 * np.pi * 20.0 * 30.0) < 1e-9 * Wt.sum()
    np.testing.assert_allclose(np.linalg.norm(N, axis=1), 1.0)


def test_workload_points_have_no_near_duplicates():
    b = W.batched_workload(nsusp=3, max_cells=4)
    for a, e in zip(b.susp_ptr[:-1], b.susp_ptr[1:]):
        assert _min_nonzero_distance(b.pts[a:e]) > 0.01
    p = W.p2p_workload(ncell=20, radius=12.0, n_wall_patch=12, max_leaf=64)
    assert _min_nonzero_distance(p.pts) > 0.01


def test_rbc_quadrature_area_and_volume():
    for p in (12, 16, 24):
        X, n, w = G.rbc_surface(p)
        assert X.shape[0] == (p + 1) * 2 * p
        assert abs(w.sum() - 134.09) < 0.05
        assert abs((w * (X * n).sum(1)).sum() / 3 - 94.10) < 0.05
