"""The octree/U-list input builder against brute force on its stated definition."""
import numpy as np

from synth.octree import build_octree
from synth.workloads import random_cells_in_box, rng_for


def test_leaves_partition_points_and_respect_capacity():
    rng = rng_for(51)
    s = random_cells_in_box(rng, 5, 20.0, 8)
    t = build_octree(s.pts, 48)
    sz = np.diff(t.leaf_ptr)
    assert sz.min() >= 1 and sz.max() <= 48 and t.leaf_ptr[-1] == s.n
    assert np.array_equal(np.sort(t.perm), np.arange(s.n))
    # every point lies in its leaf's half-open box
    P = s.pts[t.perm]
    scale = (1 << 21) / t.root_size
    ijk = np.floor((P - t.root_lo) * scale).astype(np.int64)
    for b in range(t.nleaf):
        sl = slice(t.leaf_ptr[b], t.leaf_ptr[b + 1])
        assert np.all(ijk[sl] >= t.leaf_lo[b]) and np.all(ijk[sl] < t.leaf_hi[b])


def test_ulist_is_closed_box_adjacency():
    rng = rng_for(52)
    s = random_cells_in_box(rng, 4, 18.0, 8)
    t = build_octree(s.pts, 40)
    L = t.nleaf
    for b in range(L):
        want = []
        for a in range(L):
            touch = all(t.leaf_lo[a][k] <= t.leaf_hi[b][k] and t.leaf_lo[b][k] <= t.leaf_hi[a][k]
                        for k in range(3))
            if touch:
                want.append(a)
        got = list(t.ulist_idx[t.ulist_ptr[b]:t.ulist_ptr[b + 1]])
        assert got == want
        assert b in got


def test_pair_count():
    rng = rng_for(53)
    s = random_cells_in_box(rng, 3, 16.0, 8)
    t = build_octree(s.pts, 32)
    sz = np.diff(t.leaf_ptr)
    brute = sum(int(sz[b]) * int(sz[a]) for b in range(t.nleaf)
                for a in t.ulist_idx[t.ulist_ptr[b]:t.ulist_ptr[b + 1]])
    assert t.pair_count() == brute
