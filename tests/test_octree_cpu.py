"""The library's host octree and interaction lists (stokes_octree_build)
against the input generator's (synth.octree), which follow the same
definitions box by box: identical permutation, leaves, U-lists, boxes and
V, W, X lists, down to depth-21 clusters and coincident points; and the
argument checks.  No GPU is needed."""
import ctypes

import numpy as np
import pytest

from paper_1909_11085_gb300 import _abi as A
from paper_1909_11085_gb300 import build as B
from paper_1909_11085_gb300 import ops
from synth import octree as O
from synth import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _clustered(rng):
    c = rng.uniform(0, 1, (2000, 3))
    c[:600] = 0.5 + 1e-7 * rng.normal(size=(600, 3))  # a cluster that splits to depth 21
    return c


CASES = {
    "uniform_shallow": (lambda rng: rng.uniform(0, 1, (300, 3)), 64),
    "heavy_tailed": (lambda rng: rng.normal(size=(5000, 3)) ** 3, 16),
    "cells_and_wall": (lambda rng: W.p2p_workload(ncell=12, radius=10.0, n_wall_patch=6,
                                                  max_leaf=16).pts, 16),
    "depth21_cluster": (_clustered, 8),
    "coincident": (lambda rng: np.zeros((40, 3)), 8),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_matches_the_generator(name):
    make, max_leaf = CASES[name]
    pts = make(np.random.default_rng(3))
    ref = O.build_octree(pts, max_leaf)
    fl = O.far_lists(ref)
    got = ops.octree(pts, max_leaf)
    pairs = [("perm", ref.perm), ("leaf_ptr", ref.leaf_ptr), ("ulist_ptr", ref.ulist_ptr),
             ("ulist_idx", ref.ulist_idx), ("root_lo", ref.root_lo), ("box_depth", fl.depth),
             ("box_anchor", fl.anchor), ("box_parent", fl.parent), ("box_leaf", fl.leaf),
             ("v_ptr", fl.v_ptr), ("v_idx", fl.v_idx), ("w_ptr", fl.w_ptr), ("w_idx", fl.w_idx),
             ("x_ptr", fl.x_ptr), ("x_idx", fl.x_idx)]
    for key, want in pairs:
        have = np.asarray(got[key])
        assert have.shape == np.asarray(want).shape and np.array_equal(have, want), key
    assert got["root_size"] == ref.root_size
    assert got["max_depth"] == int(fl.depth.max())
    # the far field's tree arrays accept it as they accept the generator's, and
    # derive the same colleague table the library exports
    t = ops.fmm_tree_arrays(**ops.fmm_tree_args(got))
    assert t["max_depth"] == got["max_depth"]
    np.testing.assert_array_equal(t["colleague"], got["colleague"])


def test_rejects_bad_arguments():
    L = A.lib()
    h = ctypes.c_void_p()
    pts = np.zeros((4, 3))
    assert L.stokes_octree_build(pts.ctypes.data, 0, 8, ctypes.byref(h)) == A.STK_EINVAL
    assert L.stokes_octree_build(pts.ctypes.data, 4, 0, ctypes.byref(h)) == A.STK_EINVAL
    assert L.stokes_octree_build(None, 4, 8, ctypes.byref(h)) == A.STK_EINVAL
    assert L.stokes_octree_build(pts.ctypes.data, 4, 8, None) == A.STK_EINVAL
    pts[2, 1] = np.nan
    assert L.stokes_octree_build(pts.ctypes.data, 4, 8, ctypes.byref(h)) == A.STK_EINVAL
    assert not h.value
    assert b"finite" in L.stokes_last_error()
    with pytest.raises(ValueError):
        ops.octree(np.zeros((5, 2)))


def test_fmm_plan_set_up_on_the_host():
    """FmmPlan builds the library's octree once and plans the near and far
    fields on it (host logic; a CPU device keeps every buffer on the host)."""
    import torch
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    rng = np.random.default_rng(9)
    shuffled = rng.permutation(wl.pts.shape[0])
    plan = ops.FmmPlan(wl.pts[shuffled], max_leaf=32, p=4, mu=wl.mu, device=torch.device("cpu"))
    assert np.array_equal(np.sort(plan.perm), np.arange(wl.pts.shape[0]))
    # the tree of the shuffled points, in leaf order, is the workload's tree
    assert np.array_equal(plan.tree["leaf_ptr"], wl.tree.leaf_ptr)
    assert np.array_equal(plan.tree["ulist_idx"], wl.tree.ulist_idx)
    assert plan.far.flux and plan.near.kernels == 3 and plan.near.nleaf == wl.tree.nleaf
    sl_only = ops.FmmPlan(wl.pts, max_leaf=32, kernels=1, device=torch.device("cpu"))
    assert not sl_only.far.flux
    with pytest.raises(ValueError):
        ops.FmmPlan(wl.pts, kernels=4, device=torch.device("cpu"))
