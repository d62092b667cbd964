"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/stokesgpu.h, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1909_11085_gb300 import _abi as A
from paper_1909_11085_gb300 import build as B

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "stokesgpu.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return A.lib()


def declared_symbols():
    text = open(HDR).read()
    return sorted(set(re.findall(r"\b(stokes_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) <= set(A.EXPORTS) | set(syms)


def test_wait_policy_validated_on_host(L):
    assert L.stokes_set_wait_policy(-5, 0) == A.STK_EINVAL
    assert L.stokes_set_wait_policy(0, 3) == A.STK_EINVAL
    assert L.stokes_set_wait_policy(1000, 0) == A.STK_OK
    assert L.stokes_set_wait_policy(0, 0) == A.STK_OK


def test_default_opts(L):
    o = A.StkOpts()
    L.stokes_default_opts(ctypes.byref(o))
    assert o.precision == A.STK_MIXED and o.near_ratio == 1.0 and o.accumulate == 0


def test_invalid_arguments_rejected_on_host(L):
    o = A.make_opts()
    nb = ctypes.c_size_t(0)
    assert L.stokes_direct_workspace_size(-1, 4, 1, ctypes.byref(o), ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_direct_workspace_size(4, 4, 7, ctypes.byref(o), ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_direct_workspace_size(4, 4, 1, None, ctypes.byref(nb)) == A.STK_EINVAL
    bad = A.make_opts(near_ratio=-1.0)
    assert L.stokes_direct_workspace_size(4, 4, 1, ctypes.byref(bad), ctypes.byref(nb)) == A.STK_EINVAL
    bad = A.make_opts()
    bad.precision = 9
    assert L.stokes_p2p_workspace_size(4, 1, 3, ctypes.byref(bad), ctypes.byref(nb)) == A.STK_EINVAL
    # NULL density with a non-empty problem
    s = L.stokes_sl_eval(ctypes.c_void_p(16), None, ctypes.c_void_p(16), None, 4, ctypes.c_void_p(16),
                         4, 1.0, ctypes.c_void_p(16), ctypes.byref(o), ctypes.c_void_p(256), 1 << 20, None)
    assert s == A.STK_EINVAL
    assert b"f is NULL" in L.stokes_last_error()
    # non-positive viscosity
    s = L.stokes_sl_eval(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), None, 4,
                         ctypes.c_void_p(16), 4, 0.0, ctypes.c_void_p(16), ctypes.byref(o),
                         ctypes.c_void_p(256), 1 << 20, None)
    assert s == A.STK_EINVAL
    # empty problems are valid no-ops
    assert L.stokes_sl_eval(None, None, None, None, 0, None, 0, 1.0, None, ctypes.byref(o), None, 0,
                            None) == A.STK_OK
    assert L.stokes_p2p_leaflists(None, None, None, None, None, None, 0, None, 0, None, None, 0, 3,
                                  1.0, None, ctypes.byref(o), None, 0, None) == A.STK_OK


def test_tile_configs_validated_on_host(L):
    nb = ctypes.c_size_t(0)
    n_cfg = L.stokes_tile_config_count()
    assert n_cfg >= 2
    sizes = []
    for c in range(-1, n_cfg):
        o = A.make_opts(tile_config=c)
        assert L.stokes_p2p_workspace_size(10000, 50, 3, ctypes.byref(o), ctypes.byref(nb)) == A.STK_OK
        sizes.append(nb.value)
    assert min(sizes) > 0
    for c in (n_cfg, 99, -2):
        bad = A.make_opts(tile_config=c)
        assert L.stokes_p2p_workspace_size(4, 1, 3, ctypes.byref(bad), ctypes.byref(nb)) == A.STK_EINVAL
    # graph and tuning entry points check their handles before touching a device
    assert L.stokes_graph_launch(None, None) == A.STK_EINVAL
    assert L.stokes_graph_destroy(None) == A.STK_OK


def test_tuning_cache_roundtrip(tmp_path):
    from paper_1909_11085_gb300 import tuning
    path = str(tmp_path / "tiles.json")
    o = A.make_opts()
    k1 = tuning.key("p2p", o, 1_000_000, 4096, 3)
    k2 = tuning.key("p2p", o, 1_048_576, 4000, 3)   # same size class
    k3 = tuning.key("p2p", A.make_opts("fp64"), 1_000_000, 4096, 3)
    assert k1 == k2 and k1 != k3
    assert tuning.lookup(path, k1) is None
    tuning.store(path, k1, 2, 1.5)
    tuning.store(path, k3, 1, 9.0)
    assert tuning.lookup(path, k2) == 2 and tuning.lookup(path, k3) == 1
    assert tuning.lookup(None, k1) is None
    tuning.store(None, k1, 3, 0.1)  # disabled cache: no-op


def test_patch_surface_entry_points_validated_on_host(L):
    """The check-point, BIE and near-zone entry points reject bad sizes and
    options before any device work; the near-zone workspace grows with the
    targets (a list of them) and with the patches."""
    o = A.make_opts()
    nb = ctypes.c_size_t(0)
    assert L.stokes_checkpoint_workspace_size(0, 6, 10, 2, 10, 4, ctypes.byref(o), ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_checkpoint_workspace_size(2, 6, 10, 2, 10, 4, ctypes.byref(o), None) == A.STK_EINVAL
    assert L.stokes_bie_workspace_size(6, 10, 2, 4, None, ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_near_search_workspace_size(-1, 10, 0, ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_near_search_workspace_size(4, 1, 0, ctypes.byref(nb)) == A.STK_EUNSUPPORTED
    assert L.stokes_near_search_workspace_size(4, 10, -1, ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_near_search_workspace_size(4, 10, 1 << 31, ctypes.byref(nb)) == A.STK_EINVAL
    sizes = []
    for npatch, nt in ((4, 0), (4, 1000), (400, 1000)):
        assert L.stokes_near_search_workspace_size(npatch, 10, nt, ctypes.byref(nb)) == A.STK_OK
        sizes.append(nb.value)
    assert sizes[0] < sizes[1] < sizes[2]
    # no targets: nothing to do, whatever the pointers
    assert L.stokes_near_patch_search(None, 4, 10, None, 0, 1.0, None, None, None, None, None,
                                      None, 0, None) == A.STK_OK
    assert L.stokes_near_patch_search(None, 4, 10, None, 5, -1.0, None, None, None, None, None,
                                      None, 0, None) == A.STK_EINVAL


def test_fmm_far_entry_points_validated_on_host(L):
    """The far field's size query and its argument checks (tree shape, p,
    viscosity, operators, workspace) run on the host and fail before any
    device call; an empty point set is a no-op."""
    import numpy as np
    dptr = np.array([0, 1, 9], dtype=np.int32)  # a root and 8 children
    t = A.StkFmmTree()
    t.nbox, t.nleaf, t.max_depth = 9, 8, 1
    t.depth_ptr = dptr.ctypes.data
    for k in ("depth", "anchor", "parent", "child_ptr", "box_leaf", "leaf_box", "leaf_ptr",
              "v_ptr", "w_ptr", "x_ptr"):
        setattr(t, k, 16)  # never dereferenced on the host
    t.root_size = 1.0
    nb = ctypes.c_size_t(0)
    assert L.stokes_fmm_far_workspace_size(4, 1, 0, 0, 10, ctypes.byref(t), ctypes.byref(nb)) == A.STK_OK
    ns = 4 ** 3 - 2 ** 3
    assert nb.value >= 8 * (3 * ns + 9 * (3 + 4 + 3) * ns)
    assert L.stokes_fmm_far_workspace_size(13, 1, 0, 0, 10, ctypes.byref(t), ctypes.byref(nb)) == A.STK_EINVAL
    assert L.stokes_fmm_far_workspace_size(4, 1, 0, 0, 10, None, ctypes.byref(nb)) == A.STK_EINVAL
    bad = np.array([0, 2, 9], dtype=np.int32)
    t.depth_ptr = bad.ctypes.data
    t.max_depth = 2  # depth_ptr then ends at index 3, which is not nbox
    assert L.stokes_fmm_far_workspace_size(4, 1, 0, 0, 10, ctypes.byref(t), ctypes.byref(nb)) == A.STK_EINVAL
    t.depth_ptr, t.max_depth = dptr.ctypes.data, 1
    t.root_size = float("nan")
    assert L.stokes_fmm_far_workspace_size(4, 1, 0, 0, 10, ctypes.byref(t), ctypes.byref(nb)) == A.STK_EINVAL
    t.root_size = 1.0
    ws, x = ctypes.c_void_p(4096), ctypes.c_void_p(4096)

    def call(n=10, f=x, phi=None, nrm=None, mu=1.0, uc=None, dc=None, wsb=0, p=4, prec=0):
        return L.stokes_fmm_far_eval(x, f, phi, nrm, x, n, ctypes.byref(t), p, 1, uc, dc, None,
                                     prec, mu, x, 0, ws, wsb, None)

    assert call(n=0) == A.STK_OK
    assert call(n=-1) == A.STK_EINVAL
    assert call(f=None) == A.STK_EINVAL  # neither layer
    assert call(phi=x) == A.STK_EINVAL  # phi without normals
    assert call(mu=0.0) == A.STK_EINVAL
    assert call(p=1) == A.STK_EINVAL
    assert call(wsb=16) == A.STK_ENOMEM
    assert call(prec=7) == A.STK_EINVAL
    keep = np.array([0, 1, 2, 9], dtype=np.int32)
    t.max_depth, t.depth_ptr = 2, keep.ctypes.data
    assert call(wsb=1 << 30) == A.STK_EINVAL  # a far field without operators
    assert b"uc2e" in L.stokes_last_error()
