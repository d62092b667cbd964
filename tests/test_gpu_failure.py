"""The failure path of the mixed engine's bounded waits, taken without any
device fault: stokes_set_wait_policy(0, 1) makes the first chunk wait of every
work item report expiry although its copy completes normally.  The call must
then leave STK_ETIMEOUT in its workspace's error word (stokes_device_status),
the device must stay usable, and the next call without the flag must be
correct again."""
import ctypes

import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests._util import cuda, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    from paper_1909_11085_gb300 import _abi as A
    return P, A


@pytest.fixture(scope="module")
def small():
    return W.p2p_workload(ncell=24, radius=12.0, n_wall_patch=12, max_leaf=64)


def _expect_timeout(A, status_call):
    with pytest.raises(A.StokesError) as e:
        status_call()
    assert e.value.status == A.STK_ETIMEOUT


def test_forced_expiry_reports_timeout_then_next_call_is_correct(lib, small):
    import torch
    P, A = lib
    c, t = small, small.tree
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = P.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    L = A.lib()
    A.check(L.stokes_set_wait_policy(0, 1))
    try:
        plan(pts, f, phi, nrm, w, h, 1.0)
    finally:
        A.check(L.stokes_set_wait_policy(0, 0))
    torch.cuda.synchronize()
    _expect_timeout(A, plan.device_status)
    plan.device_status()  # the read cleared the word
    u = plan(pts, f, phi, nrm, w, h, 1.0).cpu().numpy()
    plan.device_status()
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, 1.0)
    assert rel_l2(u, ref) <= 1e-6


def test_forced_expiry_on_the_direct_sum(lib):
    import torch
    P, A = lib
    d = W.sl_direct_workload(ncell=3, box=20.0)
    src, f, w, h = cuda(d.src, d.f, d.w, d.h)
    n = d.src.shape[0]
    # the work-item engine (named tile shape): the small one-launch form has no waits
    o = A.make_opts("mixed", tile_config=0)
    nb = ctypes.c_size_t(0)
    L = A.lib()
    A.check(L.stokes_direct_workspace_size(n, n, 1, ctypes.byref(o), ctypes.byref(nb)))
    ws = A.workspace(nb.value, src.device)
    out = torch.empty((n, 3), dtype=torch.float64, device=src.device)
    call = lambda: A.check(L.stokes_sl_eval(A.ptr(src), A.ptr(f), A.ptr(w), A.ptr(h), n, A.ptr(src),
                                            n, 1.0, A.ptr(out), ctypes.byref(o), A.ptr(ws),
                                            ws.numel(), A.stream_ptr(src.device)))
    A.check(L.stokes_set_wait_policy(0, 1))
    try:
        call()
    finally:
        A.check(L.stokes_set_wait_policy(0, 0))
    torch.cuda.synchronize()
    _expect_timeout(A, lambda: A.check(L.stokes_device_status(A.ptr(ws), ws.numel())))
    call()
    torch.cuda.synchronize()
    A.check(L.stokes_device_status(A.ptr(ws), ws.numel()))
    ref = oracle.sl(d.src, d.f, d.w, d.src, 1.0)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-6


def test_wait_policy_arguments_checked(lib):
    P, A = lib
    L = A.lib()
    assert L.stokes_set_wait_policy(-1, 0) == A.STK_EINVAL
    assert L.stokes_set_wait_policy(0, 2) == A.STK_EINVAL
    A.check(L.stokes_set_wait_policy(0, 0))


def test_small_direct_form_has_no_waits(lib):
    """With the default options a small mixed direct sum runs as one launch
    without device waits: a forced expiry leaves its status word at 0 and the
    result at the oracle's."""
    import torch
    P, A = lib
    d = W.sl_direct_workload(ncell=3, box=20.0)
    src, f, w, h = cuda(d.src, d.f, d.w, d.h)
    n = d.src.shape[0]
    o = A.make_opts("mixed")
    nb = ctypes.c_size_t(0)
    L = A.lib()
    A.check(L.stokes_direct_workspace_size(n, n, 1, ctypes.byref(o), ctypes.byref(nb)))
    ws = A.workspace(nb.value, src.device)
    out = torch.empty((n, 3), dtype=torch.float64, device=src.device)
    A.check(L.stokes_set_wait_policy(0, 1))
    try:
        A.check(L.stokes_sl_eval(A.ptr(src), A.ptr(f), A.ptr(w), A.ptr(h), n, A.ptr(src), n, 1.0,
                                 A.ptr(out), ctypes.byref(o), A.ptr(ws), ws.numel(),
                                 A.stream_ptr(src.device)))
    finally:
        A.check(L.stokes_set_wait_policy(0, 0))
    torch.cuda.synchronize()
    A.check(L.stokes_device_status(A.ptr(ws), ws.numel()))
    ref = oracle.sl(d.src, d.f, d.w, d.src, 1.0)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
