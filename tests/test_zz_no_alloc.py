"""The no-allocation single-layer entry point against the workspace one and
the FP64 oracle.

stokes_sl_eval_noalloc serves callers that cannot allocate device memory
when they need a velocity (an application that owns every device allocation,
a real-time pipeline that forbids cudaMalloc after start-up); it evaluates
the same sum as stokes_sl_eval in a fixed device buffer of the library.  This
file is collected last so that a run stopping at the first failure has run
every other test; it also passes on its own in a fresh process.
"""
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


def _noalloc(A, src, f, w, h, trg, mu, precision, source_splits=0):
    import torch
    out = torch.empty((trg.shape[0], 3), dtype=torch.float64, device=src.device)
    o = A.make_opts(precision, source_splits=source_splits)
    s = A.lib().stokes_sl_eval_noalloc(A.ptr(src), A.ptr(f), A.ptr(w), A.ptr(h), src.shape[0],
                                       A.ptr(trg), trg.shape[0], float(mu), A.ptr(out),
                                       ctypes.byref(o), A.stream_ptr(src.device))
    A.check(s)
    return out


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-12)])
def test_noalloc_matches_workspace_entry_point_twice(lib, precision, tol):
    P, A = lib
    c = W.sl_direct_workload()
    rng = W.rng_for(77)
    src, f, w, h = cuda(c.src, c.f, c.w, c.h)
    trg, = cuda(c.trg + rng.normal(scale=0.2, size=c.trg.shape))
    f2, = cuda(rng.uniform(-1, 1, c.f.shape))
    for dens in (f, f2):  # two calls in a row share the fixed buffer
        want = P.sl(src, dens, w, trg, 0.8, h=h, precision=precision).cpu().numpy()
        got = _noalloc(A, src, dens, w, h, trg, 0.8, precision).cpu().numpy()
        assert rel_l2(got, want) <= tol, rel_l2(got, want)
        # and against the FP64 oracle directly
        ref = oracle.sl(c.src, dens.cpu().numpy(), c.w, trg.cpu().numpy(), 0.8)
        assert rel_l2(got, ref) <= tol, rel_l2(got, ref)
    # no bounded wait ran out in the fixed buffer's last call
    A.check(A.lib().stokes_device_status(None, 0))


def test_noalloc_largest_size_lowers_the_source_splits(lib):
    """ns = nt = 65,536 (the limit) in mixed precision with 1,024 source splits
    asked for: that workspace does not fit the fixed buffer, so the call lowers
    the splits until it does, and still matches the workspace entry point."""
    P, A = lib
    c = W.sl_direct_workload(ncell=121, box=90.0)
    m = 65536
    src, f, w, h = cuda(c.src[:m], c.f[:m], c.w[:m], c.h[:m])
    want = P.sl(src, f, w, None, 1.0, h=h, precision="mixed").cpu().numpy()
    got = _noalloc(A, src, f, w, h, src, 1.0, "mixed", source_splits=1024).cpu().numpy()
    assert rel_l2(got, want) <= 1e-6, rel_l2(got, want)
    pick = np.sort(W.rng_for(78).choice(m, 256, replace=False))
    ref = oracle.sl(c.src[:m], c.f[:m], c.w[:m], c.src[:m][pick], 1.0)
    assert rel_l2(got[pick], ref) <= 1e-6, rel_l2(got[pick], ref)
    A.check(A.lib().stokes_device_status(None, 0))


def test_noalloc_wait_expiry_is_visible_to_the_caller(lib):
    """A bounded device wait that runs out inside the fixed buffer is reported
    by stokes_device_status(NULL, 0); the next call clears it (forced expiry:
    no device fault is involved)."""
    import torch
    P, A = lib
    c = W.sl_direct_workload(ncell=2, box=20.0)
    src, f, w, h = cuda(c.src, c.f, c.w, c.h)
    L = A.lib()
    A.check(L.stokes_set_wait_policy(0, 1))
    try:
        _noalloc(A, src, f, w, h, src, 1.0, "mixed")
    finally:
        A.check(L.stokes_set_wait_policy(0, 0))
    torch.cuda.synchronize()
    assert L.stokes_device_status(None, 0) == A.STK_ETIMEOUT
    got = _noalloc(A, src, f, w, h, src, 1.0, "mixed").cpu().numpy()
    A.check(L.stokes_device_status(None, 0))
    ref = oracle.sl(c.src, c.f, c.w, c.src, 1.0)
    assert rel_l2(got, ref) <= 1e-6


def test_noalloc_rejects_sizes_beyond_the_buffer(lib):
    import torch
    P, A = lib
    x = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    wv = torch.ones(65537, dtype=torch.float64, device="cuda")
    o = A.make_opts()
    s = A.lib().stokes_sl_eval_noalloc(A.ptr(x), A.ptr(x), A.ptr(wv), None, 65537, A.ptr(x), 4,
                                       1.0, A.ptr(x), ctypes.byref(o), A.stream_ptr())
    assert s == A.STK_EUNSUPPORTED
    assert b"65536" in A.lib().stokes_last_error()
