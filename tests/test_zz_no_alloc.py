"""The no-allocation single-layer entry point against the workspace one.

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


def _noalloc(A, src, f, w, h, trg, mu, precision):
    import torch
    out = torch.empty((trg.shape[0], 3), dtype=torch.float64, device=src.device)
    o = A.make_opts(precision)
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
