"""The library's FP64 <-> FP32 conversions on the integer pipe (used by the
packing, the hi/lo splits and the near pairs' FP64 difference and 1/|r|)
against CUDA's own conversions, bit for bit: round to nearest, ties to even,
over the whole FP64 exponent range, with ties, carries into the exponent,
the edges of the normal FP32 range, subnormal results, signed zeros,
infinities and NaN."""
import numpy as np
import pytest

from tests._util import cuda

pytestmark = pytest.mark.gpu


def _values():
    rng = np.random.default_rng(20191125)
    # random doubles over exponents -160 .. 160 (beyond both ends of FP32)
    m = rng.uniform(1.0, 2.0, 200_000)
    e = rng.integers(-160, 161, 200_000)
    s = rng.choice([-1.0, 1.0], 200_000)
    v = [s * np.ldexp(m, e)]
    # exact FP32 values, and those +- half an FP32 ulp (ties) and +- a little more
    f = rng.uniform(-1e6, 1e6, 50_000).astype(np.float32).astype(np.float64)
    ulp = np.abs(np.spacing(f.astype(np.float32))).astype(np.float64)
    for k in (0.0, 0.5, -0.5, 0.5 + 2.0 ** -20, 0.5 - 2.0 ** -20, 0.25, 0.75):
        v.append(f + k * ulp)
    # just below powers of two (the rounding carries into the exponent)
    p2 = np.ldexp(1.0, np.arange(-130, 130))
    v += [p2, p2 * (1 - 2.0 ** -25), p2 * (1 - 2.0 ** -24), p2 * (1 - 2.0 ** -30), -p2]
    fmax = float(np.finfo(np.float32).max)
    fmin = float(np.finfo(np.float32).tiny)
    v.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax,
                       fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), 2.0 ** 128,
                       fmin, fmin * (1 - 2.0 ** -30), fmin / 2, fmin * 2.0 ** -30,
                       5e-324, 1.7976931348623157e308]))
    return np.concatenate(v)


def test_conversions_match_cuda_bit_for_bit():
    import torch
    from paper_1909_11085_gb300 import build
    build.build()
    from paper_1909_11085_gb300 import _abi as A
    v = _values()
    n = v.shape[0]
    (x,) = cuda(v)
    no = torch.empty(n, dtype=torch.float32, device=x.device)
    nc = torch.empty_like(no)
    wo = torch.empty(n, dtype=torch.float64, device=x.device)
    wc = torch.empty_like(wo)
    A.check(A.lib().stokes_convert_check(A.ptr(x), n, A.ptr(no), A.ptr(nc), A.ptr(wo), A.ptr(wc),
                                         A.stream_ptr(x.device)))
    torch.cuda.synchronize()
    no, nc = no.cpu().numpy().view(np.uint32), nc.cpu().numpy().view(np.uint32)
    wo, wc = wo.cpu().numpy().view(np.uint64), wc.cpu().numpy().view(np.uint64)
    bad = np.nonzero(no != nc)[0]
    assert bad.size == 0, f"narrowing differs at {v[bad[:5]]}"
    bad = np.nonzero(wo != wc)[0]
    assert bad.size == 0, f"widening differs at {v[bad[:5]]}"
    # and CUDA's narrowing is numpy's IEEE rounding where both are defined
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32).view(np.uint32)
    fin = ~np.isnan(v)
    assert np.array_equal(nc[fin], ref[fin])


def test_convert_check_arguments():
    from paper_1909_11085_gb300 import build
    build.build()
    from paper_1909_11085_gb300 import _abi as A
    L = A.lib()
    assert L.stokes_convert_check(None, -1, None, None, None, None, None) == A.STK_EINVAL
    A.check(L.stokes_convert_check(None, 0, None, None, None, None, None))
    assert L.stokes_convert_check(None, 4, None, None, None, None, None) == A.STK_EINVAL
