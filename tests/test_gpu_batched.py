"""GPU parity of the batched suspensions (one persistent launch) against the oracle."""
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
    return P


@pytest.fixture(scope="module")
def small():
    return W.batched_workload(nsusp=12, max_cells=6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_batched_small_all_targets(lib, small, precision, tol):
    c = small
    ref = oracle.batched(c.pts, c.f, c.phi, c.nrm, c.w, c.susp_ptr, c.n_cell, 1.0)
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    u = lib.batched(pts, f, phi, nrm, w, c.susp_ptr, c.n_cell, 1.0, h=h,
                    precision=precision).cpu().numpy()
    per = [rel_l2(u[a:b], ref[a:b]) for a, b in zip(c.susp_ptr[:-1], c.susp_ptr[1:])]
    assert rel_l2(u, ref) <= tol and max(per) <= 10 * tol, (rel_l2(u, ref), max(per))
