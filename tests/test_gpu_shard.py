"""Each rank's part of a sharded evaluation is an ordinary single-GPU call on
the local arrays.  Here the parts of a 3-way partition run one after another
on one GPU (no collective, no kernel waits on another) and are assembled on
the host; the result must match the unsharded call and the oracle."""
import numpy as np
import pytest

import oracle
from paper_1909_11085_gb300 import shard as S
from synth import workloads as W
from tests._util import cuda, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    return P


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_p2p_shards_assemble_to_full_result(lib, precision, tol):
    c = W.p2p_workload(ncell=60, radius=14.0, n_wall_patch=24, max_leaf=96)
    t = c.tree
    n = c.pts.shape[0]
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, 1.0)
    full = np.zeros((n, 3))
    world = 3
    for r in range(world):
        sh = S.shard_p2p(t.leaf_ptr, t.ulist_ptr, t.ulist_idx, world, r)
        rows = sh.rows
        pts, f, phi, nrm, w, h = cuda(c.pts[rows], c.f[rows], c.phi[rows], c.nrm[rows], c.w[rows],
                                      c.h[rows])
        plan = lib.P2PPlan(sh.n_local, sh.leaf_ptr, sh.ulist_ptr, sh.ulist_idx, 3,
                           precision=precision)
        u = plan(pts, f, phi, nrm, w, h).cpu().numpy()
        plan.device_status()
        assert not np.any(u[sh.n_owned:])  # halo leaves are sources only
        full[rows[:sh.n_owned]] = u[:sh.n_owned]
    assert rel_l2(full, ref) <= tol, rel_l2(full, ref)


def test_batched_shards_assemble_to_full_result(lib):
    b = W.batched_workload(nsusp=12, max_cells=6)
    ref = oracle.batched(b.pts, b.f, b.phi, b.nrm, b.w, b.susp_ptr, b.n_cell, 1.0)
    full = np.zeros_like(ref)
    for r in range(2):
        bs = S.shard_batched(b.susp_ptr, b.n_cell, 2, r)
        rows = bs.rows
        pts, f, phi, nrm, w, h = cuda(b.pts[rows], b.f[rows], b.phi[rows], b.nrm[rows], b.w[rows],
                                      b.h[rows])
        u = lib.batched(pts, f, phi, nrm, w, bs.susp_ptr, bs.n_cell, 1.0, h=h).cpu().numpy()
        full[rows] = u
    assert rel_l2(full, ref) <= 1e-6
