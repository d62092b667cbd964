"""GPU parity of the FMM near field (P2P over octree U-lists) against the oracle."""
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
    # 60 cells + wall in a thin cylinder, leaves of <= 96 points (many ragged leaves)
    return W.p2p_workload(ncell=60, radius=14.0, n_wall_patch=24, max_leaf=96)


@pytest.mark.parametrize("kernels", [1, 2, 3])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_p2p_small_all_targets(lib, small, kernels, precision, tol):
    c, t = small, small.tree
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, kernels,
                     0.9)
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    u = lib.p2p(pts, f, phi, nrm, w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, kernels, 0.9, h=h,
                precision=precision).cpu().numpy()
    assert rel_l2(u, ref) <= tol, rel_l2(u, ref)


def test_p2p_single_leaf_is_direct_sum(lib, small):
    c = small
    n = c.pts.shape[0]
    ref = oracle.sldl(c.pts, c.f, c.nrm, c.phi, c.w, c.pts, 1.0)
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    u = lib.p2p(pts, f, phi, nrm, w, [0, n], [0, 1], [0], 3, 1.0, h=h).cpu().numpy()
    assert rel_l2(u, ref) <= 1e-6


def test_p2p_repeat_is_deterministic(lib, small):
    import torch
    c, t = small, small.tree
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    a = plan(pts, f, phi, nrm, w, h).clone()
    b = plan(pts, f, phi, nrm, w, h)
    assert torch.equal(a, b)
    plan.device_status()


def test_p2p_caller_streams_graph_and_accumulate(lib, small):
    """The packing runs on a second stream of the library's, forked from the
    caller's stream and joined back before the engine.  Calls on two caller
    streams issued back to back without synchronising, and a captured graph of
    the call, give the same bits as a plain call; the accumulating form (which
    keeps the finish kernel, the plain one writes out directly) adds onto out."""
    import torch
    c, t = small, small.tree
    n = c.pts.shape[0]
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan_a = lib.P2PPlan(n, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    plan_b = lib.P2PPlan(n, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    ref = plan_a(pts, f, phi, nrm, w, h).clone()
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for k in range(6):
        st, plan = (s1, plan_a) if k % 2 == 0 else (s2, plan_b)
        with torch.cuda.stream(st):
            o = torch.empty_like(ref)
            plan(pts, f, phi, nrm, w, h, out=o)
            outs.append(o)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    g = plan_a.capture(pts, f, phi, nrm, w, h)
    g.out.zero_()
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(g.out, ref)
    base = torch.full_like(ref, 0.25)
    acc = plan_b(pts, f, phi, nrm, w, h, out=base.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert torch.allclose(acc - base, ref, rtol=0, atol=1e-12 * float(ref.abs().max()))
    plan_a.device_status()
    plan_b.device_status()
    exact = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, 1.0)
    assert rel_l2(ref.cpu().numpy(), exact) <= 1e-6


@pytest.fixture(scope="module")
def full():
    return W.p2p_workload()


def test_p2p_full_size_sampled(lib, full):
    """1,048,928 points, leaves <= 256, SL + DL: 2,000 sampled targets against the oracle."""
    c, t = full, full.tree
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    u = plan(pts, f, phi, nrm, w, h, 1.0).cpu().numpy()
    plan.device_status()
    rng = W.rng_for(10)
    pick = np.sort(rng.choice(c.pts.shape[0], 2000, replace=False))
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, 1.0,
                     targets=pick)
    assert rel_l2(u[pick], ref) <= 1e-6, rel_l2(u[pick], ref)
    plan64 = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, precision="fp64")
    u64 = plan64(pts, f, phi, nrm, w, h, 1.0).cpu().numpy()
    assert rel_l2(u64[pick], ref) <= 1e-12
