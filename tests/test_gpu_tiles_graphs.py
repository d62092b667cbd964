"""Every work-item shape (tile configuration) against the oracle; the
autotuners; CUDA-graph replay of the P2P and batched calls against a direct
call on the same inputs."""
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
def p2p_case():
    c = W.p2p_workload(ncell=60, radius=14.0, n_wall_patch=24, max_leaf=96)
    t = c.tree
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, 1.0)
    return c, ref


@pytest.fixture(scope="module")
def batched_case():
    c = W.batched_workload(nsusp=12, max_cells=6)
    ref = oracle.batched(c.pts, c.f, c.phi, c.nrm, c.w, c.susp_ptr, c.n_cell, 1.0)
    return c, ref


def _ncfg(lib):
    from paper_1909_11085_gb300 import _abi as A
    return A.lib().stokes_tile_config_count()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_p2p_every_tile_config(lib, p2p_case, precision, tol):
    c, ref = p2p_case
    t = c.tree
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, precision=precision)
    for cfg in range(_ncfg(lib)):
        plan.opts.tile_config = cfg
        u = plan(pts, f, phi, nrm, w, h, 1.0).cpu().numpy()
        plan.device_status()
        assert rel_l2(u, ref) <= tol, (cfg, rel_l2(u, ref))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_batched_every_tile_config(lib, batched_case, precision, tol):
    c, ref = batched_case
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.BatchedPlan(c.pts.shape[0], c.susp_ptr, c.n_cell, precision=precision)
    for cfg in range(_ncfg(lib)):
        plan.opts.tile_config = cfg
        u = plan(pts, f, phi, nrm, w, h, 1.0).cpu().numpy()
        plan.device_status()
        assert rel_l2(u, ref) <= tol, (cfg, rel_l2(u, ref))


def test_direct_every_tile_config(lib):
    import ctypes
    import torch
    from paper_1909_11085_gb300 import _abi as A
    rng = W.rng_for(77)
    ns, nt = 3001, 1777
    src = rng.standard_normal((ns, 3)) * 3.0
    trg = rng.standard_normal((nt, 3)) * 3.0
    f = rng.standard_normal((ns, 3))
    wts = rng.uniform(0.5, 1.5, ns)
    ref = oracle.sl(src, f, wts, trg, 1.0)
    s, fd, wd, td = cuda(src, f, wts, trg)
    for cfg in range(_ncfg(lib)):
        out = torch.zeros((nt, 3), dtype=torch.float64, device="cuda")
        o = A.make_opts(tile_config=cfg)
        nb = ctypes.c_size_t(0)
        A.check(A.lib().stokes_direct_workspace_size(ns, nt, 1, ctypes.byref(o), ctypes.byref(nb)))
        ws = A.workspace(nb.value, "cuda")
        A.check(A.lib().stokes_sl_eval(A.ptr(s), A.ptr(fd), A.ptr(wd), None, ns, A.ptr(td), nt,
                                       1.0, A.ptr(out), ctypes.byref(o), A.ptr(ws), ws.numel(),
                                       A.stream_ptr()))
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) <= 1e-6, cfg


def test_p2p_autotune_and_cache(lib, p2p_case, tmp_path):
    c, ref = p2p_case
    t = c.tree
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    cache = str(tmp_path / "tiles.json")
    best = plan.autotune(pts, f, phi, nrm, w, h, cache=cache)
    assert 0 <= best < _ncfg(lib) and plan.opts.tile_config == best
    plan2 = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3)
    assert plan2.autotune(pts, f, phi, nrm, w, h, cache=cache) == best  # from the cache
    u = plan(pts, f, phi, nrm, w, h).cpu().numpy()
    assert rel_l2(u, ref) <= 1e-6


def test_batched_autotune(lib, batched_case):
    c, ref = batched_case
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.BatchedPlan(c.pts.shape[0], c.susp_ptr, c.n_cell)
    best = plan.autotune(pts, f, phi, nrm, w, h)
    assert 0 <= best < _ncfg(lib)
    u = plan(pts, f, phi, nrm, w, h).cpu().numpy()
    assert rel_l2(u, ref) <= 1e-6


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_p2p_graph_replay_matches_direct_call(lib, p2p_case, precision):
    import torch
    c, ref = p2p_case
    t = c.tree
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.P2PPlan(c.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, precision=precision)
    g = plan.capture(pts, f, phi, nrm, w, h)
    u1 = g.launch().clone()
    torch.cuda.synchronize()
    plan.device_status()
    direct = plan(pts, f, phi, nrm, w, h)
    assert torch.equal(u1, direct)
    # new densities written in place are seen by the next replay
    f.mul_(-2.0)
    phi.mul_(0.5)
    u2 = g.launch()
    torch.cuda.synchronize()
    direct2 = plan(pts, f, phi, nrm, w, h)
    assert torch.equal(u2, direct2)
    ref2 = oracle.p2p(c.pts, -2.0 * c.f, 0.5 * c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr,
                      t.ulist_idx, 3, 1.0)
    tol = 1e-6 if precision == "mixed" else 1e-12
    assert rel_l2(u2.cpu().numpy(), ref2) <= tol
    del g


def test_batched_graph_replay_matches_direct_call(lib, batched_case):
    import torch
    c, ref = batched_case
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.BatchedPlan(c.pts.shape[0], c.susp_ptr, c.n_cell)
    g = plan.capture(pts, f, phi, nrm, w, h)
    for _ in range(3):
        u = g.launch()
    torch.cuda.synchronize()
    plan.device_status()
    direct = plan(pts, f, phi, nrm, w, h)
    assert torch.equal(u, direct)
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-6
    # moved points (a time step) are picked up by the replay
    pts.add_(0.01)
    u2 = g.launch().clone()
    torch.cuda.synchronize()
    assert torch.equal(u2, plan(pts, f, phi, nrm, w, h))


@pytest.mark.parametrize("kernels", [1, 2, 3])
@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-12)])
def test_direct_graph_replay(lib, kernels, precision, tol):
    """DirectPlan: a captured direct sum replays bit-identically to a direct
    call on the same buffers, follows densities rewritten in place, and matches
    the oracle (targets = sources, the 4,352-point single-layer workload's
    geometry)."""
    import torch
    c = W.sl_direct_workload()
    rng = W.rng_for(41)
    phi_np, nrm_np = rng.uniform(-1, 1, c.f.shape), c.nrm
    src, f, w, h, nrm, phi = cuda(c.src, c.f, c.w, c.h, nrm_np, phi_np)
    n = c.src.shape[0]
    plan = lib.DirectPlan(n, n, kernels, precision)
    want = plan(src, f, nrm, phi, w, None, 0.9, h).clone()
    out = torch.empty_like(want)
    g = plan.capture(src, f, nrm, phi, w, None, 0.9, h, out)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    if kernels & 1:
        ref = oracle.sl(c.src, c.f, c.w, c.src, 0.9)
    else:
        ref = np.zeros_like(c.src)
    if kernels & 2:
        ref = ref + oracle.dl(c.src, nrm_np, phi_np, c.w, c.src)
    assert rel_l2(out.cpu().numpy(), ref) <= tol, rel_l2(out.cpu().numpy(), ref)
    f.mul_(2.0)
    phi.mul_(2.0)
    g.launch()
    torch.cuda.synchronize()
    plan.device_status()
    np.testing.assert_allclose(out.cpu().numpy(), 2 * want.cpu().numpy(), rtol=1e-12,
                               atol=1e-12 * float(want.abs().max()))
