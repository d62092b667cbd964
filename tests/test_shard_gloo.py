"""Multi-rank partition of the sums (one GPU per rank in production), run as
world-size-2 gloo ranks on the CPU with the oracle as each rank's evaluator.
Checks that sharded evaluation plus gather reproduces the unsharded sums, and
the partition invariants (every target owned once, halos complete, LPT and
prefix balance)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1909_11085_gb300 import shard as S
from synth import workloads as W


def test_balanced_ranges_and_lpt():
    rng = np.random.default_rng(5)
    c = rng.exponential(size=1000)
    for world in (1, 2, 3, 8):
        b = S.balanced_ranges(c, world)
        assert b[0] == 0 and b[-1] == 1000 and (np.diff(b) >= 0).all()
        loads = [c[b[r]:b[r + 1]].sum() for r in range(world)]
        assert max(loads) - min(loads) <= 2 * c.max() + 1e-9
        parts = S.lpt_assign(c, world)
        allp = np.sort(np.concatenate(parts))
        assert (allp == np.arange(1000)).all()
        lp = [c[p].sum() for p in parts]
        # Graham's bound for LPT: max load <= (4/3 - 1/(3m)) * optimum <= that * mean-based bound
        assert max(lp) <= (4 / 3) * max(c.sum() / world, c.max()) + 1e-9
    assert list(S.balanced_ranges(np.zeros(4), 2)) == [0, 2, 4]
    lo, hi = S.direct_target_range(10, 3, 2)
    assert (lo, hi) == (7, 10)


def test_p2p_shard_invariants():
    c = W.p2p_workload(ncell=40, radius=12.0, n_wall_patch=16, max_leaf=64)
    t = c.tree
    n = c.pts.shape[0]
    owned = np.zeros(n, dtype=np.int64)
    for world in (2, 3):
        owned[:] = 0
        pairs = 0
        for r in range(world):
            sh = S.shard_p2p(t.leaf_ptr, t.ulist_ptr, t.ulist_idx, world, r)
            owned[sh.rows[:sh.n_owned]] += 1
            # local U-lists reach only local leaves, halo leaves are sources only
            nl = sh.leaf_ptr.shape[0] - 1
            assert (np.diff(sh.ulist_ptr)[sh.leaf_range[1] - sh.leaf_range[0]:] == 0).all()
            assert sh.ulist_idx.max(initial=0) < nl
            sz = np.diff(sh.leaf_ptr)
            pairs += int((sz[:sh.leaf_range[1] - sh.leaf_range[0]] *
                          np.array([sz[sh.ulist_idx[a:b]].sum() for a, b in
                                    zip(sh.ulist_ptr[:-1], sh.ulist_ptr[1:])])[:sh.leaf_range[1] -
                                                                               sh.leaf_range[0]]).sum())
        assert (owned == 1).all()
        assert pairs == c.pairs()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        # P2P: target leaves + halo
        c = W.p2p_workload(ncell=40, radius=12.0, n_wall_patch=16, max_leaf=64)
        t = c.tree
        sh = S.shard_p2p(t.leaf_ptr, t.ulist_ptr, t.ulist_idx, world, rank)
        r = sh.rows
        loc = oracle.p2p(c.pts[r], c.f[r], c.phi[r], c.nrm[r], c.w[r], sh.leaf_ptr, sh.ulist_ptr,
                         sh.ulist_idx, 3, 1.0, targets=np.arange(sh.n_owned))
        full = S.gather_rows(torch.as_tensor(loc), r[:sh.n_owned], c.pts.shape[0])
        res["p2p"] = full.numpy()
        # batched: whole suspensions by LPT
        b = W.batched_workload(nsusp=9, max_cells=4)
        bs = S.shard_batched(b.susp_ptr, b.n_cell, world, rank)
        r = bs.rows
        loc = (oracle.batched(b.pts[r], b.f[r], b.phi[r], b.nrm[r], b.w[r], bs.susp_ptr,
                              bs.n_cell, 1.0) if r.size else np.zeros((0, 3)))
        res["batched"] = S.gather_rows(torch.as_tensor(loc), r, b.pts.shape[0]).numpy()
        # direct: contiguous target ranges, sources replicated
        rng = W.rng_for(3)
        src, f, wts = rng.standard_normal((300, 3)), rng.standard_normal((300, 3)), np.ones(300)
        trg = rng.standard_normal((101, 3))
        lo, hi = S.direct_target_range(101, world, rank)
        loc = oracle.sl(src, f, wts, trg[lo:hi], 1.0)
        res["direct"] = S.gather_rows(torch.as_tensor(loc), np.arange(lo, hi), 101).numpy()
        if rank == 0:
            np.savez(out_path, **res)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reproduce_unsharded_sums(tmp_path):
    import torch.multiprocessing as mp
    oracle.build()
    out_path = str(tmp_path / "rank0.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), out_path), nprocs=2, join=True,
                       start_method="spawn")
    res = np.load(out_path)
    c = W.p2p_workload(ncell=40, radius=12.0, n_wall_patch=16, max_leaf=64)
    t = c.tree
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, 1.0)
    np.testing.assert_allclose(res["p2p"], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    b = W.batched_workload(nsusp=9, max_cells=4)
    refb = oracle.batched(b.pts, b.f, b.phi, b.nrm, b.w, b.susp_ptr, b.n_cell, 1.0)
    np.testing.assert_allclose(res["batched"], refb, rtol=0, atol=1e-13 * np.abs(refb).max())
    rng = W.rng_for(3)
    src, f, wts = rng.standard_normal((300, 3)), rng.standard_normal((300, 3)), np.ones(300)
    trg = rng.standard_normal((101, 3))
    np.testing.assert_array_equal(res["direct"], oracle.sl(src, f, wts, trg, 1.0))


def _sharded_main(rank, world, port, out_path):
    """The sharded near-field step as bench.py --shard runs it (ShardedP2P),
    with the oracle as each rank's evaluator on CPU tensors."""
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = W.p2p_workload(ncell=40, radius=12.0, n_wall_patch=16, max_leaf=64)
        t = c.tree

        def make_eval(sh):
            def ev(L):
                u = oracle.p2p(L["pts"].numpy(), L["f"].numpy(), L["phi"].numpy(),
                               L["nrm"].numpy(), L["w"].numpy(), sh.leaf_ptr, sh.ulist_ptr,
                               sh.ulist_idx, 3, c.mu)
                return torch.as_tensor(u)
            return ev

        sp = S.ShardedP2P(c.pts, c.f, c.phi, c.nrm, c.w, c.h, t.leaf_ptr, t.ulist_ptr,
                          t.ulist_idx, world, rank, make_eval, "cpu")
        full = sp.step()
        pairs = torch.tensor([sp.pairs], dtype=torch.int64)
        allp = [torch.zeros_like(pairs) for _ in range(world)]
        dist.all_gather(allp, pairs)
        if rank == 0:
            np.savez(out_path, full=full.numpy(), pairs=np.array([int(x) for x in allp]))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_sharded_step_as_the_bench_runs_it(tmp_path):
    """ShardedP2P with two gloo ranks: the assembled velocity equals the
    unsharded near field, the ranks' pair counts add up to the total and are
    within 5% of each other."""
    import torch.multiprocessing as mp
    oracle.build()
    out_path = str(tmp_path / "sharded.npz")
    mp.start_processes(_sharded_main, args=(2, _free_port(), out_path), nprocs=2, join=True,
                       start_method="spawn")
    res = np.load(out_path)
    c = W.p2p_workload(ncell=40, radius=12.0, n_wall_patch=16, max_leaf=64)
    t = c.tree
    ref = oracle.p2p(c.pts, c.f, c.phi, c.nrm, c.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, c.mu)
    np.testing.assert_allclose(res["full"], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    p = res["pairs"]
    assert p.sum() == c.pairs()
    assert p.max() <= 1.05 * p.min(), p
