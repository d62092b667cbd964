"""Partitioning of the layer-potential sums across ranks (one GPU per rank).

Every form of the sum splits into independent units with no exchange inside a
kernel, so a multi-GPU run is a partition, one independent evaluation per rank
and a gather of the rows each rank owns:

* direct sums (Eq. "sl_stokes", the double-layer kernel of Sec. 2.1): the
  targets are split into contiguous ranges, every rank holds all sources;
* batched suspensions (the superposition of Sec. 2.2, one suspension per
  unit): whole suspensions are assigned to ranks by longest-processing-time
  order of their pair counts;
* the FMM near field (P2P over U-lists, Sec. 3.1): the target leaves are split
  into contiguous ranges of the leaf order with balanced pair counts; each
  rank also receives the source leaves in its leaves' U-lists (a one-off
  halo), which it holds as leaves with empty U-lists so that they are sources
  only.

This module holds index bookkeeping only: which rows a rank reads and owns,
and the local CSR arrays in the local numbering.  The evaluation itself is an
ordinary single-GPU call on the local arrays.  `gather_rows` assembles the
owned rows of every rank with one torch.distributed all_gather (NCCL between
GPUs, gloo on CPU).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def balanced_ranges(costs, world: int):
    """Splits items 0..len(costs)-1 into `world` contiguous ranges whose cost
    sums are as even as a prefix split allows; returns world+1 boundaries."""
    costs = np.asarray(costs, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    n = costs.shape[0]
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    if total <= 0.0:
        return np.linspace(0, n, world + 1).round().astype(np.int64)
    goals = total * np.arange(1, world) / world
    cuts = np.searchsorted(cum, goals, side="left")
    # take the nearer of the two prefix sums around each goal
    lo = np.clip(cuts - 1, 0, n)
    pick = np.where(np.abs(cum[lo] - goals) <= np.abs(cum[np.clip(cuts, 0, n)] - goals), lo, cuts)
    bounds = np.concatenate([[0], np.clip(pick, 0, n), [n]]).astype(np.int64)
    return np.maximum.accumulate(bounds)


def lpt_assign(costs, world: int):
    """Longest-processing-time assignment: items in decreasing cost, each to the
    least-loaded rank (ties to the lower rank).  Returns one sorted index array
    per rank."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    owner = np.empty(costs.shape[0], dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return [np.flatnonzero(owner == r) for r in range(world)]


def direct_target_range(nt: int, world: int, rank: int):
    """Contiguous target range [lo, hi) of `rank` for a direct sum."""
    b = balanced_ranges(np.ones(int(nt)), world)
    return int(b[rank]), int(b[rank + 1])


@dataclass
class BatchedShard:
    """The suspensions a rank owns, in the local numbering.

    rows[k] is the global row of local point k; susp_ptr and n_cell describe
    the local suspensions exactly as the single-GPU batched call expects."""
    suspensions: np.ndarray
    rows: np.ndarray
    susp_ptr: np.ndarray
    n_cell: np.ndarray


def shard_batched(susp_ptr, n_cell, world: int, rank: int) -> BatchedShard:
    susp_ptr = np.asarray(susp_ptr, dtype=np.int64)
    n_cell = np.asarray(n_cell, dtype=np.int64)
    sizes = np.diff(susp_ptr)
    mine = lpt_assign(sizes.astype(np.float64) ** 2, world)[rank]
    rows = (np.concatenate([np.arange(susp_ptr[s], susp_ptr[s + 1]) for s in mine])
            if mine.size else np.zeros(0, dtype=np.int64))
    ptr = np.concatenate([[0], np.cumsum(sizes[mine])]).astype(np.int64)
    return BatchedShard(mine, rows.astype(np.int64), ptr, n_cell[mine].copy())


@dataclass
class P2PShard:
    """One rank's part of a P2P evaluation over U-lists.

    Local points are the owned leaves (targets, rows 0..n_owned-1) followed by
    the halo leaves (sources only).  rows[k] is the global row of local point
    k.  leaf_ptr / ulist_ptr / ulist_idx are the local CSR arrays: owned leaf i
    keeps its U-list renumbered, halo leaves have empty U-lists."""
    leaf_range: tuple
    rows: np.ndarray
    n_owned: int
    leaf_ptr: np.ndarray
    ulist_ptr: np.ndarray
    ulist_idx: np.ndarray
    halo_leaves: np.ndarray

    @property
    def n_local(self) -> int:
        return int(self.rows.shape[0])


def p2p_leaf_costs(leaf_ptr, ulist_ptr, ulist_idx):
    """Pairs of each target leaf B: |B| * sum over A in U(B) of |A|."""
    leaf_ptr = np.asarray(leaf_ptr, dtype=np.int64)
    ulist_ptr = np.asarray(ulist_ptr, dtype=np.int64)
    ulist_idx = np.asarray(ulist_idx, dtype=np.int64)
    size = np.diff(leaf_ptr)
    cs = np.concatenate([[0], np.cumsum(size[ulist_idx])])
    src = cs[ulist_ptr[1:]] - cs[ulist_ptr[:-1]]
    return size.astype(np.float64) * src.astype(np.float64)


def shard_p2p(leaf_ptr, ulist_ptr, ulist_idx, world: int, rank: int) -> P2PShard:
    leaf_ptr = np.asarray(leaf_ptr, dtype=np.int64)
    ulist_ptr = np.asarray(ulist_ptr, dtype=np.int64)
    ulist_idx = np.asarray(ulist_idx, dtype=np.int64)
    nleaf = leaf_ptr.shape[0] - 1
    b = balanced_ranges(p2p_leaf_costs(leaf_ptr, ulist_ptr, ulist_idx), world)
    l0, l1 = int(b[rank]), int(b[rank + 1])
    owned = np.arange(l0, l1)
    used = ulist_idx[ulist_ptr[l0]:ulist_ptr[l1]]
    halo = np.setdiff1d(np.unique(used), owned)
    local_leaves = np.concatenate([owned, halo]).astype(np.int64)
    local_id = np.full(nleaf, -1, dtype=np.int64)
    local_id[local_leaves] = np.arange(local_leaves.shape[0])
    size = np.diff(leaf_ptr)[local_leaves]
    lptr = np.concatenate([[0], np.cumsum(size)]).astype(np.int64)
    rows = (np.concatenate([np.arange(leaf_ptr[a], leaf_ptr[a + 1]) for a in local_leaves])
            if local_leaves.size else np.zeros(0, dtype=np.int64))
    counts = np.concatenate([np.diff(ulist_ptr)[l0:l1], np.zeros(halo.shape[0], dtype=np.int64)])
    uptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    uidx = local_id[used]
    assert (uidx >= 0).all()
    n_owned = int(leaf_ptr[l1] - leaf_ptr[l0])
    return P2PShard((l0, l1), rows.astype(np.int64), n_owned, lptr.astype(np.int32),
                    uptr.astype(np.int32), uidx.astype(np.int32), halo)


def gather_rows(local_out, global_rows, n_global: int, group=None):
    """Assembles rows owned by every rank into the full [n_global, ...] array on
    every rank: global_rows[k] is the global row of local_out[k].  One
    all_gather of the padded blocks (and one of their lengths)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = local_out.device
    idx = torch.as_tensor(np.asarray(global_rows, dtype=np.int64), device=dev)
    n_loc = torch.tensor([idx.shape[0]], dtype=torch.int64, device=dev)
    lens = [torch.zeros_like(n_loc) for _ in range(world)]
    dist.all_gather(lens, n_loc, group=group)
    m = int(max(int(x.item()) for x in lens))
    tail = tuple(local_out.shape[1:])
    pad_v = torch.zeros((m,) + tail, dtype=local_out.dtype, device=dev)
    pad_v[:idx.shape[0]] = local_out
    pad_i = torch.full((m,), -1, dtype=torch.int64, device=dev)
    pad_i[:idx.shape[0]] = idx
    all_v = [torch.empty_like(pad_v) for _ in range(world)]
    all_i = [torch.empty_like(pad_i) for _ in range(world)]
    dist.all_gather(all_v, pad_v, group=group)
    dist.all_gather(all_i, pad_i, group=group)
    full = torch.zeros((int(n_global),) + tail, dtype=local_out.dtype, device=dev)
    for v, i, ln in zip(all_v, all_i, lens):
        k = int(ln.item())
        full[i[:k]] = v[:k]
    return full


class ShardedP2P:
    """One rank's part of the near-field step (P2P over U-lists) sharded over
    the ranks of a process group: the partition of shard_p2p, the rank's
    inputs (owned leaves and halo leaves) copied to its device once, and a step
    that evaluates the local sum and assembles every rank's owned rows with
    gather_rows.

    make_eval(shard) returns the rank's evaluator, a callable taking the dict
    of local input tensors (pts, f, phi, nrm, w, h) and returning the local
    velocities [n_local, 3] (a P2PPlan on a GPU).  pairs is the rank's pair
    count (its owned leaves against their U-lists)."""

    def __init__(self, pts, f, phi, nrm, w, h, leaf_ptr, ulist_ptr, ulist_idx, world: int,
                 rank: int, make_eval, device, group=None):
        import torch
        self.world, self.rank, self.group = int(world), int(rank), group
        self.n_global = int(np.asarray(pts).shape[0])
        self.shard = shard_p2p(leaf_ptr, ulist_ptr, ulist_idx, world, rank)
        r = self.shard.rows
        T = lambda a: None if a is None else torch.as_tensor(
            np.ascontiguousarray(np.asarray(a)[r]), dtype=torch.float64, device=device)
        self.local = {"pts": T(pts), "f": T(f), "phi": T(phi), "nrm": T(nrm), "w": T(w), "h": T(h)}
        self.owned_rows = r[:self.shard.n_owned]
        self.evaluate = make_eval(self.shard)
        costs = p2p_leaf_costs(self.shard.leaf_ptr, self.shard.ulist_ptr, self.shard.ulist_idx)
        self.pairs = int(costs.sum())
        # the row map of the gather is fixed: exchanged once, so that a step
        # moves only the velocities (one all_gather, no host synchronisation)
        import torch.distributed as dist
        ws = dist.get_world_size(group)
        n_loc = torch.tensor([self.shard.n_owned], dtype=torch.int64, device=device)
        lens = [torch.zeros_like(n_loc) for _ in range(ws)]
        dist.all_gather(lens, n_loc, group=group)
        self.lens = [int(x.item()) for x in lens]
        self.m = max(self.lens)
        pad_i = torch.full((self.m,), -1, dtype=torch.int64, device=device)
        pad_i[:self.shard.n_owned] = torch.as_tensor(self.owned_rows, device=device)
        all_i = [torch.empty_like(pad_i) for _ in range(ws)]
        dist.all_gather(all_i, pad_i, group=group)
        self.gather_index = torch.cat([i[:k] for i, k in zip(all_i, self.lens)])
        self.pad_v = torch.zeros((self.m, 3), dtype=torch.float64, device=device)
        self.all_v = [torch.empty_like(self.pad_v) for _ in range(ws)]
        self.full = torch.zeros((self.n_global, 3), dtype=torch.float64, device=device)

    def step(self):
        """Local evaluation + gather of the owned rows: the full [n, 3] velocity
        on every rank (the same buffer each step)."""
        import torch
        import torch.distributed as dist
        out = self.evaluate(self.local)
        self.pad_v[:self.shard.n_owned] = out[:self.shard.n_owned]
        dist.all_gather(self.all_v, self.pad_v, group=self.group)
        vals = torch.cat([v[:k] for v, k in zip(self.all_v, self.lens)])
        self.full[self.gather_index] = vals
        return self.full
