"""Adaptive octree and U-lists (near-field interaction lists) for P2P inputs.

The far evaluation of the paper (Sec. 3.1 "Far evaluation") is a
kernel-independent FMM; its near field is the direct (P2P) sum of every leaf
B with the leaves in its U-list.  The paper does not describe the tree, so
this module fixes one reading of it:

  * root: the bounding cube of all points, grown by 1e-9 (relative) so that
    every point lies strictly inside;
  * a box is split into its 8 children while it holds more than `max_leaf`
    points (up to depth 21); a point belongs to the child whose half-open
    box [lo, hi) contains it; empty children are dropped;
  * no 2:1 balance;
  * U(B) = { leaves A : closed(A) intersects closed(B) }, which contains B.

Boxes are kept as integer anchors on the depth-21 grid so that the adjacency
test is exact.  Leaves are numbered in Morton (depth-first) order and the
points are permuted so that every leaf is one contiguous range.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MAX_DEPTH = 21


def _spread_bits(v: np.ndarray) -> np.ndarray:
    """Insert two zero bits between the low 21 bits of v (for 3-D Morton keys)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_keys(ijk: np.ndarray) -> np.ndarray:
    return (_spread_bits(ijk[:, 0]) << np.uint64(2)) | (_spread_bits(ijk[:, 1]) << np.uint64(1)) \
        | _spread_bits(ijk[:, 2])


@dataclass
class Octree:
    perm: np.ndarray        # sorted position -> original point index
    leaf_ptr: np.ndarray    # int32 [L+1], ranges of leaves in sorted order
    ulist_ptr: np.ndarray   # int32 [L+1]
    ulist_idx: np.ndarray   # int32 [sum |U(B)|], ascending leaf numbers
    leaf_lo: np.ndarray     # int64 [L, 3] closed box, depth-21 integer units
    leaf_hi: np.ndarray     # int64 [L, 3]
    leaf_depth: np.ndarray  # int32 [L]
    root_lo: np.ndarray     # float64 [3]
    root_size: float

    @property
    def nleaf(self) -> int:
        return int(self.leaf_ptr.size - 1)

    def pair_count(self) -> int:
        """Exact number of (target, source) pairs the U-list P2P evaluates."""
        sz = np.diff(self.leaf_ptr).astype(np.int64)
        tot = 0
        for b in range(self.nleaf):
            a = self.ulist_idx[self.ulist_ptr[b]:self.ulist_ptr[b + 1]]
            tot += int(sz[b]) * int(sz[a].sum())
        return tot


def build_octree(pts: np.ndarray, max_leaf: int = 256) -> Octree:
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    n = pts.shape[0]
    if n == 0:
        raise ValueError("empty point set")
    cmin, cmax = pts.min(0), pts.max(0)
    ext = float((cmax - cmin).max())
    if ext == 0.0:
        ext = 1.0
    size = ext * (1.0 + 1e-9) + 1e-300
    lo = 0.5 * (cmin + cmax) - 0.5 * size
    scale = float(1 << MAX_DEPTH)
    ijk = np.floor((pts - lo) / size * scale).astype(np.int64)
    ijk = np.clip(ijk, 0, (1 << MAX_DEPTH) - 1)
    keys = morton_keys(ijk)
    perm = np.argsort(keys, kind="stable")
    skeys = keys[perm]

    leaves = []  # (start, end, depth, anchor key prefix)
    stack = [(0, n, 0, np.uint64(0))]
    while stack:
        a, b, d, prefix = stack.pop()
        if b - a <= max_leaf or d == MAX_DEPTH:
            leaves.append((a, b, d, prefix))
            continue
        shift = np.uint64(3 * (MAX_DEPTH - d - 1))
        children = []
        for c in range(8):
            child = (prefix << np.uint64(3)) | np.uint64(c)
            klo = child << shift
            khi = (child + np.uint64(1)) << shift
            ca = a + int(np.searchsorted(skeys[a:b], klo, side="left"))
            cb = a + int(np.searchsorted(skeys[a:b], khi, side="left"))
            if cb > ca:
                children.append((ca, cb, d + 1, child))
        # push in reverse so that the stack pops children in Morton order
        stack.extend(reversed(children))
    leaves.sort(key=lambda t: t[0])
    L = len(leaves)
    leaf_ptr = np.zeros(L + 1, dtype=np.int64)
    depth = np.zeros(L, dtype=np.int32)
    anchor = np.zeros((L, 3), dtype=np.int64)
    for i, (a, b, d, prefix) in enumerate(leaves):
        leaf_ptr[i], leaf_ptr[i + 1] = a, b
        depth[i] = d
        # de-interleave the prefix (3 d bits) into the box index at depth d
        ix = iy = iz = 0
        pv = int(prefix)
        for lvl in range(d):
            bits = (pv >> (3 * (d - 1 - lvl))) & 7
            ix = (ix << 1) | ((bits >> 2) & 1)
            iy = (iy << 1) | ((bits >> 1) & 1)
            iz = (iz << 1) | (bits & 1)
        anchor[i] = (ix, iy, iz)
    side = (1 << (MAX_DEPTH - depth)).astype(np.int64)
    box_lo = anchor * side[:, None]
    box_hi = box_lo + side[:, None]

    ulist_ptr = np.zeros(L + 1, dtype=np.int64)
    chunks = []
    CH = 256
    for s in range(0, L, CH):
        e = min(L, s + CH)
        m = np.all((box_lo[None, :, :] <= box_hi[s:e, None, :]) &
                   (box_lo[s:e, None, :] <= box_hi[None, :, :]), axis=2)
        rows, cols = np.nonzero(m)
        counts = np.bincount(rows, minlength=e - s)
        ulist_ptr[s + 1:e + 1] = counts
        chunks.append(cols)
    ulist_ptr = np.cumsum(ulist_ptr)
    ulist_idx = np.concatenate(chunks) if chunks else np.zeros(0, dtype=np.int64)
    if leaf_ptr[-1] > np.iinfo(np.int32).max or ulist_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("octree too large for int32 indices")
    return Octree(perm=perm, leaf_ptr=leaf_ptr.astype(np.int32),
                  ulist_ptr=ulist_ptr.astype(np.int32), ulist_idx=ulist_idx.astype(np.int32),
                  leaf_lo=box_lo, leaf_hi=box_hi, leaf_depth=depth, root_lo=lo,
                  root_size=size)
