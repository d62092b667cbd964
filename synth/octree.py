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


@dataclass
class FarLists:
    """All boxes of an octree and the interaction lists of the FMM's far field.

    Boxes are numbered depth by depth (depth 0 first), Morton order within a
    depth.  `leaf[n]` is the leaf number of box n or -1; `parent[n]` is -1 for
    the root.  CSR lists over box numbers:
      V(B): children of the same-level neighbours of B's parent that do not touch B;
      W(B), B a leaf: boxes A below B's same-level neighbours that do not touch B
            while their parent does;
      X(B): the leaves A with B in W(A).
    "Touch" is the closed-box intersection of the U-lists."""
    depth: np.ndarray      # int32 [M]
    anchor: np.ndarray     # int64 [M, 3] box index at its depth
    parent: np.ndarray     # int32 [M]
    leaf: np.ndarray       # int32 [M]
    v_ptr: np.ndarray
    v_idx: np.ndarray
    w_ptr: np.ndarray
    w_idx: np.ndarray
    x_ptr: np.ndarray
    x_idx: np.ndarray


def far_lists(tree: Octree) -> FarLists:
    leaves = [(int(tree.leaf_depth[b]),) + tuple(int(v) >> (MAX_DEPTH - int(tree.leaf_depth[b]))
                                                 for v in tree.leaf_lo[b]) for b in range(tree.nleaf)]
    nodes = set()
    for nd in leaves:
        d = nd[0]
        for k in range(d + 1):
            nodes.add((k,) + tuple(v >> (d - k) for v in nd[1:]))

    def mkey(nd):
        return (nd[0],) + (int(morton_keys(np.asarray([nd[1:]], dtype=np.int64))[0]),)

    order = sorted(nodes, key=mkey)
    num = {nd: i for i, nd in enumerate(order)}
    leaf_of = {nd: b for b, nd in enumerate(leaves)}
    M = len(order)
    depth = np.array([nd[0] for nd in order], dtype=np.int32)
    anchor = np.array([nd[1:] for nd in order], dtype=np.int64).reshape(M, 3)
    par = np.array([num[(nd[0] - 1,) + tuple(v >> 1 for v in nd[1:])] if nd[0] else -1
                    for nd in order], dtype=np.int32)
    leaf = np.array([leaf_of.get(nd, -1) for nd in order], dtype=np.int32)
    kids = {}
    for nd in order:
        if nd[0]:
            kids.setdefault((nd[0] - 1,) + tuple(v >> 1 for v in nd[1:]), []).append(nd)

    def touch(a, b):
        sa, sb = 1 << (MAX_DEPTH - a[0]), 1 << (MAX_DEPTH - b[0])
        return all(a[1 + i] * sa <= (b[1 + i] + 1) * sb and b[1 + i] * sb <= (a[1 + i] + 1) * sa
                   for i in range(3))

    def neighbours(nd):
        d = nd[0]
        out = []
        for o in np.ndindex(3, 3, 3):
            q = (d,) + tuple(nd[1 + i] + o[i] - 1 for i in range(3))
            if q in num:
                out.append(q)
        return out

    V = [[] for _ in range(M)]
    W = [[] for _ in range(M)]
    X = [[] for _ in range(M)]
    for nd in order:
        if nd[0] >= 2:
            pn = (nd[0] - 1,) + tuple(v >> 1 for v in nd[1:])
            V[num[nd]] = sorted(num[c] for q in neighbours(pn) for c in kids.get(q, ())
                                if not touch(c, nd))
    for nd in leaves:
        stack = [q for q in neighbours(nd) if q != nd and q not in leaf_of]
        out = []
        while stack:
            q = stack.pop()
            for c in kids.get(q, ()):
                if not touch(c, nd):
                    out.append(num[c])
                elif c not in leaf_of:
                    stack.append(c)
        W[num[nd]] = sorted(out)
        for a in out:
            X[a].append(num[nd])

    def csr(lists):
        ptr = np.zeros(M + 1, dtype=np.int64)
        ptr[1:] = np.cumsum([len(x) for x in lists])
        idx = np.array([i for x in lists for i in sorted(x)], dtype=np.int32)
        return ptr, idx

    (vp, vi), (wp, wi), (xp, xi) = csr(V), csr(W), csr(X)
    return FarLists(depth=depth, anchor=anchor, parent=par, leaf=leaf, v_ptr=vp, v_idx=vi,
                    w_ptr=wp, w_idx=wi, x_ptr=xp, x_idx=xi)
