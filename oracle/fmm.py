"""Kernel-independent FMM oracle for the far field of the layer-potential sums
(test infrastructure).

Only the tests may import this module; the GPU library neither links nor
calls it.

The paper evaluates the smooth quadrature (Eq. "smooth_double_layer_int_eq_
patches_disc", and the single layer of Eq. "sl_stokes") at all targets at once
with a kernel-independent FMM (Sec. 3.1, "Far evaluation"); it names the
method, not its constants.  This oracle takes the method's steps in order, in
plain FP64 numpy, on a uniform octree (every leaf at one depth):
  1. S2M: the sources of a leaf give a velocity on the leaf's upward check
     surface; the upward equivalent density on the upward equivalent surface
     reproduces it (least squares through a truncated pseudo-inverse);
  2. M2M: the children's equivalent densities give the parent's check
     velocity, and so its equivalent density, up to level 2;
  3. M2L: each box's downward check velocity collects the equivalent
     densities of its interaction list (children of the parent's neighbours
     that are not its own neighbours), plus L2L: its parent's downward
     equivalent density; the downward equivalent density reproduces it;
  4. L2T and P2P: at a leaf, its downward equivalent density plus the direct
     sum over the neighbouring leaves (the U-list).
Surfaces are the boundaries of p x p x p grids on cubes of half-width 1.05 r
(upward equivalent, downward check) and 2.95 r (upward check, downward
equivalent) about a box of half-width r.  The upward equivalent density has a
Stokeslet and a point source at each surface point: the double layer carries a
net flux through a closed surface, which Stokeslets (divergence-free with zero
flux) cannot represent; the downward (interior, regular) field has none, so
Stokeslets suffice there.  Direct sums come from the C oracle (stokes_oracle.c).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import sldl as _sldl

R_INNER, R_OUTER = 1.05, 2.95


def cube_surface(p: int) -> np.ndarray:
    """Points of a p x p x p grid on [-1, 1]^3 that lie on the cube's boundary."""
    g = np.linspace(-1.0, 1.0, p)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return X[np.any(np.abs(X) == 1.0, axis=1)]


def stokeslet_matrix(x, y, mu: float = 1.0) -> np.ndarray:
    """[3 nx, 3 ny]: velocity at x of unit forces at y, (I/r + d d^T/r^3)/(8 pi mu), d = x - y."""
    d = x[:, None, :] - y[None, :, :]
    r2 = (d * d).sum(-1)
    ri = np.where(r2 > 0, 1.0 / np.sqrt(np.where(r2 > 0, r2, 1.0)), 0.0)
    K = np.eye(3)[None, None] * ri[..., None, None] + d[..., :, None] * d[..., None, :] * (ri ** 3)[..., None, None]
    return (K / (8 * np.pi * mu)).transpose(0, 2, 1, 3).reshape(3 * x.shape[0], 3 * y.shape[0])


def source_matrix(x, y) -> np.ndarray:
    """[3 nx, ny]: velocity at x of unit point sources at y, d / (4 pi r^3)."""
    d = x[:, None, :] - y[None, :, :]
    r2 = (d * d).sum(-1)
    ri3 = np.where(r2 > 0, np.where(r2 > 0, r2, 1.0) ** -1.5, 0.0)
    K = d * ri3[..., None] / (4 * np.pi)
    return K.transpose(0, 2, 1).reshape(3 * x.shape[0], y.shape[0])


def upward_matrix(x, y, mu: float, flux: bool) -> np.ndarray:
    """Velocity at x of upward equivalent densities at y: per point a force
    (3 columns) and, with flux, a source strength (1 column)."""
    S = stokeslet_matrix(x, y, mu).reshape(3 * x.shape[0], y.shape[0], 3)
    if not flux:
        return S.reshape(3 * x.shape[0], 3 * y.shape[0])
    Q = source_matrix(x, y)[:, :, None]
    return np.concatenate([S, Q], axis=2).reshape(3 * x.shape[0], 4 * y.shape[0])


def pinv(A, rcond: float = 1e-13) -> np.ndarray:
    return np.linalg.pinv(A, rcond=rcond)


class UniformTree:
    """A uniform octree of `depth` levels over the points' bounding cube."""

    def __init__(self, pts, depth: int):
        pts = np.asarray(pts, dtype=np.float64)
        lo, hi = pts.min(0), pts.max(0)
        self.L = float((hi - lo).max()) * (1 + 1e-9) + 1e-300
        self.lo = lo - 1e-12 * self.L
        self.depth = depth
        m = 1 << depth
        ijk = np.minimum(((pts - self.lo) / (self.L / m)).astype(np.int64), m - 1)
        self.leaf_of = (ijk[:, 0] * m + ijk[:, 1]) * m + ijk[:, 2]
        self.members = {}
        for i, b in enumerate(self.leaf_of):
            self.members.setdefault(int(b), []).append(i)

    def width(self, level: int) -> float:
        return self.L / (1 << level)

    def centre(self, level: int, ijk) -> np.ndarray:
        return self.lo + (np.asarray(ijk, dtype=np.float64) + 0.5) * self.width(level)


def _ijk(index: int, m: int):
    return index // (m * m), (index // m) % m, index % m


def _index(i, j, k, m: int) -> int:
    return (i * m + j) * m + k


def fmm(pts, f, phi, nrm, w, depth: int, p: int, mu: float = 1.0, flux: bool = True):
    """Velocity at the points (targets = sources; a point contributes nothing to
    itself) of the single layer of f and the double layer of phi."""
    pts = np.asarray(pts, dtype=np.float64)
    n = pts.shape[0]
    zeros = np.zeros((n, 3))
    f = zeros if f is None else np.asarray(f, dtype=np.float64)
    phi = zeros if phi is None else np.asarray(phi, dtype=np.float64)
    nrm = np.tile([0.0, 0.0, 1.0], (n, 1)) if nrm is None else np.asarray(nrm, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    T = UniformTree(pts, depth)
    S = cube_surface(p)
    ns = S.shape[0]
    nc = 4 if flux else 3
    D = depth

    # operators per level (they depend on the box size only)
    uc2e, dc2e = {}, {}
    for l in range(2, D + 1):
        r = T.width(l) / 2
        uc2e[l] = pinv(upward_matrix(R_OUTER * r * S, R_INNER * r * S, mu, flux))
        dc2e[l] = pinv(stokeslet_matrix(R_INNER * r * S, R_OUTER * r * S, mu))

    # 1. S2M at the leaves (a tree of depth < 2 has no far field: every leaf is
    # a neighbour of every other)
    up = {D: {}}
    for b, idx in (T.members.items() if D >= 2 else ()):
        idx = np.asarray(idx)
        c = T.centre(D, _ijk(b, 1 << D))
        r = T.width(D) / 2
        chk = _sldl(pts[idx], f[idx], nrm[idx], phi[idx], w[idx], c + R_OUTER * r * S, mu)
        up[D][b] = uc2e[D] @ chk.reshape(-1)

    # 2. M2M up to level 2
    for l in range(D - 1, 1, -1):
        up[l] = {}
        m, r = 1 << l, T.width(l) / 2
        rc = T.width(l + 1) / 2
        for cb, e in up[l + 1].items():
            ci, cj, ck = _ijk(cb, 2 * m)
            b = _index(ci // 2, cj // 2, ck // 2, m)
            pc = T.centre(l, _ijk(b, m))
            cc = T.centre(l + 1, (ci, cj, ck))
            K = upward_matrix(pc + R_OUTER * r * S, cc + R_INNER * rc * S, mu, flux)
            up[l][b] = up[l].get(b, 0.0) + K @ e
        for b in up[l]:
            up[l][b] = uc2e[l] @ up[l][b]

    # 3. M2L (interaction lists, grouped by offset) and L2L
    down = {}
    for l in range(2, D + 1):
        m, r = 1 << l, T.width(l) / 2
        h = T.width(l)
        chk = {}
        # targets: boxes with points below them
        targets = {_parent_at(b, D, l) for b in T.members}
        for o in itertools.product(range(-3, 4), repeat=3):
            if max(abs(v) for v in o) <= 1:
                continue
            M = None
            for b in targets:
                i, j, k = _ijk(b, m)
                a = (i + o[0], j + o[1], k + o[2])
                if min(a) < 0 or max(a) >= m:
                    continue
                # interaction list: parents are neighbours (or the same box)
                if max(abs(a[d] // 2 - (i, j, k)[d] // 2) for d in range(3)) > 1:
                    continue
                ai = _index(*a, m)
                if ai not in up[l]:
                    continue
                if M is None:
                    M = upward_matrix(R_INNER * r * S, np.asarray(o, float) * h + R_INNER * r * S, mu, flux)
                chk[b] = chk.get(b, 0.0) + M @ up[l][ai]
        down[l] = {}
        for b in targets:
            v = chk.get(b, np.zeros(3 * ns))
            if l > 2:
                pb = _parent_at(b, l, l - 1)
                if pb in down[l - 1]:
                    c, pc = T.centre(l, _ijk(b, m)), T.centre(l - 1, _ijk(pb, m // 2))
                    K = stokeslet_matrix(c + R_INNER * r * S, pc + R_OUTER * (2 * r) * S, mu)
                    v = v + K @ down[l - 1][pb]
            down[l][b] = dc2e[l] @ v

    # 4. L2T and P2P at the leaves
    u = np.zeros((n, 3))
    m, r = 1 << D, T.width(D) / 2
    for b, idx in T.members.items():
        idx = np.asarray(idx)
        i, j, k = _ijk(b, m)
        c = T.centre(D, (i, j, k))
        if D >= 2:
            u[idx] += (stokeslet_matrix(pts[idx], c + R_OUTER * r * S, mu) @ down[D][b]).reshape(-1, 3)
        near = []
        for o in itertools.product((-1, 0, 1), repeat=3):
            a = (i + o[0], j + o[1], k + o[2])
            if min(a) >= 0 and max(a) < m and _index(*a, m) in T.members:
                near.extend(T.members[_index(*a, m)])
        near = np.asarray(near)
        u[idx] += _sldl(pts[near], f[near], nrm[near], phi[near], w[near], pts[idx], mu)
    return u


def _parent_at(b: int, level_b: int, level: int) -> int:
    """Index at `level` of the ancestor of box b of level `level_b`."""
    mb = 1 << level_b
    i, j, k = _ijk(b, mb)
    s = level_b - level
    return _index(i >> s, j >> s, k >> s, 1 << level)


# ---------------------------------------------------------------- adaptive trees
def _adjacent(n1, n2, maxd: int) -> bool:
    """Closed boxes of nodes (depth, i, j, k) intersect (exact, in units of the
    deepest level)."""
    d1, d2 = n1[0], n2[0]
    s1, s2 = 1 << (maxd - d1), 1 << (maxd - d2)
    return all(n1[1 + a] * s1 <= (n2[1 + a] + 1) * s2 and n2[1 + a] * s2 <= (n1[1 + a] + 1) * s1
               for a in range(3))


def fmm_adaptive(tree, pts, f, phi, nrm, w, p: int, mu: float = 1.0, flux: bool = True,
                 stats: dict | None = None, lists_only: bool = False, ops: dict | None = None,
                 near: bool = True):
    """The same method on an adaptive octree (synth.octree: leaves in Morton
    order, points sorted by leaf, U-lists of adjacent leaves).  Besides the
    interaction (V) lists, a leaf B takes the upward equivalent densities of
    its W-list at its points (descendants of its same-level neighbours that do
    not touch B but whose parent does), and a node B takes the sources of its
    X-list (the leaves whose W-list holds B) on its downward check surface.

    ops, if given, maps a depth to its (upward, downward) check-to-equivalent
    operators in place of the pseudo-inverses computed here; near=False leaves
    out the U-list sum (the far field alone)."""
    pts = np.asarray(pts, dtype=np.float64)
    n = pts.shape[0]
    zeros = np.zeros((n, 3))
    f = zeros if f is None else np.asarray(f, dtype=np.float64)
    phi = zeros if phi is None else np.asarray(phi, dtype=np.float64)
    nrm = np.tile([0.0, 0.0, 1.0], (n, 1)) if nrm is None else np.asarray(nrm, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    MD = 21
    S = cube_surface(p)

    leaves = []
    for b in range(tree.nleaf):
        d = int(tree.leaf_depth[b])
        a = tuple(int(v) >> (MD - d) for v in tree.leaf_lo[b])
        leaves.append((d,) + a)
    leaf_id = {nd: b for b, nd in enumerate(leaves)}
    nodes = set()
    for nd in leaves:
        d = nd[0]
        for k in range(d + 1):
            nodes.add((k,) + tuple(v >> (d - k) for v in nd[1:]))
    children = {}
    for nd in nodes:
        if nd[0] > 0:
            par = (nd[0] - 1,) + tuple(v >> 1 for v in nd[1:])
            children.setdefault(par, []).append(nd)
    by_depth = {}
    for nd in nodes:
        by_depth.setdefault(nd[0], []).append(nd)
    maxd = max(by_depth)

    def geom(nd):
        size = tree.root_size / (1 << nd[0])
        return tree.root_lo + (np.asarray(nd[1:], dtype=np.float64) + 0.5) * size, size / 2

    def parent(nd):
        return (nd[0] - 1,) + tuple(v >> 1 for v in nd[1:])

    def colleagues(nd):
        return [q for q in by_depth[nd[0]] if _adjacent(q, nd, maxd)]

    def leaf_points(nd):
        b = leaf_id[nd]
        return np.arange(tree.leaf_ptr[b], tree.leaf_ptr[b + 1])

    uc2e, dc2e = {}, {}
    given = ops

    def ops(d):
        if d not in uc2e and given is not None and d in given:
            uc2e[d], dc2e[d] = given[d]
        if d not in uc2e:
            r = tree.root_size / (1 << d) / 2
            uc2e[d] = pinv(upward_matrix(R_OUTER * r * S, R_INNER * r * S, mu, flux))
            dc2e[d] = pinv(stokeslet_matrix(R_INNER * r * S, R_OUTER * r * S, mu))
        return uc2e[d], dc2e[d]

    # upward pass (deepest first)
    up = {}
    for d in (sorted(by_depth, reverse=True) if not lists_only else ()):
        for nd in by_depth[d]:
            c, r = geom(nd)
            if nd in leaf_id:
                idx = leaf_points(nd)
                chk = _sldl(pts[idx], f[idx], nrm[idx], phi[idx], w[idx], c + R_OUTER * r * S, mu).reshape(-1)
            else:
                chk = 0.0
                for ch in children[nd]:
                    cc, rc = geom(ch)
                    chk = chk + upward_matrix(c + R_OUTER * r * S, cc + R_INNER * rc * S, mu, flux) @ up[ch]
            up[nd] = ops(d)[0] @ chk

    # lists
    V, W, X = {}, {}, {}
    for nd in nodes:
        if nd[0] >= 2:
            V[nd] = [ch for q in colleagues(parent(nd)) for ch in children.get(q, [])
                     if not _adjacent(ch, nd, maxd)]
    for nd in leaves:
        W[nd] = []
        stack = [q for q in colleagues(nd) if q != nd and q not in leaf_id]
        while stack:
            q = stack.pop()
            for ch in children.get(q, []):
                if not _adjacent(ch, nd, maxd):
                    W[nd].append(ch)  # its parent q touches nd
                elif ch not in leaf_id:
                    stack.append(ch)
        for a in W[nd]:
            X.setdefault(a, []).append(nd)
    if stats is not None:
        stats.update(v=sum(map(len, V.values())), w=sum(map(len, W.values())),
                     x=sum(map(len, X.values())), depths=sorted(by_depth),
                     lists={"V": V, "W": W, "X": X})
    if lists_only:
        return None

    # downward pass (shallowest first); M2L matrices cached by depth and offset
    m2l = {}
    down = {}
    for d in sorted(by_depth):
        if d < 2:
            continue
        for nd in by_depth[d]:
            c, r = geom(nd)
            chk = np.zeros(3 * S.shape[0])
            for a in V[nd]:
                key = (d,) + tuple(a[i + 1] - nd[i + 1] for i in range(3))
                if key not in m2l:
                    h = 2 * r
                    m2l[key] = upward_matrix(R_INNER * r * S, np.asarray(key[1:], float) * h
                                             + R_INNER * r * S, mu, flux)
                chk += m2l[key] @ up[a]
            for a in X.get(nd, []):
                idx = leaf_points(a)
                chk += _sldl(pts[idx], f[idx], nrm[idx], phi[idx], w[idx], c + R_INNER * r * S, mu).reshape(-1)
            if d > 2:
                pc, pr = geom(parent(nd))
                chk += stokeslet_matrix(c + R_INNER * r * S, pc + R_OUTER * pr * S, mu) @ down[parent(nd)]
            down[nd] = ops(d)[1] @ chk

    # leaves: L2T, W-list, U-list
    u = np.zeros((n, 3))
    for nd in leaves:
        b = leaf_id[nd]
        idx = leaf_points(nd)
        if nd[0] >= 2:
            c, r = geom(nd)
            u[idx] += (stokeslet_matrix(pts[idx], c + R_OUTER * r * S, mu) @ down[nd]).reshape(-1, 3)
        for a in W[nd]:
            ca, ra = geom(a)
            u[idx] += (upward_matrix(pts[idx], ca + R_INNER * ra * S, mu, flux) @ up[a]).reshape(-1, 3)
        if near:
            nb = np.concatenate([leaf_points(leaves[a]) for a in
                                 tree.ulist_idx[tree.ulist_ptr[b]:tree.ulist_ptr[b + 1]]])
            u[idx] += _sldl(pts[nb], f[nb], nrm[nb], phi[nb], w[nb], pts[idx], mu)
    return u
