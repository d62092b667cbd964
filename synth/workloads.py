"""Seeded synthetic workloads with the shapes of the paper's suspensions.

The paper measures on RBC suspensions inside patient vessel meshes that are
not available (Sec. 5); these generators stand in for them with the same
discretisation (544-point p = 16 cells, 121-point wall patches).  Every
array is FP64, AoS [n, 3] for vectors.  Densities are i.i.d. U[-1, 1]^3.

Seeds: numpy Generator(PCG64(seed)), seed 11085001 ... 11085005 for the five
workloads; the batched workload draws suspension s from
SeedSequence(11085003).spawn(S)[s].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

from . import geometry as G
from .octree import Octree, build_octree

SEED_SL_DIRECT = 11085001
SEED_DL_DIRECT = 11085002
SEED_BATCHED = 11085003
SEED_P2P = 11085004
SEED_ADJOINT = 11085005


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Surfaces:
    """Points on a set of closed cells (and optionally a wall)."""
    pts: np.ndarray
    nrm: np.ndarray
    w: np.ndarray
    h: np.ndarray
    cell_id: np.ndarray            # -1 for wall points
    centres: np.ndarray = None
    rotations: list = field(default_factory=list)
    orders: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return self.pts.shape[0]


def cells_at(centres, rotations, orders, R=G.RBC_RADIUS) -> Surfaces:
    pts, nrm, w, h, cid = [], [], [], [], []
    for c, (cen, rot, p) in enumerate(zip(centres, rotations, orders)):
        X, N, W = G.rbc_surface(p, R)
        pts.append(X @ rot.T + cen)
        nrm.append(N @ rot.T)
        w.append(W)
        h.append(np.full(W.size, np.sqrt(W.sum() / W.size)))
        cid.append(np.full(W.size, c, dtype=np.int64))
    return Surfaces(np.concatenate(pts), np.concatenate(nrm), np.concatenate(w),
                    np.concatenate(h), np.concatenate(cid), np.asarray(centres),
                    list(rotations), list(orders))


def random_cells_in_box(rng, ncell: int, box: float, p: int = 16) -> Surfaces:
    rb = G.RBC_RADIUS + 0.05
    centres = G.place_in_box(rng, ncell, box, rb)
    rots = [G.random_rotation(rng) for _ in range(ncell)]
    return cells_at(centres, rots, [p] * ncell)


def densities(rng, n: int) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, size=(n, 3))


def off_surface_targets(rng, surf: Surfaces, count: int, dmin=0.05, dmax=5.0,
                        R=G.RBC_RADIUS) -> np.ndarray:
    """Targets off the cell surfaces at log-uniform distances along the outward normal.

    A cell is drawn uniformly, then a surface point from uniform (cos theta, phi),
    then a distance delta log-uniform in [dmin, dmax]; the point is rejected if any
    surface sample point is closer than 0.9 delta.
    """
    tree = cKDTree(surf.pts)
    out = []
    ncell = len(surf.centres)
    while len(out) < count:
        m = 2 * (count - len(out)) + 64
        c = rng.integers(0, ncell, size=m)
        t = rng.uniform(-1.0, 1.0, size=m)
        ph = rng.uniform(0.0, 2.0 * np.pi, size=m)
        delta = np.exp(rng.uniform(np.log(dmin), np.log(dmax), size=m))
        th = np.arccos(t)
        X, Xt, Xp = G.rbc_map(th, ph, R)
        nb = np.cross(Xt, Xp)
        nb /= np.linalg.norm(nb, axis=1)[:, None]
        rot = np.stack([surf.rotations[i] for i in c])
        base = np.einsum("mij,mj->mi", rot, X) + surf.centres[c]
        nw = np.einsum("mij,mj->mi", rot, nb)
        x = base + delta[:, None] * nw
        dist, _ = tree.query(x)
        keep = dist >= 0.9 * delta
        out.extend(list(x[keep]))
    return np.asarray(out[:count])


def interior_targets(surf: Surfaces, per_cell: int = 8, R=G.RBC_RADIUS) -> np.ndarray:
    """Points inside each cell on the rim ring z = 0, rho = 0.75 R (body frame)."""
    ang = 2.0 * np.pi * np.arange(per_cell) / per_cell
    ring = np.stack([0.75 * R * np.cos(ang), 0.75 * R * np.sin(ang), np.zeros(per_cell)], 1)
    return np.concatenate([ring @ rot.T + c for c, rot in zip(surf.centres, surf.rotations)])


# --------------------------------------------------------------------------- workloads

@dataclass
class DirectWorkload:
    name: str
    src: np.ndarray
    nrm: np.ndarray
    w: np.ndarray
    h: np.ndarray
    f: np.ndarray
    phi: np.ndarray
    trg: np.ndarray
    mu: float
    targets_are_sources: bool
    surf: Surfaces = None

    def pairs(self) -> int:
        ns, nt = self.src.shape[0], self.trg.shape[0]
        return ns * nt - (ns if self.targets_are_sources else 0)


def sl_direct_workload(ncell: int = 8, box: float = 40.0, p: int = 16,
                       seed: int = SEED_SL_DIRECT) -> DirectWorkload:
    """Direct single-layer self-sum: 8 cells (4,352 points) in a 40^3 box, mu = 1."""
    rng = rng_for(seed)
    s = random_cells_in_box(rng, ncell, box, p)
    f = densities(rng, s.n)
    phi = densities(rng, s.n)
    return DirectWorkload("sl_direct_8rbc_p16", s.pts, s.nrm, s.w, s.h, f, phi,
                          s.pts.copy(), 1.0, True, s)


def dl_direct_workload(ncell: int = 256, box: float = 120.0, p: int = 16, n_off: int = 65536,
                       seed: int = SEED_DL_DIRECT) -> DirectWorkload:
    """Direct double-layer: 256 cells (139,264 points) in a 120^3 box.

    Targets are the surface points followed by n_off off-surface points at
    0.05-5 um along the outward normal.
    """
    rng = rng_for(seed)
    s = random_cells_in_box(rng, ncell, box, p)
    phi = densities(rng, s.n)
    f = densities(rng, s.n)
    off = off_surface_targets(rng, s, n_off) if n_off else np.zeros((0, 3))
    trg = np.concatenate([s.pts, off])
    return DirectWorkload(f"dl_direct_{ncell}rbc_p16", s.pts, s.nrm, s.w, s.h, f, phi, trg,
                          1.0, False, s)


def adjoint_workload(ncell: int = 64, box: float = 48.0, p: int = 16,
                     seed: int = SEED_ADJOINT):
    """64 cells (34,816 points) in a 48^3 box, with an upstream gradient g."""
    rng = rng_for(seed)
    s = random_cells_in_box(rng, ncell, box, p)
    f = densities(rng, s.n)
    phi = densities(rng, s.n)
    g = densities(rng, s.n)
    wl = DirectWorkload(f"adjoint_{ncell}rbc_p16", s.pts, s.nrm, s.w, s.h, f, phi,
                        s.pts.copy(), 1.0, True, s)
    return wl, g


@dataclass
class P2PWorkload:
    name: str
    pts: np.ndarray      # leaf-sorted
    nrm: np.ndarray
    w: np.ndarray
    h: np.ndarray
    f: np.ndarray
    phi: np.ndarray
    tree: Octree
    mu: float
    n_cell_points: int
    n_wall_points: int

    def pairs(self) -> int:
        return self.tree.pair_count()


def dense_cylinder_suspension(rng, ncell: int, radius: float, n_wall_patch: int,
                              spacing=(8.0, 8.0, 4.0), max_tilt_deg: float = 5.0,
                              p: int = 16):
    """Cells packed on a jittered lattice inside a cylinder along z, plus its wall.

    Cells sit at lattice sites (dx, dy, dz) whose centres are at least
    R_cell + 0.2 from the wall; each cell's axis is tilted by at most
    max_tilt_deg and spun uniformly about it, which keeps neighbouring cells
    apart for the default spacing.  The cylinder length is the span of the
    layers used.  The wall is split into patches of about equal sides.
    """
    dx, dy, dz = spacing
    rmax = radius - G.RBC_RADIUS - 0.2
    nx = int(np.floor(rmax / dx))
    xs = np.arange(-nx, nx + 1) * dx
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    keep = X ** 2 + Y ** 2 <= rmax ** 2
    layer = np.stack([X[keep], Y[keep]], 1)
    nlayer = int(np.ceil(ncell / layer.shape[0]))
    length = nlayer * dz + 2.0
    sites = np.concatenate([np.column_stack([layer, np.full(layer.shape[0], 1.0 + (k + 0.5) * dz)])
                            for k in range(nlayer)])
    pick = np.sort(rng.choice(sites.shape[0], size=ncell, replace=False))
    centres = sites[pick]
    rots = []
    tilt_max = np.deg2rad(max_tilt_deg)
    for _ in range(ncell):
        spin = G.rotation_about_axis([0, 0, 1], rng.uniform(0, 2 * np.pi))
        ax = rng.normal(size=3)
        ax[2] = 0.0
        if np.linalg.norm(ax) == 0:
            ax = np.array([1.0, 0.0, 0.0])
        tilt = G.rotation_about_axis(ax, rng.uniform(0, tilt_max))
        rots.append(tilt @ spin)
    cells = cells_at(centres, rots, [p] * ncell)
    nth, nz = _patch_grid(n_wall_patch, 2 * np.pi * radius, length)
    wp, wn, ww, wh = G.cylinder_wall_patches(radius, length, nth, nz)
    return cells, (wp, wn, ww, wh), length


def _patch_grid(npatch: int, circ: float, length: float):
    """n_theta x n_z = npatch exactly, with patches as close to square as the divisors allow."""
    target = np.sqrt(npatch * circ / length)
    divs = [d for d in range(1, npatch + 1) if npatch % d == 0 and d >= 3] or [npatch]
    nth = min(divs, key=lambda d: abs(np.log(d / target)))
    return nth, npatch // nth


def p2p_workload(ncell: int = 1857, radius: float = 50.0, n_wall_patch: int = 320,
                 max_leaf: int = 256, seed: int = SEED_P2P, p: int = 16) -> P2PWorkload:
    """FMM near-field workload: 1,857 cells x 544 + 320 patches x 121 = 1,048,928 points.

    Cells fill a radius-50 um cylinder at about 30% volume fraction; all points
    carry both an SL density f and a DL density phi, and all points are both
    sources and targets.  Points are returned in octree leaf order.
    """
    rng = rng_for(seed)
    cells, (wp, wn, ww, wh), _ = dense_cylinder_suspension(rng, ncell, radius, n_wall_patch, p=p)
    pts = np.concatenate([cells.pts, wp])
    nrm = np.concatenate([cells.nrm, wn])
    w = np.concatenate([cells.w, ww])
    h = np.concatenate([cells.h, wh])
    n = pts.shape[0]
    f = densities(rng, n)
    phi = densities(rng, n)
    tree = build_octree(pts, max_leaf)
    P = tree.perm
    return P2PWorkload(f"p2p_{n}pts_leaf{max_leaf}", pts[P], nrm[P], w[P], h[P], f[P], phi[P],
                       tree, 1.0, cells.n, wp.shape[0])


@dataclass
class BatchedWorkload:
    """S independent suspensions laid end to end.

    Suspension s owns points [susp_ptr[s], susp_ptr[s+1]); the first
    n_cell[s] of them are cell points (single-layer sources), the rest are
    wall points (double-layer sources).  Targets are all points of s.
    """
    name: str
    pts: np.ndarray
    nrm: np.ndarray
    w: np.ndarray
    h: np.ndarray
    f: np.ndarray
    phi: np.ndarray
    susp_ptr: np.ndarray
    n_cell: np.ndarray
    mu: float

    @property
    def nsusp(self) -> int:
        return int(self.susp_ptr.size - 1)

    def pairs(self) -> int:
        n = np.diff(self.susp_ptr).astype(np.int64)
        return int((n * n - n).sum())


def one_suspension(rng, orders=(12, 16, 24), max_cells: int = 64):
    """One suspension: 1-64 cells (log-uniform) of mixed order inside a cylinder wall."""
    ncell = int(round(np.exp(rng.uniform(0.0, np.log(max_cells)))))
    ncell = max(1, min(max_cells, ncell))
    ps = [int(orders[i]) for i in rng.integers(0, len(orders), size=ncell)]
    radius = rng.uniform(10.0, 30.0)
    n_wall = int(rng.integers(2000, 20001))
    return suspension_of(rng, ps, radius, n_wall)


def suspension_of(rng, ps, radius: float, n_wall: int):
    """Cells of orders ps placed in a cylinder wall of the given radius and about
    n_wall wall points (11 x 11 Clenshaw-Curtis patches)."""
    ncell = len(ps)
    vol_cell = 94.1
    inner = radius - 4.0
    length = max(16.0, ncell * vol_cell / (0.10 * np.pi * inner * inner))
    centres = G.place_in_cylinder(rng, ncell, radius - 0.2, length, G.RBC_RADIUS + 0.05)
    rots = [G.random_rotation(rng) for _ in range(ncell)]
    cells = cells_at(centres, rots, ps)
    npatch = max(1, int(round(n_wall / 121)))
    circ = 2 * np.pi * radius
    nth = max(3, int(round(np.sqrt(npatch * circ / length))))
    nz = max(1, int(round(npatch / nth)))
    wp, wn, ww, wh = G.cylinder_wall_patches(radius, length, nth, nz)
    return cells, (wp, wn, ww, wh)


def batched_workload(nsusp: int = 2048, seed: int = SEED_BATCHED, max_cells: int = 64,
                     orders=(12, 16, 24)) -> BatchedWorkload:
    seqs = np.random.SeedSequence(seed).spawn(nsusp)
    pts, nrm, w, h, f, phi = [], [], [], [], [], []
    ptr = [0]
    ncl = []
    for s in range(nsusp):
        rng = np.random.Generator(np.random.PCG64(seqs[s]))
        cells, (wp, wn, ww, wh) = one_suspension(rng, orders, max_cells)
        P = np.concatenate([cells.pts, wp])
        n = P.shape[0]
        pts.append(P)
        nrm.append(np.concatenate([cells.nrm, wn]))
        w.append(np.concatenate([cells.w, ww]))
        h.append(np.concatenate([cells.h, wh]))
        f.append(densities(rng, n))
        phi.append(densities(rng, n))
        ptr.append(ptr[-1] + n)
        ncl.append(cells.n)
    return BatchedWorkload(f"batched_{nsusp}susp", np.concatenate(pts), np.concatenate(nrm),
                           np.concatenate(w), np.concatenate(h), np.concatenate(f),
                           np.concatenate(phi), np.asarray(ptr, dtype=np.int64),
                           np.asarray(ncl, dtype=np.int64), 1.0)


@dataclass
class CheckpointWorkload:
    """A vessel wall of Clenshaw-Curtis patches with its fine discretisation
    (4^eta sub-patches per patch) and a double-layer density on the coarse
    nodes; the targets are the coarse nodes themselves (closest point = node,
    normal = node normal), as in the discretised boundary integral equation
    (Sec. 3.1, Eq. "int_eq_disc")."""
    name: str
    npatch: int
    q: int
    eta: int
    pts: np.ndarray
    nrm: np.ndarray
    w: np.ndarray
    phi: np.ndarray
    fine_pts: np.ndarray
    fine_nrm: np.ndarray
    fine_w: np.ndarray
    fine_h: np.ndarray
    hc: float

    def pairs(self, p: int) -> int:
        return int(self.fine_pts.shape[0]) * int(self.pts.shape[0]) * (p + 1)


def checkpoint_wall_workload(radius: float = 50.0, length: float = 74.0, npatch: int = 320,
                             q: int = 10, eta: int = 2, seed: int = SEED_P2P) -> CheckpointWorkload:
    """The near-field benchmark's vessel wall (radius 50 um, 320 patches of 11 x 11
    nodes) with 16 sub-patches per patch for the check-point quadrature."""
    rng = rng_for(seed + 100)
    nth, nz = _patch_grid(npatch, 2 * np.pi * radius, length)
    cp, cn, cw, ch = G.cylinder_wall_patches(radius, length, nth, nz, q)
    fp, fn, fw, fh = G.cylinder_wall_fine(radius, length, nth, nz, q, 1 << eta)
    hc = float(np.sqrt(cw.sum() / cw.size))
    return CheckpointWorkload(f"wall_{npatch}patches_q{q}_eta{eta}", npatch, q, eta, cp, cn, cw,
                              densities(rng, cp.shape[0]), fp, fn, fw, fh, hc)
