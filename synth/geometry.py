"""Seeded surface geometry for the synthetic workloads.

This module builds the quadrature points, outward unit normals, quadrature
weights and local spacings on which the Stokes layer potentials are summed.
It contains no part of the potentials themselves: it only describes the
surfaces (red blood cells, spheres, vessel-wall patches), exactly as an
application would hand them to the summation code.

Discretisations follow the paper's setup (Sec. 2.2 "Overall
Discretization", Sec. 5 "Discretization and example setup"):
  * a red blood cell is a spherical-harmonic surface sampled on the
    latitude-longitude grid of order p: p+1 Gauss-Legendre latitudes in
    t = cos(theta) times 2p uniform longitudes ((p+1)*2p points, 544 at p=16);
  * the vessel wall is a set of tensor-product patches, each sampled at
    11 x 11 Clenshaw-Curtis nodes (121 points per patch).
The cell shape is the Evans-Fung biconcave profile with R = 3.91 um.
"""
from __future__ import annotations

import numpy as np

RBC_RADIUS = 3.91
# Evans-Fung profile coefficients: z = 0.5 R cos(theta) (c0 + c1 s + c2 s^2), s = sin^2(theta)
EF_C0, EF_C1, EF_C2 = 0.2072, 2.0026, -1.1228


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [-1, 1]."""
    return np.polynomial.legendre.leggauss(n)


def clenshaw_curtis(n: int):
    """Clenshaw-Curtis rule with n+1 nodes cos(k pi / n) on [-1, 1], n even.

    Weights from the cosine-series form of the rule: w_k = (c_k / n) *
    (1 - sum_{j=1}^{n/2} b_j cos(2 j k pi / n) / (4 j^2 - 1)), with c_k = 1 at
    the two end points and 2 elsewhere, b_j = 1 for j = n/2 and 2 otherwise.
    """
    if n < 2 or n % 2:
        raise ValueError("clenshaw_curtis needs an even n >= 2")
    k = np.arange(n + 1)
    x = np.cos(np.pi * k / n)
    w = np.zeros(n + 1)
    for kk in range(n + 1):
        s = 1.0
        for j in range(1, n // 2 + 1):
            b = 1.0 if j == n // 2 else 2.0
            s -= b * np.cos(2.0 * j * kk * np.pi / n) / (4.0 * j * j - 1.0)
        c = 1.0 if kk in (0, n) else 2.0
        w[kk] = c * s / n
    return x, w


def sph_grid(p: int):
    """Latitude-longitude grid of order p.

    Returns (theta, phi, w_t) flattened over the (p+1) x 2p grid (latitude
    major): theta from the Gauss-Legendre nodes in t = cos(theta), phi_k =
    2 pi k / (2p), and w_t = (2 pi / 2p) * w_GL, the weight in (t, phi).
    """
    t, wgl = gauss_legendre(p + 1)
    nphi = 2 * p
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    theta = np.arccos(t)
    TH, PH = np.meshgrid(theta, phi, indexing="ij")
    WT, _ = np.meshgrid(wgl * (2.0 * np.pi / nphi), phi, indexing="ij")
    return TH.ravel(), PH.ravel(), WT.ravel()


def rbc_map(theta, phi, R: float = RBC_RADIUS):
    """Evans-Fung biconcave surface X(theta, phi) and its two tangents.

    x = R sin(theta) cos(phi), y = R sin(theta) sin(phi),
    z = 0.5 R cos(theta) (c0 + c1 s + c2 s^2) with s = sin^2(theta).
    Returns X, X_theta, X_phi, each of shape [..., 3].
    """
    st, ct = np.sin(theta), np.cos(theta)
    sp, cp = np.sin(phi), np.cos(phi)
    s = st * st
    g = EF_C0 + EF_C1 * s + EF_C2 * s * s
    dg_ds = EF_C1 + 2.0 * EF_C2 * s
    X = np.stack([R * st * cp, R * st * sp, 0.5 * R * ct * g], axis=-1)
    # d/dtheta of 0.5 R cos(theta) g(sin^2 theta)
    dz = 0.5 * R * (-st * g + ct * dg_ds * 2.0 * st * ct)
    Xt = np.stack([R * ct * cp, R * ct * sp, dz], axis=-1)
    Xp = np.stack([-R * st * sp, R * st * cp, np.zeros_like(st)], axis=-1)
    return X, Xt, Xp


def sphere_map(theta, phi, a: float = 1.0):
    st, ct = np.sin(theta), np.cos(theta)
    sp, cp = np.sin(phi), np.cos(phi)
    X = np.stack([a * st * cp, a * st * sp, a * ct], axis=-1)
    Xt = np.stack([a * ct * cp, a * ct * sp, -a * st], axis=-1)
    Xp = np.stack([-a * st * sp, a * st * cp, np.zeros_like(st)], axis=-1)
    return X, Xt, Xp


def _surface_from_map(mapping, p: int, **kw):
    theta, phi, wt = sph_grid(p)
    X, Xt, Xp = mapping(theta, phi, **kw)
    cr = np.cross(Xt, Xp)
    jac = np.linalg.norm(cr, axis=-1)
    nrm = cr / jac[:, None]
    # dA = |X_theta x X_phi| dtheta dphi and dtheta = -dt / sin(theta)
    w = wt * jac / np.sin(theta)
    return X, nrm, w


def rbc_surface(p: int = 16, R: float = RBC_RADIUS):
    """One cell in its body frame: points [(p+1)2p, 3], outward normals, weights."""
    return _surface_from_map(rbc_map, p, R=R)


def sphere_surface(p: int, a: float = 1.0):
    """Sphere of radius a on the order-p grid: points, outward normals, weights."""
    return _surface_from_map(sphere_map, p, a=a)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a unit quaternion (Shoemake's method)."""
    u1, u2, u3 = rng.random(3)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    qx, qy = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    qz, qw = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def rotation_about_axis(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def place_in_box(rng, n: int, box: float, r_bound: float, gap: float = 0.2,
                 max_tries: int = 200000) -> np.ndarray:
    """Random centres in [r_bound, box - r_bound]^3 whose bounding spheres do not touch."""
    centres = []
    tries = 0
    dmin = 2.0 * r_bound + gap
    while len(centres) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place cells; box too small")
        c = rng.uniform(r_bound, box - r_bound, size=3)
        if centres:
            d = np.linalg.norm(np.asarray(centres) - c, axis=1)
            if d.min() < dmin:
                continue
        centres.append(c)
    return np.asarray(centres)


def place_in_cylinder(rng, n: int, radius: float, length: float, r_bound: float,
                      gap: float = 0.2, max_tries: int = 200000) -> np.ndarray:
    """Random centres inside a cylinder along z (axis through the origin) by rejection."""
    centres = []
    tries = 0
    dmin = 2.0 * r_bound + gap
    rmax = radius - r_bound - gap
    if rmax <= 0:
        raise ValueError("cylinder too thin for the cells")
    while len(centres) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place cells; cylinder too small")
        x, y = rng.uniform(-rmax, rmax, size=2)
        if x * x + y * y > rmax * rmax:
            continue
        z = rng.uniform(r_bound, length - r_bound)
        c = np.array([x, y, z])
        if centres:
            d = np.linalg.norm(np.asarray(centres) - c, axis=1)
            if d.min() < dmin:
                continue
        centres.append(c)
    return np.asarray(centres)


def cylinder_wall_patches(radius: float, length: float, n_theta: int, n_z: int, q: int = 10):
    """Cylinder x^2 + y^2 = radius^2, 0 <= z <= length, as n_theta x n_z patches.

    Each patch is a tensor-product Clenshaw-Curtis grid with q+1 nodes per
    direction ((q+1)^2 = 121 points at q = 10), the vessel discretisation of
    the paper's setup.  Normals point radially outward (out of the fluid that
    fills the vessel).  Points are grouped patch by patch.  Returns
    (points, normals, weights, spacing) with spacing the per-patch
    sqrt(area / points).
    """
    xc, wc = clenshaw_curtis(q)
    dth = 2.0 * np.pi / n_theta
    dz = length / n_z
    pts, nrm, wts, hs = [], [], [], []
    U, V = np.meshgrid(xc, xc, indexing="ij")
    WU, WV = np.meshgrid(wc, wc, indexing="ij")
    u, v = U.ravel(), V.ravel()
    wuv = (WU * WV).ravel()
    npp = u.size
    for iz in range(n_z):
        for it in range(n_theta):
            # shared patch edges coincide exactly, including the seam at theta = 0
            th = np.mod(it + 0.5 * (u + 1.0), n_theta) * dth
            z = (iz + 0.5 * (v + 1.0)) * dz
            c, s = np.cos(th), np.sin(th)
            pts.append(np.stack([radius * c, radius * s, z], axis=-1))
            nrm.append(np.stack([c, s, np.zeros_like(c)], axis=-1))
            # area element radius dtheta dz; the map from [-1,1]^2 has Jacobian (dth/2)(dz/2)
            w = wuv * radius * (dth / 2.0) * (dz / 2.0)
            wts.append(w)
            hs.append(np.full(npp, np.sqrt(w.sum() / npp)))
    return (np.concatenate(pts), np.concatenate(nrm), np.concatenate(wts),
            np.concatenate(hs))


# --------------------------------------------------------------- patch surfaces
# Patch surfaces for the check-point quadrature (Sec. 3.1, "Singular and
# near-singular integral quadrature").  Every patch is the image of
# [-1, 1]^2; its coarse nodes are the (q+1) x (q+1) Clenshaw-Curtis nodes
# (u_i, v_j) = (cos(i pi / q), cos(j pi / q)), ordered i-major.  The fine
# discretisation splits each patch into m x m square sub-patches (m = 2^eta,
# k = 4^eta sub-patches) with the same node set on each; fine nodes are
# ordered by patch, then sub-patch (su-major), then node (i-major).  A
# sub-patch (su, sv) covers u in [-1 + 2 su/m, -1 + 2 (su+1)/m] and likewise
# in v.  Weights are the tensor-product Clenshaw-Curtis weights times the
# area element; spacings are sqrt(area / nodes) per (sub-)patch.

def _patch_grid_nodes(q: int, m: int):
    """Parameter values of the nodes of the m x m sub-patches, as (m*m, q+1) u and v arrays
    (sub-patch su-major) together with the 1-D CC weights scaled to a sub-interval."""
    x, w = clenshaw_curtis(q)
    us, vs = [], []
    for su in range(m):
        for sv in range(m):
            ua, va = -1.0 + 2.0 * su / m, -1.0 + 2.0 * sv / m
            us.append(ua + (x + 1.0) / m)
            vs.append(va + (x + 1.0) / m)
    return np.array(us), np.array(vs), w / m


def _patches_from_map(mapping, npatch: int, q: int, m: int):
    us, vs, w1 = _patch_grid_nodes(q, m)
    WU, WV = np.meshgrid(w1, w1, indexing="ij")
    wuv = (WU * WV).ravel()
    pts, nrm, wts, hs = [], [], [], []
    for pch in range(npatch):
        for s in range(m * m):
            U, V = np.meshgrid(us[s], vs[s], indexing="ij")
            P, N, J = mapping(pch, U.ravel(), V.ravel())
            w = wuv * J
            pts.append(P)
            nrm.append(N)
            wts.append(w)
            hs.append(np.full(w.size, np.sqrt(w.sum() / w.size)))
    return (np.concatenate(pts), np.concatenate(nrm), np.concatenate(wts),
            np.concatenate(hs))


# the six faces of the cube as (axis, sign)
_CUBE_FACES = ((2, 1.0), (2, -1.0), (0, 1.0), (0, -1.0), (1, 1.0), (1, -1.0))


def _cubed_sphere_map(a: float):
    def mapping(pch, u, v):
        ax, sg = _CUBE_FACES[pch]
        o = [(ax + 1) % 3, (ax + 2) % 3]  # cyclic axes: dP/du x dP/dv points outward
        c = np.zeros((u.size, 3))
        c[:, ax] = sg
        c[:, o[0]] = u
        c[:, o[1]] = v * sg
        r = np.linalg.norm(c, axis=1)
        n = c / r[:, None]
        # gnomonic projection of a cube face: area element a^2 / |c|^3
        return a * n, n, a * a / r ** 3
    return mapping


def cubed_sphere_patches(a: float = 1.0, q: int = 10, m: int = 1):
    """Sphere of radius a as 6 gnomonic cube-face patches; m = 1 gives the coarse
    nodes, m = 2^eta the fine discretisation.  Returns (points, normals,
    weights, spacing)."""
    return _patches_from_map(_cubed_sphere_map(a), 6, q, m)


def cylinder_wall_fine(radius: float, length: float, n_theta: int, n_z: int, q: int = 10,
                       m: int = 4):
    """The fine discretisation of cylinder_wall_patches (same patch order)."""
    dth, dz = 2.0 * np.pi / n_theta, length / n_z

    def mapping(pch, u, v):
        iz, it = divmod(pch, n_theta)
        th = np.mod(it + 0.5 * (u + 1.0), n_theta) * dth
        z = (iz + 0.5 * (v + 1.0)) * dz
        c, s = np.cos(th), np.sin(th)
        return (np.stack([radius * c, radius * s, z], axis=-1),
                np.stack([c, s, np.zeros_like(c)], axis=-1),
                np.full(u.size, radius * (dth / 2.0) * (dz / 2.0)))
    return _patches_from_map(mapping, n_theta * n_z, q, m)
