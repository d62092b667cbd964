"""Brute-force oracle of the near-zone search (test infrastructure).

Only the tests and the benchmark's CPU-baseline leg may import this module;
the GPU library neither links nor calls it.

Sec. 3.2 ("closest point" search, steps a-e) finds, for each target x, the
patch of the surface closest to x when x lies within the near zone d_eps of
the surface, with the closest point y = P(u*, v*) and its parameters.  The
GPU path gets there through inflated bounding boxes, a spatial hash and a
per-candidate Newton iteration; this oracle states the result directly:
  * a patch P is the image of [-1, 1]^2 under the degree-q tensor-product
    interpolant through its (q+1) x (q+1) Clenshaw-Curtis nodes
    (u_i, v_j) = (cos(i pi/q), cos(j pi/q)), node index i (q+1) + j;
  * dist(x, P) = min over (u, v) in [-1, 1]^2 of |x - P(u, v)|, found by a
    dense grid over the parameter square followed by a bounded quasi-Newton
    refinement (scipy's L-BFGS-B) from the best grid point;
  * the answer is the patch of least distance if that distance is at most
    d_eps (ties to the lower patch index), else none (-1).
The unit normal reported at y is (dP/du x dP/dv) / |dP/du x dP/dv|.
"""
from __future__ import annotations

import numpy as np


def _cc(q):
    return np.cos(np.pi * np.arange(q + 1) / q)


def _bary_weights(q):
    return np.array([(-1.0) ** i * (0.5 if i in (0, q) else 1.0) for i in range(q + 1)])


def lagrange(q: int, t):
    """Values and first derivatives of the q+1 Lagrange basis polynomials on the
    CC nodes at the points t (rows), from the polynomial's definition: the
    basis is the unique degree-q interpolant of the unit vectors; derivatives
    by the product rule on l_i(t) = prod_{k != i} (t - x_k) / (x_i - x_k)."""
    x = _cc(q)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    L = np.ones((t.size, q + 1))
    D = np.zeros((t.size, q + 1))
    for i in range(q + 1):
        others = [k for k in range(q + 1) if k != i]
        den = np.prod([x[i] - x[k] for k in others])
        fac = np.stack([t - x[k] for k in others], axis=1)  # [nt, q]
        L[:, i] = np.prod(fac, axis=1) / den
        for a in range(q):
            D[:, i] += np.prod(np.delete(fac, a, axis=1), axis=1) / den
    return L, D


def patch_eval(nodes, q: int, u, v):
    """P(u, v), dP/du, dP/dv for one patch (nodes [(q+1)^2, 3])."""
    X = np.asarray(nodes).reshape(q + 1, q + 1, 3)
    Lu, Du = lagrange(q, u)
    Lv, Dv = lagrange(q, v)
    P = np.einsum("ti,tj,ijc->tc", Lu, Lv, X)
    Pu = np.einsum("ti,tj,ijc->tc", Du, Lv, X)
    Pv = np.einsum("ti,tj,ijc->tc", Lu, Dv, X)
    return P, Pu, Pv


def closest_on_patch(nodes, q: int, x, grid: int = 41):
    """(distance, u, v, y) of the point of the patch closest to x."""
    from scipy.optimize import minimize

    g = np.linspace(-1.0, 1.0, grid)
    U, V = np.meshgrid(g, g, indexing="ij")
    P, _, _ = patch_eval(nodes, q, U.ravel(), V.ravel())
    d2 = ((P - x) ** 2).sum(1)
    k = int(np.argmin(d2))
    u0, v0 = U.ravel()[k], V.ravel()[k]

    def fun(z):
        P1, Pu, Pv = patch_eval(nodes, q, z[0], z[1])
        r = P1[0] - x
        return float(r @ r), np.array([2.0 * r @ Pu[0], 2.0 * r @ Pv[0]])

    res = minimize(fun, np.array([u0, v0]), jac=True, method="L-BFGS-B",
                   bounds=[(-1.0, 1.0), (-1.0, 1.0)],
                   options={"ftol": 1e-15, "gtol": 1e-13, "maxiter": 200})
    u, v = res.x
    y, _, _ = patch_eval(nodes, q, u, v)
    return float(np.linalg.norm(y[0] - x)), float(u), float(v), y[0]


def near_patch_search(nodes, npatch: int, q: int, targets, d_eps: float):
    """For each target: (patch or -1, u, v, y[3], n[3], distance)."""
    nodes = np.asarray(nodes).reshape(npatch, (q + 1) ** 2, 3)
    targets = np.asarray(targets)
    nt = targets.shape[0]
    patch = np.full(nt, -1, dtype=np.int64)
    uv = np.zeros((nt, 2))
    y = np.zeros((nt, 3))
    n = np.zeros((nt, 3))
    dist = np.full(nt, np.inf)
    for t in range(nt):
        best = (np.inf, -1, 0.0, 0.0, None)
        for p in range(npatch):
            d, u, v, yy = closest_on_patch(nodes[p], q, targets[t])
            if d < best[0]:
                best = (d, p, u, v, yy)
        if best[0] <= d_eps:
            d, p, u, v, yy = best
            patch[t], uv[t], y[t], dist[t] = p, (u, v), yy, d
            _, Pu, Pv = patch_eval(nodes[p], q, u, v)
            c = np.cross(Pu[0], Pv[0])
            n[t] = c / np.linalg.norm(c)
    return patch, uv, y, n, dist
