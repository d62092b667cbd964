"""FP64 oracle of the check-point quadrature (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module; the GPU library neither links nor calls it.

It evaluates a layer potential at targets on or near a patch surface by the
steps of Sec. 3.1 ("Singular and near-singular integral quadrature"), in that
order, in plain FP64 numpy:
  1. upsample the density from each patch's (q+1) x (q+1) Clenshaw-Curtis
     nodes to the fine discretisation (k = 4^eta sub-patches per patch, the
     same node set on each) by tensor-product polynomial interpolation;
  2. the closest point y on the surface and the unit normal n there are
     inputs (for a target on a node, y is the node itself);
  3. check points c_i = y - (R + i r) n, i = 0..p;
  4. the velocity at the check points by the smooth quadrature
     (Eq. "smooth_double_layer_int_eq_patches_disc") on the fine
     discretisation -- the direct sums of stokes_oracle.c;
  5. 1-D polynomial extrapolation of those values along the line to the
     target: u(x) = sum_i e_i u(c_i), e_i the Lagrange weights of the nodes
     t_i = R + i r evaluated at the target's t = (y - x) . n.
Node orderings are those of synth.geometry's patch surfaces.
"""
from __future__ import annotations

import numpy as np

from . import dl as _dl, sl as _sl, sldl as _sldl


def cc_nodes(q: int) -> np.ndarray:
    """Clenshaw-Curtis (Chebyshev extreme) nodes cos(i pi / q), i = 0..q."""
    return np.cos(np.pi * np.arange(q + 1) / q)


def interp_matrix(q: int, t) -> np.ndarray:
    """Rows: the degree-q interpolant through the CC nodes evaluated at t
    (second barycentric form; weights (-1)^i, halved at the two ends)."""
    x = cc_nodes(q)
    w = np.array([(-1.0) ** i * (0.5 if i in (0, q) else 1.0) for i in range(q + 1)])
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    M = np.zeros((t.size, q + 1))
    for a, ta in enumerate(t):
        d = ta - x
        hit = np.flatnonzero(d == 0.0)
        if hit.size:
            M[a, hit[0]] = 1.0
        else:
            c = w / d
            M[a] = c / c.sum()
    return M


def fine_nodes_1d(q: int, m: int) -> np.ndarray:
    """Parameter values of the nodes of m sub-intervals of [-1, 1], sub-interval-major."""
    x = cc_nodes(q)
    return np.concatenate([-1.0 + 2.0 * s / m + (x + 1.0) / m for s in range(m)])


def upsample(v, npatch: int, q: int, m: int) -> np.ndarray:
    """Step 1: values [npatch * (q+1)^2, c] on the coarse nodes -> values on the
    fine nodes [npatch * m^2 * (q+1)^2, c]."""
    v = np.asarray(v, dtype=np.float64)
    c = v.shape[1]
    U1 = interp_matrix(q, fine_nodes_1d(q, m))               # [m(q+1), q+1]
    v = v.reshape(npatch, q + 1, q + 1, c)
    f = np.einsum("ai,pijc,bj->pabc", U1, v, U1)              # [npatch, m(q+1), m(q+1), c]
    f = f.reshape(npatch, m, q + 1, m, q + 1, c).transpose(0, 1, 3, 2, 4, 5)
    return np.ascontiguousarray(f.reshape(npatch * m * m * (q + 1) ** 2, c))


def extrapolation_weights(tn, t) -> np.ndarray:
    """Step 5: Lagrange weights of the nodes tn evaluated at t."""
    tn = np.asarray(tn, dtype=np.float64)
    e = np.ones(tn.size)
    for i in range(tn.size):
        for j in range(tn.size):
            if j != i:
                e[i] *= (t - tn[j]) / (tn[i] - tn[j])
    return e


def check_points(y, n, R: float, r: float, p: int) -> np.ndarray:
    """Step 3: c_i = y - (R + i r) n, as [nt, p+1, 3]."""
    tn = R + r * np.arange(p + 1)
    return np.asarray(y)[:, None, :] - tn[None, :, None] * np.asarray(n)[:, None, :]


def checkpoint_eval(kernels: int, f, phi, npatch: int, q: int, m: int, fine_pts, fine_nrm,
                    fine_w, trg, y, n, R: float, r: float, p: int, mu: float = 1.0) -> np.ndarray:
    """Velocity at the targets (kernels 1 = SL[f], 2 = DL[phi], 3 = both)."""
    nt = np.asarray(trg).shape[0]
    c = check_points(y, n, R, r, p).reshape(-1, 3)
    if kernels == 1:
        uc = _sl(fine_pts, upsample(f, npatch, q, m), fine_w, c, mu)
    elif kernels == 2:
        uc = _dl(fine_pts, fine_nrm, upsample(phi, npatch, q, m), fine_w, c)
    else:
        uc = _sldl(fine_pts, upsample(f, npatch, q, m), fine_nrm, upsample(phi, npatch, q, m),
                   fine_w, c, mu)
    uc = uc.reshape(nt, p + 1, 3)
    tn = R + r * np.arange(p + 1)
    tx = np.einsum("tk,tk->t", np.asarray(y) - np.asarray(trg), np.asarray(n))
    out = np.empty((nt, 3))
    for i in range(nt):
        out[i] = extrapolation_weights(tn, tx[i]) @ uc[i]
    return out


def null_space_term(phi, nodes_n, nodes_w, trg_n) -> np.ndarray:
    """(N phi)(x) = sum_m w_m (n(x) . phi_m) n_m, the rank-completing operator of
    Eq. "double_layer_int_eq" discretised on the coarse nodes: M = sum_m w_m n_m
    phi_m^T (3 x 3), then N phi(x) = M n(x)."""
    M = np.einsum("m,mi,mj->ij", np.asarray(nodes_w), np.asarray(nodes_n), np.asarray(phi))
    return np.asarray(trg_n) @ M.T


def bie_matvec(phi, npatch: int, q: int, m: int, nodes, nodes_n, nodes_w, fine_pts, fine_nrm,
               fine_w, R: float, r: float, p: int) -> np.ndarray:
    """The boundary-integral operator of Eq. "double_layer_int_eq" / "int_eq_disc"
    applied to a density on the coarse nodes, at the coarse nodes: the limit of
    the double layer from the fluid side (check points c = y - (R + i r) n,
    extrapolated to the node) plus N phi.  With the kernel orientation of this
    build (a constant density gives -c on the fluid side) that limit is
    (D - I/2) phi; the paper's +I/2 belongs to the opposite orientation of n."""
    u = checkpoint_eval(2, None, phi, npatch, q, m, fine_pts, fine_nrm, fine_w, nodes, nodes,
                        nodes_n, R, r, p)
    return u + null_space_term(phi, nodes_n, nodes_w, nodes_n)
