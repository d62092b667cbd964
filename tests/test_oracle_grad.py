"""Pins of the oracle's analytic adjoint to central finite differences of its forward.

L = sum_i g_i . (SL[f] + DL[phi])(x_i); the gradient with respect to the
densities, source positions, normals and target positions must match FP64
central differences (h = 1e-6) of the forward to 1e-4 relative, and the
density gradients must satisfy the linearity identities <dL/df, f> = L_SL and
<dL/dphi, phi> = L_DL exactly up to rounding.
"""
import numpy as np

import oracle
from synth.workloads import random_cells_in_box, rng_for


def _case(seed=41):
    rng = rng_for(seed)
    s = random_cells_in_box(rng, 2, 18.0, 6)
    f, phi, g = (rng.uniform(-1, 1, (s.n, 3)) for _ in range(3))
    return s, f, phi, g, rng


def _loss(y, f, n, phi, w, x, g, mu):
    return float(np.sum(g * oracle.sldl(y, f, n, phi, w, x, mu)))


def test_gradients_match_central_differences():
    s, f, phi, g, rng = _case()
    mu = 0.8
    trg = s.pts + 0.3 * s.nrm  # targets off the sources so that x and y are separate inputs
    G = oracle.sldl_grad(s.pts, f, s.nrm, phi, s.w, trg, g, mu)
    h = 1e-6
    args = {"y": s.pts, "f": f, "n": s.nrm, "phi": phi, "x": trg}
    keymap = {"y": "grad_y", "f": "grad_f", "n": "grad_n", "phi": "grad_phi", "x": "grad_x"}
    for name, arr in args.items():
        ref = G[keymap[name]]
        rms = np.sqrt(np.mean(ref ** 2))
        for idx in rng.choice(arr.size, 16, replace=False):
            i, k = divmod(int(idx), 3)
            vals = []
            for sgn in (1, -1):
                a2 = dict(args)
                a2[name] = arr.copy()
                a2[name][i, k] += sgn * h
                vals.append(_loss(a2["y"], a2["f"], a2["n"], a2["phi"], s.w, a2["x"], g, mu))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - ref[i, k]) <= 1e-4 * max(abs(fd), rms), (name, i, k, fd, ref[i, k])


def test_density_gradients_are_linear_forms():
    s, f, phi, g, _ = _case(43)
    G = oracle.sldl_grad(s.pts, f, s.nrm, phi, s.w, s.pts, g, 1.0)
    lsl = np.sum(g * oracle.sl(s.pts, f, s.w, s.pts, 1.0))
    ldl = np.sum(g * oracle.dl(s.pts, s.nrm, phi, s.w, s.pts))
    assert abs(np.sum(G["grad_f"] * f) - lsl) <= 1e-12 * abs(lsl)
    assert abs(np.sum(G["grad_phi"] * phi) - ldl) <= 1e-12 * abs(ldl)
    # normals enter the double layer linearly as well
    assert abs(np.sum(G["grad_n"] * s.nrm) - ldl) <= 1e-12 * abs(ldl)


def test_translation_invariance_of_position_gradients():
    """Moving sources and targets together leaves L unchanged: sum(dL/dy) + sum(dL/dx) = 0."""
    s, f, phi, g, _ = _case(44)
    G = oracle.sldl_grad(s.pts, f, s.nrm, phi, s.w, s.pts, g, 1.0)
    tot = G["grad_y"].sum(0) + G["grad_x"].sum(0)
    scale = np.abs(G["grad_y"]).sum()
    assert np.all(np.abs(tot) <= 1e-12 * scale)
