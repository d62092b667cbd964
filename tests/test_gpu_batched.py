"""GPU parity of the batched suspensions (one persistent launch) against the oracle."""
import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests._util import cuda, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    return P


@pytest.fixture(scope="module")
def small():
    return W.batched_workload(nsusp=12, max_cells=6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_batched_small_all_targets(lib, small, precision, tol):
    c = small
    ref = oracle.batched(c.pts, c.f, c.phi, c.nrm, c.w, c.susp_ptr, c.n_cell, 1.0)
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    u = lib.batched(pts, f, phi, nrm, w, c.susp_ptr, c.n_cell, 1.0, h=h,
                    precision=precision).cpu().numpy()
    per = [rel_l2(u[a:b], ref[a:b]) for a, b in zip(c.susp_ptr[:-1], c.susp_ptr[1:])]
    assert rel_l2(u, ref) <= tol and max(per) <= 10 * tol, (rel_l2(u, ref), max(per))


@pytest.fixture(scope="module")
def full():
    """The 2,048-suspension workload as benchmarked (44M points)."""
    return W.batched_workload()


def _sample_targets(susp_ptr, frac, rng):
    """frac of the targets of every suspension (at least one each), sorted."""
    picks = []
    for a, b in zip(susp_ptr[:-1], susp_ptr[1:]):
        m = max(1, int(round(frac * (b - a))))
        picks.append(np.sort(rng.choice(np.arange(a, b), m, replace=False)))
    return np.concatenate(picks)


def test_batched_full_size_graph_replay_sampled(lib, full):
    """All 2,048 suspensions in one persistent launch replayed from a CUDA
    graph; 1% of the targets of every suspension against the oracle."""
    import torch
    c = full
    pts, f, phi, nrm, w, h = cuda(c.pts, c.f, c.phi, c.nrm, c.w, c.h)
    plan = lib.BatchedPlan(c.pts.shape[0], c.susp_ptr, c.n_cell, "mixed")
    out = torch.empty((c.pts.shape[0], 3), dtype=torch.float64, device="cuda")
    graph = plan.capture(pts, f, phi, nrm, w, h, c.mu, out)
    graph.launch()
    torch.cuda.synchronize()
    plan.device_status()
    tg = _sample_targets(c.susp_ptr, 0.01, W.rng_for(33))
    ref = oracle.batched(c.pts, c.f, c.phi, c.nrm, c.w, c.susp_ptr, c.n_cell, c.mu, targets=tg)
    u = out.cpu().numpy()[tg]
    assert rel_l2(u, ref) <= 1e-6, rel_l2(u, ref)
    sid = np.searchsorted(c.susp_ptr, tg, side="right") - 1
    worst = max(rel_l2(u[sid == s], ref[sid == s]) for s in np.unique(sid))
    assert worst <= 1e-5, worst


def test_batched_heaviest_and_largest_suspension(lib, full):
    """The 16 heaviest suspensions of the workload plus the largest one the
    generator allows (64 cells at p = 24, 76,800 points, and a 20,000-point
    wall) in one batch, FP64 and mixed, through the graph replay; 1% of the
    targets of each suspension against the oracle."""
    import torch
    c = full
    npt = np.diff(c.susp_ptr)
    heavy = np.sort(np.argsort(-(npt.astype(np.int64) ** 2))[:16])
    rng = W.rng_for(34)
    cells, (wp, wn, ww, wh) = W.suspension_of(rng, [24] * 64, 30.0, 20000)
    big = {"pts": np.concatenate([cells.pts, wp]), "nrm": np.concatenate([cells.nrm, wn]),
           "w": np.concatenate([cells.w, ww]), "h": np.concatenate([cells.h, wh])}
    nb = big["pts"].shape[0]
    big["f"], big["phi"] = W.densities(rng, nb), W.densities(rng, nb)
    assert cells.n == 64 * 25 * 48 and nb - cells.n >= 19000
    rows = [np.arange(c.susp_ptr[s], c.susp_ptr[s + 1]) for s in heavy]
    cat = lambda key: np.concatenate([getattr(c, key)[r] for r in rows] + [big[key]])
    P = {k: cat(k) for k in ("pts", "nrm", "w", "h", "f", "phi")}
    sp = np.concatenate([[0], np.cumsum([r.size for r in rows] + [nb])]).astype(np.int64)
    ncl = np.concatenate([c.n_cell[heavy], [cells.n]]).astype(np.int64)
    n = P["pts"].shape[0]
    tg = _sample_targets(sp, 0.01, W.rng_for(35))
    ref = oracle.batched(P["pts"], P["f"], P["phi"], P["nrm"], P["w"], sp, ncl, c.mu, targets=tg)
    pts, f, phi, nrm, w, h = cuda(P["pts"], P["f"], P["phi"], P["nrm"], P["w"], P["h"])
    for prec, tol in (("mixed", 1e-6), ("fp64", 1e-12)):
        plan = lib.BatchedPlan(n, sp, ncl, prec)
        out = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        graph = plan.capture(pts, f, phi, nrm, w, h, c.mu, out)
        graph.launch()
        torch.cuda.synchronize()
        plan.device_status()
        u = out.cpu().numpy()[tg]
        assert rel_l2(u, ref) <= tol, (prec, rel_l2(u, ref))
