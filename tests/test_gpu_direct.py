"""GPU parity of the direct sums against the FP64 oracle.

Bars: FP64 path rel-L2 <= 1e-12; mixed path rel-L2 <= 1e-6 (with the
maximum error relative to max|u| reported and bounded by 1e-5)."""
import numpy as np
import pytest

import oracle
from synth import workloads as W
from tests._util import cuda, max_rel, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-6


@pytest.fixture(scope="module")
def lib():
    from paper_1909_11085_gb300 import build
    build.build()
    import paper_1909_11085_gb300 as P
    return P


@pytest.fixture(scope="module")
def c1():
    return W.sl_direct_workload()


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOLMIX)])
def test_sl_self_sum_8_cells(lib, c1, precision, tol):
    ref = oracle.sl(c1.src, c1.f, c1.w, c1.trg, c1.mu)
    src, f, w, h = cuda(c1.src, c1.f, c1.w, c1.h)
    u = lib.sl(src, f, w, None, c1.mu, h=h, precision=precision).cpu().numpy()
    assert rel_l2(u, ref) <= tol, rel_l2(u, ref)
    assert max_rel(u, ref) <= 10 * tol


@pytest.fixture(scope="module")
def c2small():
    return W.dl_direct_workload(ncell=24, box=48.0, n_off=4099)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOLMIX)])
def test_dl_with_off_surface_targets(lib, c2small, precision, tol):
    c = c2small
    ref = oracle.dl(c.src, c.nrm, c.phi, c.w, c.trg)
    src, nrm, phi, w, h, trg = cuda(c.src, c.nrm, c.phi, c.w, c.h, c.trg)
    u = lib.dl(src, nrm, phi, w, trg, h=h, precision=precision).cpu().numpy()
    assert rel_l2(u, ref) <= tol, rel_l2(u, ref)
    assert max_rel(u, ref) <= 10 * tol


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOLMIX)])
def test_sldl_superposition(lib, c2small, precision, tol):
    c = c2small
    ref = oracle.sldl(c.src, c.f, c.nrm, c.phi, c.w, c.trg, 0.7)
    src, f, nrm, phi, w, h, trg = cuda(c.src, c.f, c.nrm, c.phi, c.w, c.h, c.trg)
    u = lib.sldl(src, f, nrm, phi, w, trg, 0.7, h=h, precision=precision).cpu().numpy()
    assert rel_l2(u, ref) <= tol, rel_l2(u, ref)


def test_constant_density_identity_on_gpu(lib):
    """D[c] = -c inside a closed cell (off-surface targets), through the GPU path."""
    s = W.random_cells_in_box(W.rng_for(3), 1, 12.0, 32)
    c = np.array([0.4, -1.1, 0.7])
    inside = W.interior_targets(s, 8)
    src, nrm, phi, w, h, trg = cuda(s.pts, s.nrm, np.tile(c, (s.n, 1)), s.w, s.h, inside)
    for prec, tol in (("fp64", 1e-6), ("mixed", 2e-6)):
        u = lib.dl(src, nrm, phi, w, trg, h=h, precision=prec).cpu().numpy()
        assert np.abs(u + c).max() <= tol


# (5000, 300) and (1000, 4000): the one-launch small form with many strided
# source splits whose counts differ by one, and targets that end mid-block
@pytest.mark.parametrize("ns,nt", [(1, 1), (1, 130), (7, 3), (129, 257), (300, 1000), (2, 0),
                                   (5000, 300), (1000, 4000)])
def test_ragged_sizes(lib, ns, nt):
    rng = W.rng_for(100 + ns + nt)
    y = rng.uniform(-3, 3, (ns, 3))
    x = rng.uniform(-3, 3, (nt, 3))
    f = rng.uniform(-1, 1, (ns, 3))
    phi = rng.uniform(-1, 1, (ns, 3))
    n = rng.normal(size=(ns, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    w = rng.uniform(0.1, 1.0, ns)
    h = np.full(ns, 0.3)
    ref = oracle.sldl(y, f, n, phi, w, x, 1.0)
    Y, F, N, PH, Wt, H, X = cuda(y, f, n, phi, w, h, x)
    for prec, tol in (("fp64", TOL64), ("mixed", TOLMIX)):
        u = lib.sldl(Y, F, N, PH, Wt, X, 1.0, h=H, precision=prec).cpu().numpy()
        assert u.shape == (nt, 3)
        if nt:
            assert rel_l2(u, ref) <= tol


def test_empty_sources_zero_and_accumulate(lib):
    import torch
    x = torch.rand(50, 3, dtype=torch.float64, device="cuda")
    y = torch.zeros(0, 3, dtype=torch.float64, device="cuda")
    w = torch.zeros(0, dtype=torch.float64, device="cuda")
    u = lib.sl(y, y, w, x)
    assert torch.all(u == 0)
    base = torch.rand(50, 3, dtype=torch.float64, device="cuda")
    u2 = lib.sl(y, y, w, x, out=base.clone(), accumulate=True)
    assert torch.equal(u2, base)


def test_accumulate_adds(lib, c1):
    import torch
    src, f, w, h = cuda(c1.src, c1.f, c1.w, c1.h)
    base = torch.rand(c1.src.shape[0], 3, dtype=torch.float64, device="cuda")
    u = lib.sl(src, f, w, None, 1.0, h=h, precision="fp64")
    u2 = lib.sl(src, f, w, None, 1.0, h=h, precision="fp64", out=base.clone(), accumulate=True)
    assert torch.allclose(u2, base + u, rtol=0, atol=1e-14)


def test_coincident_points_and_no_spacing(lib):
    """Duplicate points (zero distance) contribute nothing, with or without h."""
    rng = W.rng_for(7)
    y = rng.uniform(-1, 1, (40, 3))
    y = np.concatenate([y, y[:10]])
    f = rng.uniform(-1, 1, (50, 3))
    w = np.ones(50)
    ref = oracle.sl(y, f, w, y, 1.0)
    Y, F, Wt = cuda(y, f, w)
    for prec in ("fp64", "mixed"):
        u = lib.sl(Y, F, Wt, None, 1.0, h=None, precision=prec).cpu().numpy()
        assert np.all(np.isfinite(u))
        assert rel_l2(u, ref) <= (TOL64 if prec == "fp64" else TOLMIX)


def test_far_offset_translation(lib, c1):
    """Mixed path accuracy is set by local frames, not by absolute coordinates."""
    off = np.array([1.0e4, -2.5e4, 7.0e3])
    ref = oracle.sl(c1.src, c1.f, c1.w, c1.trg, 1.0)
    src, f, w, h = cuda(c1.src + off, c1.f, c1.w, c1.h)
    u = lib.sl(src, f, w, None, 1.0, h=h, precision="mixed").cpu().numpy()
    assert rel_l2(u, ref) <= TOLMIX


@pytest.mark.parametrize("splits", [1, 3, 17])
def test_source_splits_and_determinism(lib, c1, splits):
    import torch
    src, f, w, h = cuda(c1.src, c1.f, c1.w, c1.h)
    a = lib.sl(src, f, w, None, 1.0, h=h, source_splits=splits)
    b = lib.sl(src, f, w, None, 1.0, h=h, source_splits=splits)
    assert torch.equal(a, b)
    ref = oracle.sl(c1.src, c1.f, c1.w, c1.trg, 1.0)
    assert rel_l2(a.cpu().numpy(), ref) <= TOLMIX


def test_dl_full_size_sampled(lib):
    """256 cells (139,264 sources) x 204,800 targets, as benchmarked; 512 targets checked."""
    c = W.dl_direct_workload()
    src, nrm, phi, w, h, trg = cuda(c.src, c.nrm, c.phi, c.w, c.h, c.trg)
    rng = W.rng_for(9)
    pick = np.sort(rng.choice(c.trg.shape[0], 512, replace=False))
    ref = oracle.dl(c.src, c.nrm, c.phi, c.w, c.trg[pick])
    for prec, tol in (("mixed", TOLMIX), ("fp64", TOL64)):
        u = lib.dl(src, nrm, phi, w, trg, h=h, precision=prec).cpu().numpy()
        assert rel_l2(u[pick], ref) <= tol, (prec, rel_l2(u[pick], ref))


def test_nearly_coincident_pairs_take_the_fp64_path(lib):
    """Pairs 1e-9 apart: the near path keeps full relative accuracy (no FP32 overflow)."""
    rng = W.rng_for(17)
    y = rng.uniform(-1, 1, (64, 3))
    x = y + 1e-9 * rng.normal(size=(64, 3))
    f, phi = rng.uniform(-1, 1, (64, 3)), rng.uniform(-1, 1, (64, 3))
    n = rng.normal(size=(64, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    w = np.ones(64)
    h = np.full(64, 0.1)
    ref = oracle.sldl(y, f, n, phi, w, x, 1.0)
    Y, F, N, PH, Wt, H, X = cuda(y, f, n, phi, w, h, x)
    u = lib.sldl(Y, F, N, PH, Wt, X, 1.0, h=H, precision="mixed").cpu().numpy()
    assert np.all(np.isfinite(u))
    assert rel_l2(u, ref) <= 1e-6


@pytest.mark.parametrize("splits", [1, 3])
def test_dense_cluster_all_pairs_near(lib, splits):
    """3,001 points in a ball of radius 1 with spacing 5: every pair is near, so
    every item holds more candidate sources than the engine lists for the near
    kernel, which then scans the item's sources itself."""
    rng = W.rng_for(23)
    n = 3001
    y = rng.normal(size=(n, 3))
    y /= np.maximum(1.0, np.linalg.norm(y, axis=1))[:, None]
    f, phi = rng.uniform(-1, 1, (n, 3)), rng.uniform(-1, 1, (n, 3))
    nr = rng.normal(size=(n, 3))
    nr /= np.linalg.norm(nr, axis=1)[:, None]
    w = rng.uniform(0.5, 1.5, n)
    h = np.full(n, 5.0)
    ref = oracle.sldl(y, f, nr, phi, w, y, 1.0)
    Y, F, N, PH, Wt, H = cuda(y, f, nr, phi, w, h)
    u = lib.sldl(Y, F, N, PH, Wt, Y, 1.0, h=H, precision="mixed",
                 source_splits=splits).cpu().numpy()
    assert rel_l2(u, ref) <= TOLMIX, rel_l2(u, ref)
