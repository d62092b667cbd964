"""Host-side bookkeeping of bench.py, checked by brute force on small cases:
the pair counts behind the throughput figures, the single/double-layer split of
a batch behind its flop count, and the rule that a recorded DRAM traffic figure
is reported only while the engine sources it was measured on are unchanged."""
import os

import numpy as np

import bench
from synth import workloads as W


def test_sample_pairs_counts_ulist_sources():
    wl = W.p2p_workload(ncell=6, radius=8.0, n_wall_patch=6, max_leaf=32)
    t = wl.tree
    rng = np.random.default_rng(3)
    tg = np.sort(rng.choice(wl.pts.shape[0], 40, replace=False))
    brute = 0
    for i in tg:
        b = int(np.searchsorted(t.leaf_ptr, i, side="right") - 1)
        for a in t.ulist_idx[t.ulist_ptr[b]:t.ulist_ptr[b + 1]]:
            brute += int(t.leaf_ptr[a + 1] - t.leaf_ptr[a])
    assert bench.sample_pairs(wl, tg) == brute
    assert bench.sample_pairs(wl, np.arange(wl.pts.shape[0])) == wl.pairs()


def test_batched_pair_split_by_enumeration():
    rng = np.random.default_rng(4)
    for _ in range(5):
        sizes = rng.integers(1, 40, 6)
        n_cell = np.array([rng.integers(0, s + 1) for s in sizes])
        susp_ptr = np.concatenate([[0], np.cumsum(sizes)])
        sl = dl = 0
        for s in range(sizes.size):
            p0, p1 = int(susp_ptr[s]), int(susp_ptr[s + 1])
            for i in range(p0, p1):
                for j in range(p0, p1):
                    if i != j:
                        if j - p0 < n_cell[s]:
                            sl += 1
                        else:
                            dl += 1
        assert bench.batched_pair_split(susp_ptr, n_cell) == (sl, dl)
    c = W.batched_workload(nsusp=3, max_cells=2, orders=(12,))
    assert sum(bench.batched_pair_split(c.susp_ptr, c.n_cell)) == c.pairs()


def test_traffic_record_follows_the_engine_sources(tmp_path, monkeypatch):
    rec = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.measured_traffic() is None  # no record
    rec.write_text(f"engine_source_sha256_16: {bench.engine_sha()}\ndram_bytes_per_launch: 1234\n")
    assert bench.measured_traffic() == 1234.0
    rec.write_text("engine_source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 1234\n")
    assert bench.measured_traffic() is None  # taken on other sources
    # the committed record matches the engine sources as they stand
    monkeypatch.setattr(bench, "TRAFFIC_FILE",
                        os.path.join(os.path.dirname(bench.__file__), "profiles",
                                     "engine_mixed_p2p_traffic.txt"))
    assert bench.measured_traffic() is not None
