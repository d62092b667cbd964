#!/usr/bin/env python
"""Benchmark of the Stokes layer-potential hot path on GB300.

Workload (one "step"): the FMM near field of the paper's method (Sec. 3.1
"Far evaluation"), i.e. P2P over octree U-lists of single- plus double-layer
sums, on 1,048,928 synthetic points (1,857 red blood cells at p = 16 packed
at about 30% volume fraction in a radius-50 um vessel, plus 320 wall patches
of 121 points), leaves of at most 256 points.  One step is one full call of
stokes_p2p_leaflists (pack, work-item build and sort, engine, scatter) with
inputs resident in HBM.  The FP64 form runs on the same inputs for
comparison; accuracy of both is measured against the FP64 CPU oracle on a
sample of targets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own copy of the workload
(independent units, no data-path collective): weak scaling.  With --shard the
one workload is split over the ranks instead (strong scaling): target leaves
balanced by pair count, a one-off halo, one all_gather per step.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpair-interactions/s + % FP32 peak, mixed vs FP64 on one GB300 at stated rel-L2 error"
UNIT = "Gpair/s"
# Algorithmic FP32 flops per (target, source) pair by the fixed convention of
# the measurement plan (FMA = 2, rsqrt not counted): a single-layer pair 28
# (d 3, r^2 5, r^-3 2, d.q 5, scale 1, two 3-vector FMAs 12), a double-layer
# pair 29 (d 3, r^2 5, r^-2 1, d.n 5, d.psi 5, products and r^-5 4, one 3-vector
# FMA 6); a pair of the SL + DL step carries both, 57.
FLOPS_PER_PAIR = {"SL": 28, "DL": 29, "SLDL": 57}
# What the kernels execute per pair: SL 27 (r^-3 folded into the final FMA),
# DL 29, SL + DL 40 (d, r^2 and r^-2 shared: d 3, r^2 5, r^-2 1, d.q 5, d.psi 5,
# d.n 5, (d.psi)(d.n) 1, combine 2 + 1, two 3-vector FMAs 12).
EXEC_FLOPS_PER_PAIR = {"SL": 27, "DL": 29, "SLDL": 40}
FLOPS_PER_PAIR_SLDL = FLOPS_PER_PAIR["SLDL"]
# The same convention with the difference d (3) and |r|^2 (5) counted once for
# the fused SL + DL pair, which evaluates them once for both kernels: 49.
FUSED_FLOPS_PER_PAIR = FLOPS_PER_PAIR_SLDL - 8
# The adjoint's pair terms as stated (and written) for both kernels, counted the
# same way: shared d 3, |r|^2 5, r^-2, r^-3, r^-5 3, d.g 5; source-major pass
# + single layer 48 + double layer 55 + 3 = 122; target-major pass + 35 + 43 + 3 = 97.
ADJ_FLOPS_PER_PAIR = {"src": 122, "trg": 97}
FP32_LANES_PER_SM = 128
# near-pair threshold: |r| < NEAR_RATIO * h_j takes the FP64 difference and 1/r
NEAR_RATIO = 1.0
L2_FLUSH_BYTES = 256 << 20
ENGINE_SOURCES = ["paper_1909_11085_gb300/csrc/engine_mixed.cu",
                  "paper_1909_11085_gb300/csrc/common.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "engine_mixed_p2p_traffic.txt")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def engine_sha() -> str:
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic():
    """DRAM bytes per engine launch from the committed ncu summary, if it is current."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("engine_source_sha256_16") != engine_sha():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, util, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                s, m, u = float(parts[0]), float(parts[1]), float(parts[3])
            except ValueError:
                continue
            sm.append(s)
            mx.append(m)
            util.append(u)
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        loaded = [s for s, u in zip(sm, util) if u >= 50] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "samples_under_load": len([u for u in util if u >= 50])}


class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, read-only queries) inside the timed region, right after each
    step is queued, while the GPU has work: the samples the 100 ms nvidia-smi
    poll misses when the whole timed region lasts a few tens of milliseconds."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device):
        self.ok, self.sm, self.reasons, self.max = False, [], set(), None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return
        if lib.nvmlInit_v2() != 0:
            return
        h = ctypes.c_void_p()
        found = False
        try:  # the CUDA device by PCI bus id (NVML may number the GPUs differently)
            import torch
            pr = torch.cuda.get_device_properties(device)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            found = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        except (AttributeError, RuntimeError):
            found = False
        if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(0), ctypes.byref(h)) != 0:
            return
        self.lib, self.h = lib, h
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:
            self.max = mx.value
        self.reason_fn = (getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or
                          getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None))
        self.ok = True

    def sample(self, busy: bool):
        if not self.ok or not busy:
            return
        c = ctypes.c_uint()
        if self.lib.nvmlDeviceGetClockInfo(self.h, ctypes.c_int(1), ctypes.byref(c)) == 0:
            self.sm.append(c.value)
        if self.reason_fn is not None:
            r = ctypes.c_ulonglong()
            if self.reason_fn(self.h, ctypes.byref(r)) == 0:
                for bit, name in self.REASONS.items():
                    if r.value & bit:
                        self.reasons.add(name)

    def merge(self, clocks: dict) -> dict:
        """The nvidia-smi record with the in-region NVML samples: the SM clock
        becomes their median, the reasons the union."""
        if not self.ok or not self.sm:
            return clocks
        out = dict(clocks)
        out["sm_mhz"] = float(statistics.median(self.sm))
        if self.max:
            out["sm_max_mhz"] = float(self.max)
        out["reasons"] = sorted(set(clocks.get("reasons") or []) | self.reasons)
        out["nvml_samples_in_region"] = len(self.sm)
        out["nvml_sm_mhz_min"] = float(min(self.sm))
        out["source"] = ("NVML after each step was queued (GPU busy), reasons from NVML and "
                         "nvidia-smi")
        return out


def oracle_sample(wl, targets):
    import oracle
    t = wl.tree
    return oracle.p2p(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3,
                      wl.mu, targets=targets)


def sample_pairs(wl, targets) -> int:
    t = wl.tree
    sz = np.diff(t.leaf_ptr).astype(np.int64)
    leaf = np.searchsorted(t.leaf_ptr, targets, side="right") - 1
    nsrc = np.array([sz[t.ulist_idx[t.ulist_ptr[b]:t.ulist_ptr[b + 1]]].sum() for b in range(t.nleaf)])
    return int(nsrc[leaf].sum())


def batched_pair_split(susp_ptr, n_cell):
    """(single-layer pairs, double-layer pairs) of a batch: every point of a
    suspension is a target of its cells' single layer and of its wall's double
    layer, the point itself excluded."""
    npt = np.diff(np.asarray(susp_ptr)).astype(np.int64)
    ncl = np.asarray(n_cell, dtype=np.int64)
    nwl = npt - ncl
    return int((npt * ncl - ncl).sum()), int((npt * nwl - nwl).sum())


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model as the kernel reports it (x86 "model name", or the
    Arm implementer / part codes), for the CPU baseline's record."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name"):
        for line in info:
            if line.split(":")[0].strip() == key:
                return line.split(":", 1)[1].strip()
    imp = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
    if imp and part:
        return f"Arm CPU implementer {imp[0]}, part {part[0]}"
    return "unknown"


def one_core_rate(wl, rng, targets: int = 200) -> float:
    """The oracle on one thread over a small target sample (Gpair/s)."""
    import oracle
    tg = np.sort(rng.choice(wl.pts.shape[0], targets, replace=False))
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle_sample(wl, tg)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(cpu_cores())
    return sample_pairs(wl, tg) / dt / 1e9


def timed_oracle(wl, seconds: float, rng):
    """Runs the oracle on a random target sample sized for about `seconds` of CPU time."""
    import oracle
    oracle.set_threads(cpu_cores())
    n = wl.pts.shape[0]
    probe = np.sort(rng.choice(n, 2000, replace=False))
    t0 = time.perf_counter()
    oracle_sample(wl, probe)
    dt = max(time.perf_counter() - t0, 1e-3)
    m = int(min(n, max(2000, 2000 * seconds / dt)))
    tg = np.sort(rng.choice(n, m, replace=False))
    t0 = time.perf_counter()
    ref = oracle_sample(wl, tg)
    dt = time.perf_counter() - t0
    return tg, ref, dt


def workload_config(wl, pairs):
    return {"workload": f"p2p_ulist_sl+dl_{wl.pts.shape[0]}pts_leaf256",
            "points": int(wl.pts.shape[0]), "cells": int(wl.n_cell_points // 544),
            "cell_order_p": 16, "wall_patches": int(wl.n_wall_points // 121),
            "leaves": int(wl.tree.nleaf),
            "ulist_entries": int(wl.tree.ulist_idx.size), "pairs_per_step": int(pairs),
            "kernels": "SL+DL", "near_ratio": NEAR_RATIO,
            "l2": "256 MiB buffer written between timed steps (outside the step events)"}


def _time_ms(fn, stream, flush, reps, warm=1):
    """Median device time of fn() over reps calls (L2 flushed before each)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ev = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def run_peaks(dev, stream):
    """Measured throughput of the pipes the kernels are bound by (the library's
    stokes_pipe_probe): FP32 FMA, packed FP32 FMA, FP64 FMA (TFLOP/s) and the
    MUFU reciprocal square root (Geval/s), each the median of 3 timed launches
    after one warm-up, with CUDA events on the launching stream."""
    import ctypes
    import torch
    from paper_1909_11085_gb300 import _abi as A
    L = A.lib()
    nb = ctypes.c_size_t(0)
    A.check(L.stokes_pipe_probe_size(ctypes.byref(nb)))
    sink = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    res = {}
    for op, name, iters, unit in ((0, "ffma", 16384, "TFLOP/s"), (1, "ffma2", 8192, "TFLOP/s"),
                                  (2, "dfma", 256, "TFLOP/s"), (3, "rsqrt", 2048, "Geval/s")):
        ops = ctypes.c_double(0)
        launch = lambda: A.check(L.stokes_pipe_probe(op, iters, A.ptr(sink), sink.numel(),
                                                      ctypes.byref(ops), A.stream_ptr(dev)))
        launch()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            launch()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        res[name] = {"value": ops.value / (ms / 1e3) / scale, "unit": unit, "ms": ms}
    log(f"[peaks] {res}")
    return res


def near_fraction(wl, tg, alpha):
    """Fraction of the (target, U-list source) pairs of the sample tg that are
    near at this alpha (|x - y| < alpha h_y, the self pair excluded)."""
    t = wl.tree
    leaf = np.searchsorted(t.leaf_ptr, tg, side="right") - 1
    near, tot = 0, 0
    for lf in np.unique(leaf):
        xs = wl.pts[tg[leaf == lf]]
        src = np.concatenate([np.arange(t.leaf_ptr[b], t.leaf_ptr[b + 1])
                              for b in t.ulist_idx[t.ulist_ptr[lf]:t.ulist_ptr[lf + 1]]])
        d2 = ((xs[:, None, :] - wl.pts[src][None, :, :]) ** 2).sum(-1)
        hh = (alpha * wl.h[src]) ** 2
        near += int(((d2 < hh[None, :]) & (d2 > 0)).sum())
        tot += int((d2 > 0).sum())
    return near / max(tot, 1)


def run_alpha_sweep(wl, dev, stream, flush, pts, f, phi, nrm, w, h, alphas=(1.0, 2.0, 4.0)):
    """The near-pair threshold alpha (|r| < alpha h_j takes the FP64 path):
    for each alpha the near-pair fraction (host-counted on a target sample),
    the P2P step time and the mixed form's rel-L2 and max error against the
    oracle on the same sample."""
    import torch
    import oracle
    import paper_1909_11085_gb300 as P
    t = wl.tree
    n = wl.pts.shape[0]
    rng = np.random.default_rng(7)
    tg = np.sort(rng.choice(n, 2000, replace=False))
    ref = oracle_sample(wl, tg)
    out = torch.empty((n, 3), dtype=torch.float64, device=dev)
    res = {"sample": f"{tg.size} random targets with all their U-list sources"}
    for a in alphas:
        plan = P.P2PPlan(n, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, "mixed", a, dev)
        ms = _time_ms(lambda: plan(pts, f, phi, nrm, w, h, wl.mu, out), stream, flush, 10, warm=2)
        plan.device_status()
        u = out.cpu().numpy()[tg]
        res[f"alpha_{a:g}"] = {
            "near_pair_fraction": near_fraction(wl, tg, a), "ms_per_step": ms,
            "Gpair/s": wl.pairs() / ms / 1e6,
            "rel_l2": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
            "max_rel": float(np.abs(u - ref).max() / np.abs(ref).max())}
        log(f"[alpha] {a}: {res[f'alpha_{a:g}']}")
        del plan
    return res


def fmm_pass_times(plan, args, out, stream, flush):
    """Device time of each pass of one mixed far-field call (the library's
    per-launch events, stokes_fmm_set_pass_events), summed per pass name."""
    import ctypes
    import torch
    from paper_1909_11085_gb300 import _abi as A
    L = A.lib()
    cap = 1024
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(cap)]
    for e in evs:
        e.record(stream)
    torch.cuda.synchronize()
    handles = (ctypes.c_void_p * cap)(*[e.cuda_event for e in evs])
    names = (ctypes.c_char_p * (cap // 2))()
    cnt = ctypes.c_int32(0)
    flush.zero_()
    A.check(L.stokes_fmm_set_pass_events(handles, cap, names, ctypes.byref(cnt)))
    try:
        plan(*args, out=out)
    finally:
        A.check(L.stokes_fmm_set_pass_events(None, 0, None, None))
    torch.cuda.synchronize()
    per = {}
    for k in range(cnt.value):
        nm = names[k].decode()
        per[nm] = per.get(nm, 0.0) + evs[2 * k].elapsed_time(evs[2 * k + 1])
    return per


def kmulp_roofline(ms, v_pairs, p, parents):
    """The spectral M2L products (tcgen05, 3xTF32) against the tensor peak:
    algorithmic work 12 complex multiply-adds = 96 flops per V-list pair and
    frequency; executed, a [128 parents] x [48] x [8 x 208 slots] real product
    per parent tile, frequency and hi/lo term (3 terms), zero blocks included."""
    if not ms:
        return None
    nf = 4 * p * p * (p + 1)
    algo = 96.0 * v_pairs * nf
    executed = 2.0 * 48 * 8 * 208 * 3 * parents * nf
    meas = {}
    try:
        meas = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    bf16 = meas.get("bf16_tflops") or 1900.0
    peak = bf16 * 1.1 / 2.25  # TF32 dense = bf16 dense x (1.1 / 2.25), nominal ratio
    ach = algo / (ms / 1e3) / 1e12
    return {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": peak,
            "frac": ach / peak, "executed_tflops": executed / (ms / 1e3) / 1e12,
            "executed_frac": executed / (ms / 1e3) / 1e12 / peak,
            "peak_basis": "TF32 dense = measured bf16 burst x 1.1 / 2.25 (of measured)",
            "flops_basis": "96 per V-list pair and frequency (12 complex multiply-adds)"}


def run_fmm_far(wl, near, near_ms_step, dev, stream, flush, p=4):
    """The whole single-GPU FMM: the far field (stokes_fmm_far_eval) on the
    near-field workload's own octree beside the timed near-field step.  Host
    set-up time (the library's octree and V, W, X lists, the same tree as the
    workload's U-lists; per-depth operators; each plan's device copies), device
    time per call in FP64 and mixed precision with dense and Fourier-space M2L,
    far + near time, and far field + the step's near field against the direct
    sum on 256 sampled targets (the FMM's approximation error at this p, not a
    parity figure)."""
    import torch
    import oracle
    from paper_1909_11085_gb300 import ops
    t0 = time.perf_counter()
    tn = ops.octree(wl.pts, 256)  # the workload's leaf size
    t = ops.fmm_tree_arrays(**ops.fmm_tree_args(tn))
    lists_s = time.perf_counter() - t0
    if not np.array_equal(tn["leaf_ptr"], wl.tree.leaf_ptr):
        raise RuntimeError("the library's octree differs from the workload's U-list tree")
    t0 = time.perf_counter()
    U, D = ops.fmm_operators(p, t["root_size"], t["max_depth"], wl.mu, True)
    ops_s = time.perf_counter() - t0
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    pts, f, phi, nrm, w = (T(a) for a in (wl.pts, wl.f, wl.phi, wl.nrm, wl.w))
    rng = np.random.default_rng(1909)
    tg = np.sort(rng.choice(wl.pts.shape[0], 256, replace=False))
    ref = oracle.sldl(wl.pts, wl.f, wl.nrm, wl.phi, wl.w, wl.pts[tg], wl.mu)
    un = near.cpu().numpy()[tg]
    res = {"p": p, "boxes": int(t["depth"].size), "leaves": int(t["leaf_box"].size),
           "max_depth": int(t["max_depth"]), "v_pairs": int(tn["v_idx"].size),
           "w_entries": int(tn["w_idx"].size), "x_entries": int(tn["x_idx"].size),
           "host_lists_s": lists_s, "host_operators_s": ops_s,
           "near_only_rel_l2": float(np.linalg.norm(un - ref) / np.linalg.norm(ref))}
    near_ms = near_ms_step
    res["near_field_ms"] = near_ms
    for prec in ("mixed", "fp64"):
        for m2l in ("fft", "dense"):
            t0 = time.perf_counter()
            plan = ops.FmmFarPlan(t, p=p, mu=wl.mu, flux=True, uc2e=U, dc2e=D, m2l=m2l,
                                  precision=prec)
            plan_s = time.perf_counter() - t0
            far = torch.zeros_like(pts)
            reps = 10 if prec == "mixed" else 2
            ms = _time_ms(lambda: plan(pts, f, phi, nrm, w, out=far), stream, flush, reps)
            u = far.cpu().numpy()[tg] + un
            key = f"{prec}_{m2l}"
            res[key] = {"far_ms": ms, "far_plus_near_ms": ms + near_ms,
                        "host_plan_s": plan_s, "workspace_MB": plan.ws.numel() / 1e6,
                        "rel_l2_vs_direct": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
                        "max_rel_vs_direct": float(np.abs(u - ref).max() / np.abs(ref).max())}
            if prec == "mixed":
                res[key]["passes_ms"] = fmm_pass_times(plan, (pts, f, phi, nrm, w), far, stream,
                                                       flush)
                if m2l == "fft":
                    res[key]["kmulp_roofline"] = kmulp_roofline(
                        res[key]["passes_ms"].get("kmulp"), int(tn["v_idx"].size), p,
                        int(np.sum(np.diff(t["child_ptr"]) > 0) - 1))
            log(f"[fmm] {key}: {res[key]}")
            del plan, far
    torch.cuda.empty_cache()
    return res


def run_nearzone(dev, flush, stream, c6=None, x6=None):
    """The near-zone search (Sec. 3.2): 2^20 points spread through the vessel
    against the 320 wall patches, d_eps = 2 h_c; on the cylinder the closest
    point is the radial projection, which checks every hit away from the open
    ends."""
    import torch
    import paper_1909_11085_gb300 as P
    from synth import workloads as W
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    if c6 is None:
        c6 = W.checkpoint_wall_workload()
        x6 = T(c6.pts)
    rng9 = np.random.default_rng(11085009)
    m9, Rv, Lv = 1 << 20, 50.0, 74.0
    rho9 = Rv * np.sqrt(rng9.uniform(0.0, 1.0, m9))
    th9 = rng9.uniform(0.0, 2.0 * np.pi, m9)
    z9 = rng9.uniform(0.0, Lv, m9)
    x9 = np.stack([rho9 * np.cos(th9), rho9 * np.sin(th9), z9], axis=1)
    d9 = 2.0 * c6.hc
    X9 = T(x9)
    ms9 = _time_ms(lambda: P.near_patch_search(x6, c6.npatch, X9, d9, c6.q), stream, flush, 3)
    p9, _, y9, _, dist9 = (t.cpu().numpy() for t in P.near_patch_search(x6, c6.npatch, X9, d9, c6.q))
    inner = (z9 > d9) & (z9 < Lv - d9)
    want = inner & (Rv - rho9 <= d9 * (1 - 1e-9))
    got = inner & (p9 >= 0)
    yref = np.stack([Rv * np.cos(th9), Rv * np.sin(th9), z9], axis=1)
    res = {
        "targets": m9, "patches": int(c6.npatch), "d_eps": d9, "ms": ms9,
        "Mtargets/s": m9 / ms9 / 1e3, "targets_within_d_eps": int((p9 >= 0).sum()),
        "closed_form": {"hit_mismatch": int((want != got).sum()),
                        "max_dist_err": float(np.abs(dist9[want & got] - (Rv - rho9[want & got])).max()),
                        "max_y_err": float(np.abs(y9[want & got] - yref[want & got]).max())},
        "note": "FP64 closest-point Newton per candidate patch; hits checked against the radial "
                "projection for targets away from the open ends"}
    log(f"[forms] near-zone search: {res}")
    del X9
    return res


def run_forms(dev, flush, stream, peak_tflops):
    """The paper's other workloads on the same GPU: direct single layer (8 cells),
    direct double layer (256 cells + 65,536 off-surface targets), 2,048 batched
    suspensions (autotuned tile, CUDA-graph replay), the check-point quadrature
    of the double layer on the 320-patch vessel wall and the adjoint of SL + DL
    (64 cells).  Each: device time per call, Gpair/s, % FP32 peak (mixed) and the
    rel-L2 error against the FP64 oracle on the stated sample."""
    import torch
    import oracle
    import paper_1909_11085_gb300 as P
    from synth import workloads as W
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    err = lambda u, r: float(np.linalg.norm(u - r) / np.linalg.norm(r))
    pct = lambda pairs, ms, kind: 100.0 * pairs * FLOPS_PER_PAIR[kind] / (ms / 1e3) / 1e12 / peak_tflops
    pct_x = lambda pairs, ms, kind: (100.0 * pairs * EXEC_FLOPS_PER_PAIR[kind] / (ms / 1e3) / 1e12
                                     / peak_tflops)
    forms = {}
    rng = np.random.default_rng(1909)

    c1 = W.sl_direct_workload()
    n1 = c1.src.shape[0]
    src, f, w, h = T(c1.src), T(c1.f), T(c1.w), T(c1.h)
    ref = oracle.sl(c1.src, c1.f, c1.w, c1.src, c1.mu)
    e = {}
    for prec in ("fp64", "mixed"):
        # a small sum is bound by its launches: replayed from a CUDA graph
        plan1 = P.DirectPlan(n1, n1, 1, prec)
        out = torch.empty((n1, 3), dtype=torch.float64, device=dev)
        g1 = plan1.capture(src, f, None, None, w, None, c1.mu, h, out)
        ms = _time_ms(lambda: g1.launch(stream), stream, flush, 20, warm=3)
        plan1.device_status()
        ms_call = _time_ms(lambda: P.sl(src, f, w, None, c1.mu, h=h, precision=prec), stream,
                           flush, 10)
        e[prec] = {"ms": ms, "ms_direct_call": ms_call, "Gpair/s": n1 * (n1 - 1) / ms / 1e6,
                   "rel_l2": err(out.cpu().numpy(), ref), "path": "graph replay (DirectPlan)"}
        del g1, plan1
    e["mixed"]["pct_fp32_peak"] = pct(n1 * (n1 - 1), e["mixed"]["ms"], "SL")
    e["mixed"]["pct_fp32_peak_executed"] = pct_x(n1 * (n1 - 1), e["mixed"]["ms"], "SL")
    forms["direct_sl_8rbc_4352pts"] = dict(pairs=n1 * (n1 - 1), sample="all targets", **e)
    log(f"[forms] direct SL: {e}")

    c2 = W.dl_direct_workload()
    ns2, nt2 = c2.src.shape[0], c2.trg.shape[0]
    src, nrm, phi, w, h, trg = (T(a) for a in (c2.src, c2.nrm, c2.phi, c2.w, c2.h, c2.trg))
    pick = np.sort(rng.choice(nt2, 512, replace=False))
    ref = oracle.dl(c2.src, c2.nrm, c2.phi, c2.w, c2.trg[pick])
    pairs2 = ns2 * nt2 - ns2
    e = {}
    for prec, reps in (("mixed", 5), ("fp64", 2)):
        out = torch.empty((nt2, 3), dtype=torch.float64, device=dev)
        ms = _time_ms(lambda: P.dl(src, nrm, phi, w, trg, h=h, precision=prec, out=out), stream,
                      flush, reps)
        e[prec] = {"ms": ms, "Gpair/s": pairs2 / ms / 1e6,
                   "rel_l2": err(out.cpu().numpy()[pick], ref)}
    e["mixed"]["pct_fp32_peak"] = pct(pairs2, e["mixed"]["ms"], "DL")
    e["mixed"]["pct_fp32_peak_executed"] = pct_x(pairs2, e["mixed"]["ms"], "DL")
    forms["direct_dl_256rbc_139264src_204800trg"] = dict(
        pairs=pairs2, sample="512 random targets", **e)
    log(f"[forms] direct DL: {e}")
    del src, nrm, phi, w, h, trg

    t0 = time.perf_counter()
    c3 = W.batched_workload()
    log(f"[forms] batched workload: {c3.pts.shape[0]} points, {c3.nsusp} suspensions, "
        f"{time.perf_counter() - t0:.1f}s")
    n3 = c3.pts.shape[0]
    pairs3 = c3.pairs()
    pts, f, phi, nrm, w, h = (T(a) for a in (c3.pts, c3.f, c3.phi, c3.nrm, c3.w, c3.h))
    # tile configuration from the autotuner, timed on the first 256 suspensions
    m = int(c3.susp_ptr[256])
    small = P.BatchedPlan(m, c3.susp_ptr[:257], c3.n_cell[:256])
    cfg = small.autotune(pts[:m], f[:m], phi[:m], nrm[:m], w[:m], h[:m], c3.mu)
    del small
    plan = P.BatchedPlan(n3, c3.susp_ptr, c3.n_cell)
    plan.opts.tile_config = cfg
    out = torch.empty((n3, 3), dtype=torch.float64, device=dev)
    graph = plan.capture(pts, f, phi, nrm, w, h, c3.mu, out)
    ms = _time_ms(lambda: graph.launch(stream), stream, flush, 3)
    plan.device_status()
    u = out.cpu().numpy()
    sus = np.sort(rng.choice(c3.nsusp, 4, replace=False))
    rows = np.concatenate([np.arange(c3.susp_ptr[s], c3.susp_ptr[s + 1]) for s in sus])
    sp = np.concatenate([[0], np.cumsum(np.diff(c3.susp_ptr)[sus])])
    refb = oracle.batched(c3.pts[rows], c3.f[rows], c3.phi[rows], c3.nrm[rows], c3.w[rows],
                          sp, c3.n_cell[sus], c3.mu)
    sl3, dl3 = batched_pair_split(c3.susp_ptr, c3.n_cell)
    fl3 = (sl3 * FLOPS_PER_PAIR["SL"] + dl3 * FLOPS_PER_PAIR["DL"]) / (ms / 1e3) / 1e12
    fx3 = (sl3 * EXEC_FLOPS_PER_PAIR["SL"] + dl3 * EXEC_FLOPS_PER_PAIR["DL"]) / (ms / 1e3) / 1e12
    forms["batched_2048_suspensions_graph"] = {
        "pairs": pairs3, "sl_pairs": sl3, "dl_pairs": dl3, "points": n3, "tile_config": cfg,
        "mixed": {"ms": ms, "Gpair/s": pairs3 / ms / 1e6, "rel_l2": err(u[rows], refb),
                  "pct_fp32_peak": 100.0 * fl3 / peak_tflops,
                  "pct_fp32_peak_executed": 100.0 * fx3 / peak_tflops},
        "sample": f"4 whole suspensions ({rows.size} targets)"}
    log(f"[forms] batched: {forms['batched_2048_suspensions_graph']}")
    del graph, plan, pts, f, phi, nrm, w, h, out
    torch.cuda.empty_cache()

    c6 = W.checkpoint_wall_workload()
    p6 = 4
    R6, r6 = 3.0 * c6.hc, c6.hc
    x6, n6, phi6 = T(c6.pts), T(c6.nrm), T(c6.phi)
    fp6, fn6, fw6, fh6 = T(c6.fine_pts), T(c6.fine_nrm), T(c6.fine_w), T(c6.fine_h)
    plan6 = P.CheckpointPlan(c6.npatch, fp6, fn6, fw6, fh6, x6, x6, n6, R6, r6, p6, c6.q, c6.eta,
                             kernels=2)
    out6 = torch.empty((c6.pts.shape[0], 3), dtype=torch.float64, device=dev)
    ms = _time_ms(lambda: plan6(None, phi6, out=out6), stream, flush, 3)
    import oracle.checkpoint as OCK
    pick = np.sort(rng.choice(c6.pts.shape[0], 32, replace=False))
    ref6 = OCK.checkpoint_eval(2, None, c6.phi, c6.npatch, c6.q, 1 << c6.eta, c6.fine_pts,
                               c6.fine_nrm, c6.fine_w, c6.pts[pick], c6.pts[pick], c6.nrm[pick],
                               R6, r6, p6)
    pairs6 = c6.pairs(p6)
    amp = float(np.abs(OCK.extrapolation_weights(R6 + r6 * np.arange(p6 + 1), 0.0)).sum())
    forms["checkpoint_dl_wall_320patches"] = {
        "pairs": pairs6, "targets": int(c6.pts.shape[0]), "fine_nodes": int(c6.fine_pts.shape[0]),
        "check_points_per_target": p6 + 1, "R_over_hc": 3.0, "r_over_hc": 1.0, "eta": c6.eta,
        "mixed": {"ms": ms, "Gpair/s": pairs6 / ms / 1e6,
                  "rel_l2": err(out6.cpu().numpy()[pick], ref6),
                  "pct_fp32_peak": pct(pairs6, ms, "DL"),
                  "pct_fp32_peak_executed": pct_x(pairs6, ms, "DL")},
        "extrapolation_amplification": amp,
        "sample": "32 random wall nodes (oracle: same steps in FP64)"}
    log(f"[forms] checkpoint: {forms['checkpoint_dl_wall_320patches']}")
    # the boundary-integral operator (D - I/2 + N) on the same wall
    w6 = T(c6.w)
    bie = P.BIEPlan(c6.npatch, x6, n6, w6, fp6, fn6, fw6, fh6, R6, r6, p6, c6.q, c6.eta)
    outb = torch.empty_like(out6)
    msb = _time_ms(lambda: bie.matvec(phi6, out=outb), stream, flush, 3)
    nterm = outb.cpu().numpy() - out6.cpu().numpy()
    nref = OCK.null_space_term(c6.phi, c6.nrm, c6.w, c6.nrm)
    forms["bie_matvec_wall_320patches"] = {
        "pairs": pairs6, "mixed": {"ms": msb, "Gpair/s": pairs6 / msb / 1e6,
                                   "null_term_rel_l2": err(nterm, nref)},
        "note": "(D - I/2 + N) phi at all 38,720 nodes; D - I/2 by the check points above"}
    log(f"[forms] bie matvec: {forms['bie_matvec_wall_320patches']}")
    del plan6, bie, fp6, fn6, fw6, fh6
    forms["nearzone_search_wall_320patches"] = run_nearzone(dev, flush, stream, c6, x6)

    c5, g5 = W.adjoint_workload()
    n5 = c5.src.shape[0]
    src, f, nrm, phi, w, h, g = (T(a) for a in (c5.src, c5.f, c5.nrm, c5.phi, c5.w, c5.h, g5))
    def fwd_bwd():
        s_, f_, n_, p_ = (t.detach().requires_grad_(True) for t in (src, f, nrm, phi))
        u = P.StokesLayerFn.apply(s_, f_, n_, p_, w, s_, c5.mu, h)
        u.backward(g)
    ms = _time_ms(fwd_bwd, stream, flush, 5)
    # forward pass + source-major and target-major adjoint passes
    pairs5 = n5 * (n5 - 1)
    fl5 = FLOPS_PER_PAIR["SLDL"] + ADJ_FLOPS_PER_PAIR["src"] + ADJ_FLOPS_PER_PAIR["trg"]
    fx5 = EXEC_FLOPS_PER_PAIR["SLDL"] + ADJ_FLOPS_PER_PAIR["src"] + ADJ_FLOPS_PER_PAIR["trg"]
    forms["adjoint_sldl_64rbc_34816pts"] = {
        "pairs_per_pass": pairs5, "passes": 3,
        "flops_per_pair": {"forward": FLOPS_PER_PAIR["SLDL"], **ADJ_FLOPS_PER_PAIR},
        "mixed": {"ms_forward_backward": ms, "Gpair/s": 3 * pairs5 / ms / 1e6,
                  "pct_fp32_peak": 100.0 * pairs5 * fl5 / (ms / 1e3) / 1e12 / peak_tflops,
                  "pct_fp32_peak_executed": 100.0 * pairs5 * fx5 / (ms / 1e3) / 1e12 / peak_tflops},
        "accuracy": "checked in the GPU test suite (oracle gradient and finite differences)"}
    log(f"[forms] adjoint: {forms['adjoint_sldl_64rbc_34816pts']}")
    return forms


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from synth import workloads as W
    wl = W.p2p_workload(ncell=args.ncell, n_wall_patch=args.wall_patches)
    pairs = wl.pairs()
    rng = np.random.default_rng(11085)
    import oracle
    oracle.build()
    oracle.set_threads(cpu_cores())
    n = wl.pts.shape[0]
    per_step = 4000
    for _ in range(args.warmup):
        oracle_sample(wl, np.sort(rng.choice(n, per_step, replace=False)))
    tot_pairs, tot_t = 0, 0.0
    for _ in range(args.steps):
        tg = np.sort(rng.choice(n, per_step, replace=False))
        t0 = time.perf_counter()
        oracle_sample(wl, tg)
        tot_t += time.perf_counter() - t0
        tot_pairs += sample_pairs(wl, tg)
    val = tot_pairs / tot_t / 1e9
    sample = f"{per_step} random targets per step (all their U-list sources), {args.steps} steps"
    line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, pairs),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, rank, world, local_rank):
    """--shard: the one 1,048,928-point near-field step split over the ranks
    (strong scaling): shard.ShardedP2P partitions the target leaves by pair
    count with a one-off halo of U-list source leaves (copied to each GPU
    before the timed region); each timed step is the local P2P call plus the
    NCCL all_gather that assembles the full velocity on every rank.  value =
    the global pairs per step x K / the slowest rank's time.  e2e repeats the
    steps with each rank's inputs copied in from pinned host memory and the
    assembled velocity read back every step."""
    import torch
    import torch.distributed as dist
    import paper_1909_11085_gb300 as P
    from paper_1909_11085_gb300 import shard as S
    from synth import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        from paper_1909_11085_gb300 import build as B
        B.build()
    dist.barrier()
    wl = W.p2p_workload(ncell=args.ncell, n_wall_patch=args.wall_patches)
    t = wl.tree
    pairs = wl.pairs()
    bufs = {}

    def make_eval(sh):
        plan = P.P2PPlan(sh.n_local, sh.leaf_ptr, sh.ulist_ptr, sh.ulist_idx, 3, "mixed",
                         NEAR_RATIO, dev)
        bufs["out"] = torch.empty((sh.n_local, 3), dtype=torch.float64, device=dev)
        bufs["plan"] = plan
        return lambda L: plan(L["pts"], L["f"], L["phi"], L["nrm"], L["w"], L["h"], wl.mu,
                              bufs["out"])

    sp = S.ShardedP2P(wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.h, t.leaf_ptr, t.ulist_ptr,
                      t.ulist_idx, world, rank, make_eval, dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 0)):
        sp.step()
    torch.cuda.synchronize()
    bufs["plan"].device_status()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    dist.barrier()
    from paper_1909_11085_gb300 import _abi as A
    nvml = NvmlClocks(dev)
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    launches0 = A.lib().stokes_launch_count()
    for i in range(K):
        flush.zero_()
        ev[i][0].record(stream)
        full = sp.step()
        ev[i][1].record(stream)
        nvml.sample(not stream.query())
    torch.cuda.synchronize()
    launches = A.lib().stokes_launch_count() - launches0
    clocks = nvml.merge(sampler.stop())
    dist.barrier()
    bufs["plan"].device_status()
    tot = torch.tensor([sum(a.elapsed_time(b) for a, b in ev) / 1e3], dtype=torch.float64,
                       device=dev)
    dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    tot_s = float(tot.item())
    # e2e: inputs from pinned host memory every step, full result read back
    r = sp.shard.rows
    host = {k: torch.as_tensor(np.ascontiguousarray(getattr(wl, k)[r]),
                               dtype=torch.float64).pin_memory()
            for k in ("pts", "f", "phi", "nrm", "w", "h")}
    res_host = torch.empty((wl.pts.shape[0], 3), dtype=torch.float64).pin_memory()
    Ke = max(3, min(K, 20))
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        for k, v in host.items():
            sp.local[k].copy_(v, non_blocking=True)
        full = sp.step()
        res_host.copy_(full, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    te = torch.tensor([e0.elapsed_time(e1) / 1e3 / Ke], dtype=torch.float64, device=dev)
    dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())
    counts = torch.tensor([sp.pairs], dtype=torch.int64, device=dev)
    allc = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(allc, counts)
    per_rank = [int(x.item()) for x in allc]
    # accuracy of the assembled result on a target sample (rank 0)
    acc = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        oracle.set_threads(cpu_cores())
        tg = np.sort(np.random.default_rng(20191).choice(wl.pts.shape[0], 2000, replace=False))
        ref = oracle_sample(wl, tg)
        u = full.cpu().numpy()[tg]
        acc = {"vs": "FP64 CPU oracle, 2000 random targets of the assembled result",
               "mixed_rel_l2": float(np.linalg.norm(u - ref) / np.linalg.norm(ref))}
    if rank != 0:
        return 0
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    result = {"metric": METRIC, "value": pairs * K / tot_s / 1e9, "unit": UNIT, "n_gpus": world,
              "steps": K, "warmup": args.warmup, "ms_per_step": tot_s / K * 1e3,
              "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
              "dtype": "f32 (f64 near pairs)", "data": "synthetic",
              "config": dict(workload_config(wl, pairs), parallelism=f"target leaves x{world}"),
              "shard": {"pairs_per_rank": per_rank,
                        "balance_max_over_min": max(per_rank) / max(min(per_rank), 1),
                        "halo": "U-list source leaves of each rank's target leaves, copied once",
                        "gather": "one NCCL all_gather of the owned rows per step"},
              "comm_nranks": world,
              "e2e": {"value": pairs / e2e_s / 1e9, "unit": UNIT,
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(res_host.numel() * 8),
                      "ms_per_step": e2e_s * 1e3, "steps": Ke},
              "gpu_launches": int(launches), "clocks": clocks}
    if acc:
        result["accuracy"] = acc
    print(json.dumps(result), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        from paper_1909_11085_gb300 import build as B
        B.build()
        import oracle
        oracle.build()
    if world > 1:
        dist.barrier()
    import paper_1909_11085_gb300 as P
    from paper_1909_11085_gb300 import _abi as A
    from synth import workloads as W

    t0 = time.perf_counter()
    wl = W.p2p_workload(ncell=args.ncell, n_wall_patch=args.wall_patches)
    pairs = wl.pairs()
    log(f"[rank {rank}] workload {wl.pts.shape[0]} pts, {wl.tree.nleaf} leaves, {pairs} pairs, "
        f"{time.perf_counter() - t0:.1f}s")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    pts, f, phi, nrm, w, h = (T(a) for a in (wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.h))
    t = wl.tree
    n = wl.pts.shape[0]
    plan = P.P2PPlan(n, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, "mixed", NEAR_RATIO, dev)
    plan64 = P.P2PPlan(n, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, "fp64", NEAR_RATIO, dev)
    out = torch.empty((n, 3), dtype=torch.float64, device=dev)
    out64 = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    L = A.lib()
    step = lambda: plan(pts, f, phi, nrm, w, h, wl.mu, out)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    plan.device_status()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    eng = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    stream = torch.cuda.current_stream(dev)
    for a, b in eng:  # materialise the event handles before passing them to the library
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    peaks = run_peaks(dev, stream) if not args.no_peaks else None
    nvml = NvmlClocks(dev)
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    launches0 = L.stokes_launch_count()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.zero_()
        ev[i][0].record(stream)
        L.stokes_set_engine_events(eng[i][0].cuda_event, eng[i][1].cuda_event)
        step()
        ev[i][1].record(stream)
        nvml.sample(not stream.query())
    L.stokes_set_engine_events(None, None)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = L.stokes_launch_count() - launches0
    clocks = nvml.merge(sampler.stop())
    if world > 1:
        dist.barrier()
    plan.device_status()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    eng_ms = [a.elapsed_time(b) for a, b in eng]
    tot_s = sum(step_ms) / 1e3
    if world > 1:
        tt = torch.tensor([tot_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tot_s = float(tt.item())
    value = pairs * K * world / tot_s / 1e9

    # FP64 form on the same inputs
    K64 = max(2, min(5, K))
    plan64(pts, f, phi, nrm, w, h, wl.mu, out64)
    torch.cuda.synchronize()
    e64 = []
    for _ in range(K64):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan64(pts, f, phi, nrm, w, h, wl.mu, out64)
        b.record(stream)
        e64.append((a, b))
    torch.cuda.synchronize()
    plan64.device_status()
    ms64 = sum(a.elapsed_time(b) for a, b in e64) / K64
    value64 = pairs / (ms64 / 1e3) / 1e9

    # end to end through the public API: pinned host inputs -> device -> result -> host
    host = {k: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64).pin_memory()
            for k, v in (("pts", wl.pts), ("f", wl.f), ("phi", wl.phi), ("nrm", wl.nrm),
                         ("w", wl.w), ("h", wl.h))}
    host_lists = {k: torch.as_tensor(v, dtype=torch.int32).pin_memory()
                  for k, v in (("leaf_ptr", t.leaf_ptr), ("ulist_ptr", t.ulist_ptr),
                               ("ulist_idx", t.ulist_idx))}
    out_host = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    dbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + \
        sum(v.numel() * v.element_size() for v in host_lists.values())
    d2h = out_host.numel() * out_host.element_size()
    Ke = max(3, min(K, 20))
    e2e = []
    for i in range(Ke + 2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k, v in host.items():
            dbuf[k].copy_(v, non_blocking=True)
        plan.leaf_ptr.copy_(host_lists["leaf_ptr"], non_blocking=True)
        plan.ulist_ptr.copy_(host_lists["ulist_ptr"], non_blocking=True)
        plan.ulist_idx.copy_(host_lists["ulist_idx"], non_blocking=True)
        plan(dbuf["pts"], dbuf["f"], dbuf["phi"], dbuf["nrm"], dbuf["w"], dbuf["h"], wl.mu, out)
        out_host.copy_(out, non_blocking=True)
        b.record(stream)
        if i >= 2:
            e2e.append((a, b))
    torch.cuda.synchronize()
    serial_ms = sum(a.elapsed_time(b) for a, b in e2e) / len(e2e)

    # the same steps as a stream of inputs: the host -> device copies of step
    # i + 1 run on a copy stream while step i computes (two plans and two sets
    # of device buffers, taken in turn); every step still copies its own
    # inputs in and its result out, and the time is steps / total time
    plans = [plan, P.P2PPlan(n, t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, "mixed", NEAR_RATIO, dev)]
    dbufs = [dbuf, {k: torch.empty_like(v, device=dev) for k, v in host.items()}]
    outs = [out, torch.empty_like(out)]
    out_hosts = [out_host, torch.empty_like(out_host).pin_memory()]
    plans[1](dbufs[0]["pts"], dbufs[0]["f"], dbufs[0]["phi"], dbufs[0]["nrm"], dbufs[0]["w"],
             dbufs[0]["h"], wl.mu, outs[1])  # first call of the second plan, untimed
    cstream = torch.cuda.Stream(dev)
    done = [None, None]

    def copy_in(sidx):
        with torch.cuda.stream(cstream):
            if done[sidx] is not None:
                cstream.wait_event(done[sidx])  # the buffers' previous step has finished
            for k, v in host.items():
                dbufs[sidx][k].copy_(v, non_blocking=True)
            plans[sidx].leaf_ptr.copy_(host_lists["leaf_ptr"], non_blocking=True)
            plans[sidx].ulist_ptr.copy_(host_lists["ulist_ptr"], non_blocking=True)
            plans[sidx].ulist_idx.copy_(host_lists["ulist_idx"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cstream)
        return ev

    Kp = max(4, min(K, 40))
    dstream = torch.cuda.Stream(dev)  # device -> host reads of the results
    read = [None, None]
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    cstream.wait_event(p0)
    copied = copy_in(0)
    for i in range(Kp):
        sidx = i % 2
        stream.wait_event(copied)
        if read[sidx] is not None:
            stream.wait_event(read[sidx])  # the result buffer's previous read is done
        copied = copy_in(1 - sidx) if i + 1 < Kp else None
        b_ = dbufs[sidx]
        plans[sidx](b_["pts"], b_["f"], b_["phi"], b_["nrm"], b_["w"], b_["h"], wl.mu, outs[sidx])
        ev = torch.cuda.Event()
        ev.record(stream)
        done[sidx] = ev
        with torch.cuda.stream(dstream):
            dstream.wait_event(ev)
            out_hosts[sidx].copy_(outs[sidx], non_blocking=True)
            rv = torch.cuda.Event()
            rv.record(dstream)
            read[sidx] = rv
    stream.wait_event(read[(Kp - 1) % 2])
    p1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = p0.elapsed_time(p1) / Kp
    # both buffer sets computed the same inputs: a copy that raced its step
    # would show as different bits
    same_bits = bool(torch.equal(out_hosts[0], out_hosts[1]))
    e2e_s = e2e_ms / 1e3
    if world > 1:
        tt = torch.tensor([e2e_s, serial_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s, serial_ms = float(tt[0].item()), float(tt[1].item())
    e2e_val = pairs * world / e2e_s / 1e9

    # roofline of the dominant kernel (FP32 ALU bound)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    eng_avg_s = sum(eng_ms) / K / 1e3
    achieved = pairs * FLOPS_PER_PAIR_SLDL / eng_avg_s / 1e12
    achieved_x = pairs * EXEC_FLOPS_PER_PAIR["SLDL"] / eng_avg_s / 1e12
    at_clock = None
    if clocks.get("sm_mhz"):
        at_clock = achieved / (sms * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12)

    # the FP64 form against the measured FP64 FMA rate, flops by the same convention
    fp64_line = {"value": value64, "unit": UNIT, "ms_per_step": ms64, "steps": K64}
    if peaks:
        a64 = pairs * FLOPS_PER_PAIR_SLDL / (ms64 / 1e3) / 1e12
        fp64_line["roofline"] = {
            "bound": "fp64", "achieved": a64, "peak": peaks["dfma"]["value"], "unit": "TFLOP/s",
            "frac": a64 / peaks["dfma"]["value"], "flops_per_pair": FLOPS_PER_PAIR_SLDL,
            "peak_basis": "measured FP64 FMA rate (stokes_pipe_probe op 2)",
            "note": "the FP64 form also spends FP64-pipe work on 1/sqrt (no FP64 rsqrt unit), "
                    "which the convention does not count"}

    if rank != 0:
        return 0
    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
              "warmup": args.warmup, "ms_per_step": tot_s / K * 1e3, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 near pairs)",
              "data": "synthetic", "config": workload_config(wl, pairs),
              "pct_fp32_peak": 100.0 * achieved / peak,
              "pct_fp32_peak_executed": 100.0 * achieved_x / peak,
              "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": measured_traffic(),
                           "kernel": "k_engine_mixed",
                           "engine_ms_per_launch": eng_avg_s * 1e3,
                           "flops_per_pair": FLOPS_PER_PAIR_SLDL,
                           "flops_per_pair_basis": "algorithmic, fixed convention: SL 28 + DL 29",
                           "executed_flops_per_pair": EXEC_FLOPS_PER_PAIR["SLDL"],
                           "frac_executed": achieved_x / peak,
                           "frac_49": pairs * FUSED_FLOPS_PER_PAIR / eng_avg_s / 1e12 / peak,
                           "frac_49_whole_step": pairs * FUSED_FLOPS_PER_PAIR / (tot_s / K) / 1e12
                           / peak,
                           "frac_49_basis": "d and |r|^2 counted once for the fused SL+DL pair: "
                                            "57 - 8 = 49 flops",
                           "frac_whole_step": achieved * eng_avg_s / (tot_s / K) / peak,
                           "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                           "frac_at_sampled_clock": at_clock},
              "fp64": fp64_line,
              "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                      "steps": Kp, "serial_ms_per_step": serial_ms,
                      "results_identical_across_buffers": same_bits,
                      "overlap": "host->device copies of step i+1 and the device->host read "
                                 "of step i-1 on their own streams during step i; the serial "
                                 "figure copies, computes and reads back one step at a time"},
              "gpu_launches": int(launches), "gpu_launches_per_step": launches / K,
              "clocks": clocks, "wall_s_timed_region": wall}
    if peaks:
        peaks["fp32_peak_from_ffma_frac_of_nominal"] = peaks["ffma"]["value"] / peak
        result["peaks"] = peaks
    if world == 1 and not args.no_forms:
        result["forms"] = run_forms(dev, flush, stream, peak)
    if world == 1 and not args.no_fmm:
        result["fmm_far"] = run_fmm_far(wl, out, tot_s / K * 1e3, dev, stream, flush)
    if world == 1 and not args.no_alpha:
        result["near"] = run_alpha_sweep(wl, dev, stream, flush, pts, f, phi, nrm, w, h)
    if world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(20191)
        tg, ref, dt = timed_oracle(wl, args.cpu_seconds, rng)
        sp = sample_pairs(wl, tg)
        um = out.cpu().numpy()[tg]
        u64 = out64.cpu().numpy()[tg]
        err = lambda u: float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
        mx = lambda u: float(np.abs(u - ref).max() / np.abs(ref).max())
        result["cpu_baseline"] = {"value": sp / dt / 1e9, "unit": UNIT, "cores": cpu_cores(),
                                  "kind": "oracle", "cpu_model": cpu_model(),
                                  "one_core_value": one_core_rate(wl, rng),
                                  "sample": (f"all {tg.size} targets" if tg.size == wl.pts.shape[0]
                                             else f"{tg.size} random targets of {wl.pts.shape[0]}")
                                            + f" with all their U-list sources ({sp} pairs), "
                                            f"{dt:.1f} s"}
        result["accuracy"] = {"vs": "FP64 CPU oracle on the cpu_baseline target sample",
                              "mixed_rel_l2": err(um), "mixed_max_rel": mx(um),
                              "fp64_rel_l2": err(u64), "fp64_max_rel": mx(u64)}
    print(json.dumps(result), flush=True)
    return 0


def run_only_form(args, dev, flush, stream):
    """One of the other forms alone, at a size small enough for a full ncu
    capture: the 4,352-point direct single layer (one-launch small form) and the
    same sum on the work-item engine; 128 batched suspensions; the check-point
    double layer on the 320-patch wall; the adjoint of SL + DL (34,816 points);
    the P2P step of the --ncell / --wall-patches workload in FP64."""
    import torch
    import paper_1909_11085_gb300 as P
    from synth import workloads as W
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    res = {}
    if args.only == "direct":
        c1 = W.sl_direct_workload()
        src, f, w, h = T(c1.src), T(c1.f), T(c1.w), T(c1.h)
        n1 = c1.src.shape[0]
        res["small_form_ms"] = _time_ms(lambda: P.sl(src, f, w, None, c1.mu, h=h), stream, flush, 10)
        # an explicit split count keeps the work-item engine
        res["engine_ms"] = _time_ms(lambda: P.sl(src, f, w, None, c1.mu, h=h, source_splits=16),
                                    stream, flush, 10)
        res["pairs"] = n1 * (n1 - 1)
    elif args.only == "batched":
        c3 = W.batched_workload(nsusp=128)
        pts, f, phi, nrm, w, h = (T(a) for a in (c3.pts, c3.f, c3.phi, c3.nrm, c3.w, c3.h))
        plan = P.BatchedPlan(c3.pts.shape[0], c3.susp_ptr, c3.n_cell)
        out = torch.empty((c3.pts.shape[0], 3), dtype=torch.float64, device=dev)
        res["ms"] = _time_ms(lambda: plan(pts, f, phi, nrm, w, h, c3.mu, out), stream, flush, 5)
        res["pairs"], res["points"] = c3.pairs(), int(c3.pts.shape[0])
    elif args.only == "checkpoint":
        c6 = W.checkpoint_wall_workload()
        p6, R6, r6 = 4, 3.0 * c6.hc, c6.hc
        x6, n6, phi6 = T(c6.pts), T(c6.nrm), T(c6.phi)
        fp6, fn6, fw6, fh6 = T(c6.fine_pts), T(c6.fine_nrm), T(c6.fine_w), T(c6.fine_h)
        plan6 = P.CheckpointPlan(c6.npatch, fp6, fn6, fw6, fh6, x6, x6, n6, R6, r6, p6, c6.q,
                                 c6.eta, kernels=2)
        out6 = torch.empty((c6.pts.shape[0], 3), dtype=torch.float64, device=dev)
        res["ms"] = _time_ms(lambda: plan6(None, phi6, out=out6), stream, flush, 3)
        res["pairs"] = c6.pairs(p6)
    elif args.only == "adjoint":
        c5, g5 = W.adjoint_workload()
        src, f, nrm, phi, w, h, g = (T(a) for a in (c5.src, c5.f, c5.nrm, c5.phi, c5.w, c5.h, g5))

        def fwd_bwd():
            s_, f_, n_, p_ = (t.detach().requires_grad_(True) for t in (src, f, nrm, phi))
            P.StokesLayerFn.apply(s_, f_, n_, p_, w, s_, c5.mu, h).backward(g)
        res["ms_forward_backward"] = _time_ms(fwd_bwd, stream, flush, 3)
        res["pairs_per_pass"] = c5.src.shape[0] * (c5.src.shape[0] - 1)
    else:  # p2p in FP64
        wl = W.p2p_workload(ncell=args.ncell, n_wall_patch=args.wall_patches)
        t = wl.tree
        plan = P.P2PPlan(wl.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, "fp64",
                         NEAR_RATIO, dev)
        a_ = tuple(T(a) for a in (wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.h))
        out = torch.empty((wl.pts.shape[0], 3), dtype=torch.float64, device=dev)
        res["fp64_ms"] = _time_ms(lambda: plan(*a_, wl.mu, out), stream, flush, 2)
    return res


def run_only(args):
    """One form alone (see --only)."""
    import torch
    from paper_1909_11085_gb300 import build as B
    B.build()
    import oracle
    oracle.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if args.only == "nearzone":
        res = run_nearzone(dev, flush, stream)
    elif args.only in ("direct", "batched", "checkpoint", "adjoint", "p2p"):
        res = run_only_form(args, dev, flush, stream)
    else:
        import paper_1909_11085_gb300 as P
        from synth import workloads as W
        wl = W.p2p_workload(ncell=args.ncell, n_wall_patch=args.wall_patches)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        t = wl.tree
        near = torch.empty((wl.pts.shape[0], 3), dtype=torch.float64, device=dev)
        plan = P.P2PPlan(wl.pts.shape[0], t.leaf_ptr, t.ulist_ptr, t.ulist_idx, 3, "mixed",
                         NEAR_RATIO, dev)
        args_ = tuple(T(a) for a in (wl.pts, wl.f, wl.phi, wl.nrm, wl.w, wl.h))
        ms = _time_ms(lambda: plan(*args_, wl.mu, near), stream, flush, 5)
        res = run_fmm_far(wl, near, ms, dev, stream, flush)
    print(json.dumps({"only": args.only, "result": res}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncell", type=int, default=1857,
                    help="cells of the near-field workload (464 with --wall-patches 80 gives "
                         "the 262,096-point case used for ncu captures)")
    ap.add_argument("--wall-patches", type=int, default=320)
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other workloads (direct, batched, adjoint)")
    ap.add_argument("--no-fmm", action="store_true",
                    help="skip the FMM's far field (FP64 and mixed passes, dense and "
                         "Fourier-space M2L) on the near-field workload's octree")
    ap.add_argument("--no-alpha", action="store_true",
                    help="skip the near-pair threshold sweep (alpha = 1, 2, 4)")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the measured FP32 / FP64 / MUFU pipe rates")
    ap.add_argument("--only", choices=["fmm", "nearzone", "direct", "batched", "checkpoint",
                                       "adjoint", "p2p"], default=None,
                    help="run one form alone and print its JSON (profiling helper: small device "
                         "footprint): the FMM far field beside the near field of the --ncell / "
                         "--wall-patches workload, the near-zone search, the small direct sum, "
                         "128 batched suspensions, the check-point wall, the adjoint, or the "
                         "FP64 P2P step")
    ap.add_argument("--shard", action="store_true",
                    help="split the one near-field step over the ranks (strong scaling: target "
                         "leaves by pair count, a one-off halo, an all_gather per step) instead "
                         "of a replica per rank; run under torchrun")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only:
        return run_only(args)
    dist_on = world > 1 or args.shard
    if dist_on:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group("nccl", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local_rank))
    try:
        if args.shard:
            return run_sharded(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if dist_on:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
