"""On-disk cache of work-item shapes chosen by the library's autotuners.

The autotuners (stokes_autotune_p2p / stokes_autotune_batched in the C ABI)
time every work-item shape on the caller's inputs and return the fastest.
The choice depends on the GPU, the precision and the problem's size class,
so it is cached in a JSON file keyed by those; a later plan with the same key
reuses it without timing anything.  cache=None disables the cache.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

_lock = threading.Lock()


def _bucket(n: int) -> int:
    """Size class: the power of two at or above n."""
    return 1 << max(0, math.ceil(math.log2(max(1, int(n)))))


def key(form: str, opts, n: int, groups: int, kernels: int) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    prec = "mixed" if opts.precision == 1 else "fp64"
    return f"{dev}|{form}|{prec}|k{kernels}|n{_bucket(n)}|g{_bucket(groups)}|a{opts.near_ratio:g}"


def lookup(path, k):
    if not path or not os.path.exists(path):
        return None
    with _lock, open(path) as fh:
        try:
            data = json.load(fh)
        except json.JSONDecodeError:
            return None
    entry = data.get(k)
    return None if entry is None else int(entry["config"])


def store(path, k, config: int, ms: float):
    if not path:
        return
    with _lock:
        data = {}
        if os.path.exists(path):
            with open(path) as fh:
                try:
                    data = json.load(fh)
                except json.JSONDecodeError:
                    data = {}
        data[k] = {"config": int(config), "ms": float(ms)}
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
