"""FP64 CPU oracle for the Stokes layer-potential sums (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The GPU library neither links nor calls it, and it
shares no code with the GPU library.  The arithmetic lives in
stokes_oracle.c (plain double loops, Neumaier-compensated); this module
compiles it with gcc and wraps it with ctypes.

Each function below follows the passage cited in stokes_oracle.c:
single layer (Eq. "sl_stokes"), double layer (Sec. 2.1), the smooth
quadrature sum (Sec. 3.1), the FMM near field restricted to U-lists
(Sec. 3.1 "Far evaluation") and the adjoint derived from those kernels.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stokes_oracle.c")
_LIB = os.path.join(_HERE, "libstokes_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "stokes_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            L.oracle_sl_scale.restype = d
            L.oracle_sl_scale.argtypes = [d]
            L.oracle_dl_scale.restype = d
            L.oracle_sl.argtypes = [i64, p, p, p, i64, p, d, p]
            L.oracle_dl.argtypes = [i64, p, p, p, p, i64, p, p]
            L.oracle_sldl.argtypes = [i64, p, p, p, p, p, i64, p, d, p]
            L.oracle_p2p.argtypes = [i64, p, p, p, p, p, i32, p, p, p, i32, d, i64, p, p]
            L.oracle_batched.argtypes = [i64, p, p, p, p, p, i32, p, p, d, i64, p, p]
            L.oracle_sldl_grad.argtypes = [i64, p, p, p, p, p, i64, p, p, d, p, p, p, p, p]
            for fn in (L.oracle_sl, L.oracle_dl, L.oracle_sldl, L.oracle_p2p, L.oracle_batched,
                       L.oracle_sldl_grad):
                fn.restype = None
            _lib = L
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int):
    """Set the OpenMP thread count for subsequent oracle calls (via omp_set_num_threads)."""
    try:
        omp = ctypes.CDLL("libgomp.so.1")
        omp.omp_set_num_threads(int(n))
    except OSError:
        os.environ["OMP_NUM_THREADS"] = str(int(n))


def sl(src, f, w, trg, mu=1.0):
    src, f, w, trg = _c(src), _c(f), _c(w), _c(trg)
    out = np.empty((trg.shape[0], 3))
    lib().oracle_sl(src.shape[0], _p(src), _p(f), _p(w), trg.shape[0], _p(trg), float(mu), _p(out))
    return out


def dl(src, nrm, phi, w, trg):
    src, nrm, phi, w, trg = _c(src), _c(nrm), _c(phi), _c(w), _c(trg)
    out = np.empty((trg.shape[0], 3))
    lib().oracle_dl(src.shape[0], _p(src), _p(nrm), _p(phi), _p(w), trg.shape[0], _p(trg), _p(out))
    return out


def sldl(src, f, nrm, phi, w, trg, mu=1.0):
    src, f, nrm, phi, w, trg = _c(src), _c(f), _c(nrm), _c(phi), _c(w), _c(trg)
    out = np.empty((trg.shape[0], 3))
    lib().oracle_sldl(src.shape[0], _p(src), _p(f), _p(nrm), _p(phi), _p(w), trg.shape[0],
                      _p(trg), float(mu), _p(out))
    return out


def p2p(pts, f, phi, nrm, w, leaf_ptr, ulist_ptr, ulist_idx, kernels=3, mu=1.0, targets=None):
    pts, f, phi, nrm, w = _c(pts), _c(f), _c(phi), _c(nrm), _c(w)
    leaf_ptr, ulist_ptr = _c(leaf_ptr, np.int32), _c(ulist_ptr, np.int32)
    ulist_idx = _c(ulist_idx, np.int32)
    tg = None if targets is None else _c(targets, np.int64)
    nt = pts.shape[0] if tg is None else tg.shape[0]
    out = np.empty((nt, 3))
    lib().oracle_p2p(pts.shape[0], _p(pts), _p(f), _p(phi), _p(nrm), _p(w), leaf_ptr.size - 1,
                     _p(leaf_ptr), _p(ulist_ptr), _p(ulist_idx), int(kernels), float(mu), nt,
                     _p(tg), _p(out))
    return out


def batched(pts, f, phi, nrm, w, susp_ptr, n_cell, mu=1.0, targets=None):
    pts, f, phi, nrm, w = _c(pts), _c(f), _c(phi), _c(nrm), _c(w)
    susp_ptr, n_cell = _c(susp_ptr, np.int64), _c(n_cell, np.int64)
    tg = None if targets is None else _c(targets, np.int64)
    nt = pts.shape[0] if tg is None else tg.shape[0]
    out = np.empty((nt, 3))
    lib().oracle_batched(pts.shape[0], _p(pts), _p(f), _p(phi), _p(nrm), _p(w), susp_ptr.size - 1,
                         _p(susp_ptr), _p(n_cell), float(mu), nt, _p(tg), _p(out))
    return out


def sldl_grad(src, f, nrm, phi, w, trg, g, mu=1.0):
    """Returns dict with grad_f, grad_phi, grad_y, grad_n, grad_x (None where not defined)."""
    src, w, trg, g = _c(src), _c(w), _c(trg), _c(g)
    f = None if f is None else _c(f)
    phi = None if phi is None else _c(phi)
    nrm = None if nrm is None else _c(nrm)
    ns, nt = src.shape[0], trg.shape[0]
    gf = np.zeros((ns, 3)) if f is not None else None
    gp = np.zeros((ns, 3)) if phi is not None else None
    gn = np.zeros((ns, 3)) if phi is not None else None
    gy, gx = np.zeros((ns, 3)), np.zeros((nt, 3))
    lib().oracle_sldl_grad(ns, _p(src), _p(f), _p(nrm), _p(phi), _p(w), nt, _p(trg), _p(g),
                           float(mu), _p(gf), _p(gp), _p(gy), _p(gn), _p(gx))
    return {"grad_f": gf, "grad_phi": gp, "grad_y": gy, "grad_n": gn, "grad_x": gx}


def sl_scale(mu=1.0) -> float:
    return lib().oracle_sl_scale(float(mu))


def dl_scale() -> float:
    return lib().oracle_dl_scale()
