"""Builds and calls the host build of the GPU far-field passes (test
infrastructure; see fmm_host_harness.cpp)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fmm_host_harness.cpp")
HDR = os.path.join(HERE, "..", "..", "paper_1909_11085_gb300", "csrc", "fmm_passes.cuh")
LIB = os.path.join(HERE, "_build", "libfmmhost.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                                    os.path.getmtime(HDR)):
            os.makedirs(os.path.dirname(LIB), exist_ok=True)
            tmp = LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, SRC])
            os.replace(tmp, LIB)
        _lib = ctypes.CDLL(LIB)
        _lib.fmm_host_far_eval.restype = ctypes.c_longlong
        _lib.fmm_host_message.restype = ctypes.c_char_p
        _lib.fmm_host_row_df.restype = ctypes.c_float
    return _lib


def row_df(a, x):
    """The mixed form's row product of an FP64 row a (split into FP32 hi + lo)
    with an FP32 vector x."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    hi = a.astype(np.float32)
    lo = (a - hi.astype(np.float64)).astype(np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    return float(lib().fmm_host_row_df(_p(hi), _p(lo), _p(x), ctypes.c_int(a.size)))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def far_eval(pts, f, phi, nrm, w, tree, p, uc2e, dc2e, mu=1.0, flux=True, out=None,
             accumulate=False, spec=None, mixed=False, blocked=True):
    """tree: dict of the arrays of the library's stk_fmm_tree (numpy, host);
    spec: M2L kernel spectra (Fourier-space M2L) or None (dense M2L);
    mixed: the FP32 evaluation passes instead of the FP64 ones; blocked: pass
    the colleague table (parent-blocked spectral products) or not (V-lists)."""
    c = lambda a, t=np.float64: None if a is None else np.ascontiguousarray(a, dtype=t)
    i = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    pts, f, phi, nrm, w = c(pts), c(f), c(phi), c(nrm), c(w)
    n = pts.shape[0]
    out = np.zeros((n, 3)) if out is None else out
    T = {k: i(v) for k, v in tree.items()
         if k not in ("root_lo", "root_size", "max_depth", "ulist_ptr", "ulist_idx")}
    colleague = T["colleague"] if blocked else None
    args = [T[k] for k in ("depth_ptr", "depth", "anchor", "parent", "child_ptr", "box_leaf",
                           "leaf_box", "leaf_ptr", "v_ptr", "v_idx", "w_ptr", "w_idx", "x_ptr",
                           "x_idx")]
    root_lo = c(tree["root_lo"])
    uc2e, dc2e, spec = c(uc2e), c(dc2e), c(spec)
    L = lib()
    r = L.fmm_host_far_eval(
        _p(pts), _p(f), _p(phi), _p(nrm), _p(w), ctypes.c_longlong(n),
        ctypes.c_int(T["depth"].size), ctypes.c_int(T["leaf_box"].size),
        ctypes.c_int(int(tree["max_depth"])), *[_p(a) for a in args], _p(colleague), _p(root_lo),
        ctypes.c_double(float(tree["root_size"])), ctypes.c_int(p), ctypes.c_int(int(flux)),
        _p(uc2e), _p(dc2e), _p(spec), ctypes.c_int(int(bool(mixed))), ctypes.c_double(mu), _p(out),
        ctypes.c_int(int(accumulate)))
    if r < 0:
        raise IndexError(L.fmm_host_message().decode())
    return out, int(r)
