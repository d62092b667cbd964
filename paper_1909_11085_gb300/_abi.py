"""ctypes binding of libstokesgpu.so (the C ABI in include/stokesgpu.h).

Argument marshalling only: tensors are checked (CUDA, float64/int32/int64,
contiguous), a workspace of the size the library asks for is taken from the
PyTorch caching allocator, and the call is enqueued on the current stream.
Every arithmetic step runs in the library's kernels.  The library must have
been built (paper_1909_11085_gb300.build.build()); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstokesgpu.so")

STK_OK, STK_EINVAL, STK_ENOMEM, STK_ECUDA, STK_ETIMEOUT, STK_EUNSUPPORTED = range(6)
STK_FP64, STK_MIXED = 0, 1
SL, DL, SLDL = 1, 2, 3

EXPORTS = [
    "stokes_default_opts", "stokes_sl_eval", "stokes_dl_eval", "stokes_sldl_eval",
    "stokes_direct_workspace_size", "stokes_p2p_leaflists", "stokes_p2p_workspace_size",
    "stokes_batched_eval", "stokes_batched_workspace_size", "stokes_device_status",
    "stokes_last_error", "stokes_version", "stokes_set_engine_events", "stokes_launch_count",
    "stokes_sl_eval_noalloc", "stokes_sldl_grad", "stokes_grad_workspace_size",
    "stokes_tile_config_count", "stokes_autotune_p2p", "stokes_autotune_batched",
    "stokes_p2p_graph_create", "stokes_batched_graph_create", "stokes_graph_launch",
    "stokes_graph_destroy", "stokes_checkpoint_eval", "stokes_checkpoint_workspace_size",
    "stokes_upsample_patches", "stokes_bie_matvec", "stokes_bie_workspace_size",
    "stokes_near_patch_search", "stokes_near_search_workspace_size",
    "stokes_fmm_surface", "stokes_fmm_check_to_equiv", "stokes_fmm_kernel_matrix",
    "stokes_fmm_far_workspace_size", "stokes_fmm_far_eval", "stokes_fmm_m2l_spectra",
    "stokes_octree_build", "stokes_octree_info", "stokes_octree_export", "stokes_octree_destroy",
    "stokes_set_wait_policy", "stokes_pipe_probe_size", "stokes_pipe_probe",
    "stokes_fmm_set_pass_events", "stokes_fmm_operators", "stokes_fmm_tree_complete",
    "stokes_direct_graph_create", "stokes_convert_check",
]


class StkOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("near_ratio", ctypes.c_double),
                ("accumulate", ctypes.c_int32), ("source_splits", ctypes.c_int32),
                ("tile_config", ctypes.c_int32)]


class StkFmmTree(ctypes.Structure):
    """stk_fmm_tree: depth_ptr is a host array, every other array a device one."""
    _fields_ = [("nbox", ctypes.c_int32), ("nleaf", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("depth_ptr", ctypes.c_void_p)] + [
        (k, ctypes.c_void_p) for k in ("depth", "anchor", "parent", "child_ptr", "box_leaf",
                                       "leaf_box", "leaf_ptr", "v_ptr", "v_idx", "w_ptr", "w_idx",
                                       "x_ptr", "x_idx", "colleague")] + [
        ("root_lo", ctypes.c_double * 3), ("root_size", ctypes.c_double)]


class StkOctreeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nleaf", ctypes.c_int32), ("nbox", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("nulist", ctypes.c_int64), ("nv", ctypes.c_int64),
                ("nw", ctypes.c_int64), ("nx", ctypes.c_int64), ("root_lo", ctypes.c_double * 3),
                ("root_size", ctypes.c_double)]


class StokesError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"stokesgpu status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1909_11085_gb300.build.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            p, i32, i64, d, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_size_t)
            po = ctypes.POINTER(StkOpts)
            psz = ctypes.POINTER(ctypes.c_size_t)
            L.stokes_default_opts.argtypes = [po]
            L.stokes_default_opts.restype = None
            L.stokes_last_error.restype = ctypes.c_char_p
            L.stokes_version.restype = ctypes.c_char_p
            L.stokes_sl_eval.argtypes = [p, p, p, p, i64, p, i64, d, p, po, p, sz, p]
            L.stokes_dl_eval.argtypes = [p, p, p, p, p, i64, p, i64, p, po, p, sz, p]
            L.stokes_sldl_eval.argtypes = [p, p, p, p, p, p, i64, p, i64, d, p, po, p, sz, p]
            L.stokes_direct_workspace_size.argtypes = [i64, i64, i32, po, psz]
            L.stokes_p2p_leaflists.argtypes = [p, p, p, p, p, p, i64, p, i32, p, p, i64, i32, d, p,
                                               po, p, sz, p]
            L.stokes_p2p_workspace_size.argtypes = [i64, i32, i32, po, psz]
            L.stokes_batched_eval.argtypes = [p, p, p, p, p, p, i64, p, p, i32, d, p, po, p, sz, p]
            L.stokes_batched_workspace_size.argtypes = [i64, i32, po, psz]
            L.stokes_device_status.argtypes = [p, sz]
            L.stokes_set_engine_events.argtypes = [p, p]
            L.stokes_set_wait_policy.argtypes = [i64, i32]
            L.stokes_pipe_probe_size.argtypes = [psz]
            L.stokes_fmm_set_pass_events.argtypes = [p, i32, p, ctypes.POINTER(ctypes.c_int32)]
            L.stokes_fmm_operators.argtypes = [i32, d, i32, d, i32, d, i32, p, p]
            L.stokes_fmm_tree_complete.argtypes = [i32, i32, p, p, p, p, p, p, p, p, p]
            L.stokes_pipe_probe.argtypes = [i32, i32, p, sz, ctypes.POINTER(ctypes.c_double), p]
            L.stokes_convert_check.argtypes = [p, i64, p, p, p, p, p]
            L.stokes_sl_eval_noalloc.argtypes = [p, p, p, p, i64, p, i64, d, p, po, p]
            L.stokes_sldl_grad.argtypes = [p, p, p, p, p, p, i64, p, i64, p, d, p, p, p, p, p, po,
                                           p, sz, p]
            L.stokes_grad_workspace_size.argtypes = [i64, i64, po, psz]
            pi32, pf, pp = (ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                            ctypes.POINTER(ctypes.c_void_p))
            L.stokes_tile_config_count.restype = ctypes.c_int32
            L.stokes_autotune_p2p.argtypes = [p, p, p, p, p, p, i64, p, i32, p, p, i64, i32, d, p,
                                              po, p, sz, p, pi32, pf]
            L.stokes_autotune_batched.argtypes = [p, p, p, p, p, p, i64, p, p, i32, d, p, po, p, sz,
                                                  p, pi32, pf]
            L.stokes_p2p_graph_create.argtypes = [p, p, p, p, p, p, i64, p, i32, p, p, i64, i32, d,
                                                  p, po, p, sz, p, pp]
            L.stokes_batched_graph_create.argtypes = [p, p, p, p, p, p, i64, p, p, i32, d, p, po, p,
                                                      sz, p, pp]
            L.stokes_graph_launch.argtypes = [p, p]
            L.stokes_direct_graph_create.argtypes = [i32, p, p, p, p, p, p, i64, p, i64, d, p, po,
                                                     p, sz, p, pp]
            L.stokes_checkpoint_eval.argtypes = [i32, p, p, i32, i32, i32, p, p, p, p, p, p, p,
                                                 i64, d, d, i32, d, p, po, p, sz, p]
            L.stokes_checkpoint_workspace_size.argtypes = [i32, i32, i32, i32, i64, i32, po, psz]
            L.stokes_upsample_patches.argtypes = [p, i32, i32, i32, i32, p, p]
            L.stokes_bie_matvec.argtypes = [p, i32, i32, i32, p, p, p, p, p, p, p, d, d, i32, p,
                                            po, p, sz, p]
            L.stokes_bie_workspace_size.argtypes = [i32, i32, i32, i32, po, psz]
            L.stokes_near_patch_search.argtypes = [p, i32, i32, p, i64, d, p, p, p, p, p, p, sz,
                                                   p]
            L.stokes_near_search_workspace_size.argtypes = [i32, i32, i64, psz]
            L.stokes_fmm_surface.argtypes = [i32, p, ctypes.POINTER(ctypes.c_int32)]
            L.stokes_fmm_check_to_equiv.argtypes = [i32, d, d, i32, i32, d, p]
            L.stokes_fmm_kernel_matrix.argtypes = [p, i32, p, i32, d, i32, p]
            pt = ctypes.POINTER(StkFmmTree)
            L.stokes_fmm_far_workspace_size.argtypes = [i32, i32, i32, i32, i64, pt, psz]
            L.stokes_fmm_far_eval.argtypes = [p, p, p, p, p, i64, pt, i32, i32, p, p, p, i32, d, p,
                                              i32, p, sz, p]
            L.stokes_fmm_m2l_spectra.argtypes = [i32, d, i32, p]
            L.stokes_octree_build.argtypes = [p, i64, i32, pp]
            L.stokes_octree_info.argtypes = [p, ctypes.POINTER(StkOctreeInfo)]
            L.stokes_octree_export.argtypes = [p] * 16
            L.stokes_octree_destroy.argtypes = [p]
            L.stokes_octree_destroy.restype = None
            L.stokes_graph_destroy.argtypes = [p]
            L.stokes_launch_count.restype = ctypes.c_int64
            for name in EXPORTS:
                fn = getattr(L, name)
                if name not in ("stokes_default_opts", "stokes_last_error", "stokes_version",
                                "stokes_launch_count", "stokes_tile_config_count",
                                "stokes_octree_destroy"):
                    fn.restype = ctypes.c_int
            _lib = L
    return _lib


def make_opts(precision="mixed", near_ratio=1.0, accumulate=False, source_splits=0,
              tile_config=-1) -> StkOpts:
    o = StkOpts()
    lib().stokes_default_opts(ctypes.byref(o))
    o.precision = STK_MIXED if precision in ("mixed", STK_MIXED) else STK_FP64
    o.near_ratio = float(near_ratio)
    o.accumulate = 1 if accumulate else 0
    o.source_splits = int(source_splits)
    o.tile_config = int(tile_config)
    return o


def check(status: int):
    if status != STK_OK:
        raise StokesError(status, lib().stokes_last_error().decode())


def ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def stream_ptr(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 512), dtype=torch.uint8, device=device)


def vec3(t, name, n=None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if t.dim() != 2 or t.shape[1] != 3:
        raise ValueError(f"{name} must have shape [n, 3]")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} has {t.shape[0]} rows, expected {n}")
    return t.contiguous()


def vec1(t, name, n, dtype=torch.float64):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name} must be a CUDA {dtype} tensor")
    if t.dim() != 1 or (n is not None and t.shape[0] != n):
        raise ValueError(f"{name} must have shape [{n}]")
    return t.contiguous()
