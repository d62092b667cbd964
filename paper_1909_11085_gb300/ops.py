"""PyTorch-facing calls of the Stokes layer-potential library.

Each function marshals tensors into one C-ABI call (include/stokesgpu.h) on
the current CUDA stream and returns the velocity [n_targets, 3] (float64).
PyTorch provides only device memory and the stream.

  sl    single layer, Eq. "sl_stokes"             u = S[f]
  dl    double layer, kernel of Sec. 2.1          u = D[phi]
  sldl  superposition, Eq. "velocity_combined"    u = S[f] + D[phi]
  p2p   FMM near field over U-lists (Sec. 3.1 "Far evaluation")
  batched  independent suspensions: S over cell points + D over wall points
  sldl_grad  adjoint of sldl: gradients wrt f, phi, source positions, normals, targets
  StokesLayerFn  torch.autograd.Function over sldl whose backward calls sldl_grad
"""
from __future__ import annotations

import contextlib
import ctypes

import torch

from . import _abi as A


def _direct(kind, src, f, nrm, phi, w, trg, mu, h, precision, near_ratio, out, accumulate,
            source_splits):
    ns = src.shape[0]
    src = A.vec3(src, "src")
    trg = src if trg is None else A.vec3(trg, "trg")
    nt = trg.shape[0]
    f = A.vec3(f, "f", ns)
    nrm = A.vec3(nrm, "nrm", ns)
    phi = A.vec3(phi, "phi", ns)
    w = A.vec1(w, "w", ns)
    h = A.vec1(h, "h", ns)
    dev = src.device
    if out is None:
        out = torch.empty((nt, 3), dtype=torch.float64, device=dev)
        if accumulate:
            out.zero_()
    else:
        out = A.vec3(out, "out", nt)
    o = A.make_opts(precision, near_ratio, accumulate, source_splits)
    nb = ctypes.c_size_t(0)
    L = A.lib()
    with torch.cuda.device(dev):
        A.check(L.stokes_direct_workspace_size(ns, nt, kind, ctypes.byref(o), ctypes.byref(nb)))
        ws = A.workspace(nb.value, dev)
        st = A.stream_ptr(dev)
        if kind == A.SL:
            s = L.stokes_sl_eval(A.ptr(src), A.ptr(f), A.ptr(w), A.ptr(h), ns, A.ptr(trg), nt,
                                 float(mu), A.ptr(out), ctypes.byref(o), A.ptr(ws), ws.numel(), st)
        elif kind == A.DL:
            s = L.stokes_dl_eval(A.ptr(src), A.ptr(nrm), A.ptr(phi), A.ptr(w), A.ptr(h), ns,
                                 A.ptr(trg), nt, A.ptr(out), ctypes.byref(o), A.ptr(ws),
                                 ws.numel(), st)
        else:
            s = L.stokes_sldl_eval(A.ptr(src), A.ptr(f), A.ptr(nrm), A.ptr(phi), A.ptr(w),
                                   A.ptr(h), ns, A.ptr(trg), nt, float(mu), A.ptr(out),
                                   ctypes.byref(o), A.ptr(ws), ws.numel(), st)
        A.check(s)
    return out


def sl(src, f, w, trg=None, mu=1.0, h=None, precision="mixed", near_ratio=1.0, out=None,
       accumulate=False, source_splits=0):
    return _direct(A.SL, src, f, None, None, w, trg, mu, h, precision, near_ratio, out,
                   accumulate, source_splits)


def dl(src, nrm, phi, w, trg=None, h=None, precision="mixed", near_ratio=1.0, out=None,
       accumulate=False, source_splits=0):
    return _direct(A.DL, src, None, nrm, phi, w, trg, 1.0, h, precision, near_ratio, out,
                   accumulate, source_splits)


def sldl(src, f, nrm, phi, w, trg=None, mu=1.0, h=None, precision="mixed", near_ratio=1.0,
         out=None, accumulate=False, source_splits=0):
    return _direct(A.SLDL, src, f, nrm, phi, w, trg, mu, h, precision, near_ratio, out,
                   accumulate, source_splits)


class DirectPlan:
    """A direct sum of fixed sizes (ns sources, nt targets; kernels 1 SL, 2 DL,
    3 SL + DL) with a reusable workspace; capture() records one call into a
    CUDA graph (stokes_direct_graph_create) whose replays read the same
    buffers, so that a small sum is not bound by the host's launch latency."""

    def __init__(self, ns, nt, kernels=1, precision="mixed", near_ratio=1.0, source_splits=0,
                 device=None):
        device = device or torch.device("cuda")
        self.ns, self.nt, self.kernels = int(ns), int(nt), int(kernels)
        self.opts = A.make_opts(precision, near_ratio, False, source_splits)
        nb = ctypes.c_size_t(0)
        with torch.cuda.device(device):
            A.check(A.lib().stokes_direct_workspace_size(self.ns, self.nt, self.kernels,
                                                         ctypes.byref(self.opts), ctypes.byref(nb)))
        self.ws = A.workspace(nb.value, device)
        self.device = device

    def _args(self, src, f, nrm, phi, w, trg, mu, h, out):
        src = A.vec3(src, "src", self.ns)
        trg = src if trg is None else A.vec3(trg, "trg", self.nt)
        if trg.shape[0] != self.nt:
            raise ValueError(f"{self.nt} targets expected")
        f = A.vec3(f, "f", self.ns) if self.kernels & 1 else None
        nrm = A.vec3(nrm, "nrm", self.ns) if self.kernels & 2 else None
        phi = A.vec3(phi, "phi", self.ns) if self.kernels & 2 else None
        w, h = A.vec1(w, "w", self.ns), A.vec1(h, "h", self.ns)
        out = A.vec3(out, "out", self.nt)
        self._keep = (src, f, nrm, phi, w, trg, h, out)
        return (A.ptr(src), A.ptr(f), A.ptr(nrm), A.ptr(phi), A.ptr(w), A.ptr(h), self.ns,
                A.ptr(trg), self.nt, float(mu), A.ptr(out))

    def __call__(self, src, f=None, nrm=None, phi=None, w=None, trg=None, mu=1.0, h=None,
                 out=None):
        out = out if out is not None else torch.empty((self.nt, 3), dtype=torch.float64,
                                                       device=src.device)
        a = self._args(src, f, nrm, phi, w, trg, mu, h, out)
        L = A.lib()
        with torch.cuda.device(src.device):
            rest = (ctypes.byref(self.opts), A.ptr(self.ws), self.ws.numel(),
                    A.stream_ptr(src.device))
            if self.kernels == A.SL:
                A.check(L.stokes_sl_eval(a[0], a[1], a[4], a[5], a[6], a[7], a[8], a[9], a[10],
                                         *rest))
            elif self.kernels == A.DL:
                A.check(L.stokes_dl_eval(a[0], a[2], a[3], a[4], a[5], a[6], a[7], a[8], a[10],
                                         *rest))
            else:
                A.check(L.stokes_sldl_eval(*a, *rest))
        return out

    def capture(self, src, f=None, nrm=None, phi=None, w=None, trg=None, mu=1.0, h=None,
                out=None):
        """Captures one call into a CUDA graph that replays on the same buffers."""
        out = out if out is not None else torch.empty((self.nt, 3), dtype=torch.float64,
                                                       device=src.device)
        a = self._args(src, f, nrm, phi, w, trg, mu, h, out)
        ge = ctypes.c_void_p(0)
        stream = torch.cuda.Stream(src.device)
        with torch.cuda.device(src.device), torch.cuda.stream(stream):
            A.check(A.lib().stokes_direct_graph_create(self.kernels, *a, ctypes.byref(self.opts),
                                                       A.ptr(self.ws), self.ws.numel(),
                                                       A.stream_ptr(src.device), ctypes.byref(ge)))
        return Graph(ge, out, self._keep + (self.ws,))

    def device_status(self):
        A.check(A.lib().stokes_device_status(A.ptr(self.ws), self.ws.numel()))


class P2PPlan:
    """Device-resident U-list structure plus a reusable workspace for repeated calls."""

    def __init__(self, n, leaf_ptr, ulist_ptr, ulist_idx, kernels=3, precision="mixed",
                 near_ratio=1.0, device=None):
        device = device or torch.device("cuda")
        as32 = lambda a: torch.as_tensor(a, dtype=torch.int32).to(device).contiguous()
        self.n = int(n)
        self.leaf_ptr, self.ulist_ptr, self.ulist_idx = as32(leaf_ptr), as32(ulist_ptr), as32(ulist_idx)
        self.nleaf = self.leaf_ptr.numel() - 1
        self.kernels = int(kernels)
        self.opts = A.make_opts(precision, near_ratio)
        nb = ctypes.c_size_t(0)
        # the size query is host logic; a CPU device plans without a GPU
        with (torch.cuda.device(device) if torch.device(device).type == "cuda"
              else contextlib.nullcontext()):
            A.check(A.lib().stokes_p2p_workspace_size(self.n, self.nleaf, self.kernels,
                                                      ctypes.byref(self.opts), ctypes.byref(nb)))
        self.ws = A.workspace(nb.value, device)
        self.device = device

    def __call__(self, pts, f=None, phi=None, nrm=None, w=None, h=None, mu=1.0, out=None,
                 accumulate=False):
        n = self.n
        pts = A.vec3(pts, "pts", n)
        f, phi, nrm = A.vec3(f, "f", n), A.vec3(phi, "phi", n), A.vec3(nrm, "nrm", n)
        w, h = A.vec1(w, "w", n), A.vec1(h, "h", n)
        if out is None:
            out = torch.zeros((n, 3), dtype=torch.float64, device=pts.device)
        self.opts.accumulate = 1 if accumulate else 0
        with torch.cuda.device(pts.device):
            A.check(A.lib().stokes_p2p_leaflists(
                A.ptr(pts), A.ptr(f), A.ptr(phi), A.ptr(nrm), A.ptr(w), A.ptr(h), n,
                A.ptr(self.leaf_ptr), self.nleaf, A.ptr(self.ulist_ptr), A.ptr(self.ulist_idx),
                self.ulist_idx.numel(), self.kernels, float(mu), A.ptr(out),
                ctypes.byref(self.opts), A.ptr(self.ws), self.ws.numel(), A.stream_ptr(pts.device)))
        return out

    def device_status(self):
        A.check(A.lib().stokes_device_status(A.ptr(self.ws), self.ws.numel()))

    def _args(self, pts, f, phi, nrm, w, h, mu, out):
        n = self.n
        pts = A.vec3(pts, "pts", n)
        f, phi, nrm = A.vec3(f, "f", n), A.vec3(phi, "phi", n), A.vec3(nrm, "nrm", n)
        w, h = A.vec1(w, "w", n), A.vec1(h, "h", n)
        out = A.vec3(out, "out", n)
        self._keep = (pts, f, phi, nrm, w, h, out)  # graphs read these buffers
        return (A.ptr(pts), A.ptr(f), A.ptr(phi), A.ptr(nrm), A.ptr(w), A.ptr(h), n,
                A.ptr(self.leaf_ptr), self.nleaf, A.ptr(self.ulist_ptr), A.ptr(self.ulist_idx),
                self.ulist_idx.numel(), self.kernels, float(mu), A.ptr(out))

    def autotune(self, pts, f, phi, nrm, w, h=None, mu=1.0, out=None, cache=None):
        """Picks the fastest work-item shape on these inputs (see tuning.py for the cache)."""
        from . import tuning
        key = tuning.key("p2p", self.opts, self.n, self.nleaf, self.kernels)
        best = tuning.lookup(cache, key)
        if best is None:
            out = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64,
                                                           device=pts.device)
            cfg, ms = ctypes.c_int32(0), ctypes.c_float(0)
            self.opts.accumulate = 0
            with torch.cuda.device(pts.device):
                A.check(A.lib().stokes_autotune_p2p(*self._args(pts, f, phi, nrm, w, h, mu, out),
                                                    ctypes.byref(self.opts), A.ptr(self.ws),
                                                    self.ws.numel(), A.stream_ptr(pts.device),
                                                    ctypes.byref(cfg), ctypes.byref(ms)))
            best = int(cfg.value)
            tuning.store(cache, key, best, float(ms.value))
        self.opts.tile_config = best
        return best

    def capture(self, pts, f, phi, nrm, w, h=None, mu=1.0, out=None):
        """Captures one evaluation into a CUDA graph that replays on the same buffers."""
        out = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64,
                                                       device=pts.device)
        self.opts.accumulate = 0
        ge = ctypes.c_void_p(0)
        stream = torch.cuda.Stream(pts.device)
        with torch.cuda.device(pts.device), torch.cuda.stream(stream):
            A.check(A.lib().stokes_p2p_graph_create(*self._args(pts, f, phi, nrm, w, h, mu, out),
                                                    ctypes.byref(self.opts), A.ptr(self.ws),
                                                    self.ws.numel(), A.stream_ptr(pts.device),
                                                    ctypes.byref(ge)))
        return Graph(ge, out, self._keep + (self.ws, self.leaf_ptr, self.ulist_ptr,
                                            self.ulist_idx))


class Graph:
    """An executable CUDA graph of one library call; launch() replays it on the
    current stream.  Keeps the buffers it reads alive."""

    def __init__(self, handle, out, keep):
        self.handle, self.out, self._keep = handle, out, keep

    def launch(self, stream=None):
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        A.check(A.lib().stokes_graph_launch(self.handle, ctypes.c_void_p(st)))
        return self.out

    def __del__(self):
        try:
            if self.handle:
                A.lib().stokes_graph_destroy(self.handle)
        except Exception:
            pass


def p2p(pts, f, phi, nrm, w, leaf_ptr, ulist_ptr, ulist_idx, kernels=3, mu=1.0, h=None,
        precision="mixed", near_ratio=1.0, out=None, accumulate=False):
    plan = P2PPlan(pts.shape[0], leaf_ptr, ulist_ptr, ulist_idx, kernels, precision, near_ratio,
                   pts.device)
    return plan(pts, f, phi, nrm, w, h, mu, out, accumulate)


class BatchedPlan:
    """Suspension descriptors on the device plus a reusable workspace."""

    def __init__(self, n, susp_ptr, n_cell, precision="mixed", near_ratio=1.0, device=None):
        device = device or torch.device("cuda")
        as64 = lambda a: torch.as_tensor(a, dtype=torch.int64).to(device).contiguous()
        self.n = int(n)
        self.susp_ptr, self.n_cell = as64(susp_ptr), as64(n_cell)
        self.nsusp = self.n_cell.numel()
        self.opts = A.make_opts(precision, near_ratio)
        nb = ctypes.c_size_t(0)
        with torch.cuda.device(device):
            A.check(A.lib().stokes_batched_workspace_size(self.n, self.nsusp,
                                                          ctypes.byref(self.opts),
                                                          ctypes.byref(nb)))
        self.ws = A.workspace(nb.value, device)
        self.device = device

    def __call__(self, pts, f, phi, nrm, w, h=None, mu=1.0, out=None, accumulate=False):
        n = self.n
        pts = A.vec3(pts, "pts", n)
        f, phi, nrm = A.vec3(f, "f", n), A.vec3(phi, "phi", n), A.vec3(nrm, "nrm", n)
        w, h = A.vec1(w, "w", n), A.vec1(h, "h", n)
        if out is None:
            out = torch.zeros((n, 3), dtype=torch.float64, device=pts.device)
        self.opts.accumulate = 1 if accumulate else 0
        with torch.cuda.device(pts.device):
            A.check(A.lib().stokes_batched_eval(
                A.ptr(pts), A.ptr(f), A.ptr(phi), A.ptr(nrm), A.ptr(w), A.ptr(h), n,
                A.ptr(self.susp_ptr), A.ptr(self.n_cell), self.nsusp, float(mu), A.ptr(out),
                ctypes.byref(self.opts), A.ptr(self.ws), self.ws.numel(), A.stream_ptr(pts.device)))
        return out

    def device_status(self):
        A.check(A.lib().stokes_device_status(A.ptr(self.ws), self.ws.numel()))

    def _args(self, pts, f, phi, nrm, w, h, mu, out):
        n = self.n
        pts = A.vec3(pts, "pts", n)
        f, phi, nrm = A.vec3(f, "f", n), A.vec3(phi, "phi", n), A.vec3(nrm, "nrm", n)
        w, h = A.vec1(w, "w", n), A.vec1(h, "h", n)
        out = A.vec3(out, "out", n)
        self._keep = (pts, f, phi, nrm, w, h, out)
        return (A.ptr(pts), A.ptr(f), A.ptr(phi), A.ptr(nrm), A.ptr(w), A.ptr(h), n,
                A.ptr(self.susp_ptr), A.ptr(self.n_cell), self.nsusp, float(mu), A.ptr(out))

    def autotune(self, pts, f, phi, nrm, w, h=None, mu=1.0, out=None, cache=None):
        """Picks the fastest work-item shape on these inputs (see tuning.py for the cache)."""
        from . import tuning
        key = tuning.key("batched", self.opts, self.n, self.nsusp, 3)
        best = tuning.lookup(cache, key)
        if best is None:
            out = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64,
                                                           device=pts.device)
            cfg, ms = ctypes.c_int32(0), ctypes.c_float(0)
            self.opts.accumulate = 0
            with torch.cuda.device(pts.device):
                A.check(A.lib().stokes_autotune_batched(
                    *self._args(pts, f, phi, nrm, w, h, mu, out), ctypes.byref(self.opts),
                    A.ptr(self.ws), self.ws.numel(), A.stream_ptr(pts.device), ctypes.byref(cfg),
                    ctypes.byref(ms)))
            best = int(cfg.value)
            tuning.store(cache, key, best, float(ms.value))
        self.opts.tile_config = best
        return best

    def capture(self, pts, f, phi, nrm, w, h=None, mu=1.0, out=None):
        """Captures one batched evaluation (one persistent engine launch and its
        staging kernels) into a CUDA graph that replays on the same buffers."""
        out = out if out is not None else torch.empty((self.n, 3), dtype=torch.float64,
                                                       device=pts.device)
        self.opts.accumulate = 0
        ge = ctypes.c_void_p(0)
        stream = torch.cuda.Stream(pts.device)
        with torch.cuda.device(pts.device), torch.cuda.stream(stream):
            A.check(A.lib().stokes_batched_graph_create(
                *self._args(pts, f, phi, nrm, w, h, mu, out), ctypes.byref(self.opts),
                A.ptr(self.ws), self.ws.numel(), A.stream_ptr(pts.device), ctypes.byref(ge)))
        return Graph(ge, out, self._keep + (self.ws, self.susp_ptr, self.n_cell))


def batched(pts, f, phi, nrm, w, susp_ptr, n_cell, mu=1.0, h=None, precision="mixed",
            near_ratio=1.0, out=None, accumulate=False):
    plan = BatchedPlan(pts.shape[0], susp_ptr, n_cell, precision, near_ratio, pts.device)
    return plan(pts, f, phi, nrm, w, h, mu, out, accumulate)


def sldl_grad(src, f, nrm, phi, w, trg, g, mu=1.0, h=None, precision="mixed", near_ratio=1.0,
              want=("f", "phi", "y", "n", "x")):
    """Gradients of L = sum_i g_i . (SL[f] + DL[phi])(x_i); returns a dict of tensors
    (keys among f, phi, y, n, x; y and n are per source, x per target)."""
    ns = src.shape[0]
    src = A.vec3(src, "src")
    trg = src if trg is None else A.vec3(trg, "trg")
    nt = trg.shape[0]
    f, nrm, phi = A.vec3(f, "f", ns), A.vec3(nrm, "nrm", ns), A.vec3(phi, "phi", ns)
    w, h = A.vec1(w, "w", ns), A.vec1(h, "h", ns)
    g = A.vec3(g, "g", nt)
    dev = src.device
    mk = lambda n: torch.empty((n, 3), dtype=torch.float64, device=dev)
    out = {}
    if "f" in want and f is not None:
        out["f"] = mk(ns)
    if "phi" in want and phi is not None:
        out["phi"] = mk(ns)
    if "y" in want:
        out["y"] = mk(ns)
    if "n" in want and phi is not None:
        out["n"] = mk(ns)
    if "x" in want:
        out["x"] = mk(nt)
    o = A.make_opts(precision, near_ratio)
    nb = ctypes.c_size_t(0)
    L = A.lib()
    with torch.cuda.device(dev):
        A.check(L.stokes_grad_workspace_size(ns, nt, ctypes.byref(o), ctypes.byref(nb)))
        ws = A.workspace(nb.value, dev)
        A.check(L.stokes_sldl_grad(
            A.ptr(src), A.ptr(f), A.ptr(nrm), A.ptr(phi), A.ptr(w), A.ptr(h), ns, A.ptr(trg), nt,
            A.ptr(g), float(mu), A.ptr(out.get("f")), A.ptr(out.get("phi")), A.ptr(out.get("y")),
            A.ptr(out.get("n")), A.ptr(out.get("x")), ctypes.byref(o), A.ptr(ws), ws.numel(),
            A.stream_ptr(dev)))
    return out


class StokesLayerFn(torch.autograd.Function):
    """u = SL[f] + DL[phi] at the targets, differentiable in f, phi, the source
    positions, the normals and the target positions (weights and spacings are
    constants).  The backward recomputes the pair terms (no O(N^2) state)."""

    @staticmethod
    def forward(ctx, src, f, nrm, phi, w, trg, mu=1.0, h=None, precision="mixed",
                near_ratio=1.0):
        ctx.save_for_backward(src, f, nrm, phi, w, trg, h)
        ctx.cfg = (float(mu), precision, float(near_ratio))
        return sldl(src, f, nrm, phi, w, trg, mu, h=h, precision=precision,
                    near_ratio=near_ratio)

    @staticmethod
    def backward(ctx, gu):
        src, f, nrm, phi, w, trg, h = ctx.saved_tensors
        mu, precision, near_ratio = ctx.cfg
        need = ctx.needs_input_grad
        want = []
        if need[0]:
            want.append("y")
        if need[1]:
            want.append("f")
        if need[2]:
            want.append("n")
        if need[3]:
            want.append("phi")
        if need[5]:
            want.append("x")
        G = sldl_grad(src, f, nrm, phi, w, trg, gu.contiguous(), mu, h=h, precision=precision,
                      near_ratio=near_ratio, want=tuple(want))
        return (G.get("y"), G.get("f"), G.get("n"), G.get("phi"), None, G.get("x"), None, None,
                None, None)


def upsample_patches(coarse, npatch, q=10, eta=2):
    """Values on each patch's (q+1)^2 Clenshaw-Curtis nodes -> values on the
    fine discretisation (4^eta sub-patches per patch), FP64 (Sec. 3.1, the
    upsampling operator U)."""
    coarse = coarse.contiguous()
    if coarse.dtype != torch.float64 or not coarse.is_cuda:
        raise TypeError("coarse must be a float64 CUDA tensor")
    ncomp = 1 if coarse.dim() == 1 else coarse.shape[1]
    m = 1 << eta
    nf = npatch * m * m * (q + 1) ** 2
    if coarse.shape[0] != npatch * (q + 1) ** 2:
        raise ValueError("coarse must have npatch * (q+1)^2 rows")
    fine = torch.empty((nf, ncomp) if coarse.dim() > 1 else (nf,), dtype=torch.float64,
                       device=coarse.device)
    with torch.cuda.device(coarse.device):
        A.check(A.lib().stokes_upsample_patches(A.ptr(coarse), int(npatch), int(q), int(eta),
                                                int(ncomp), A.ptr(fine),
                                                A.stream_ptr(coarse.device)))
    return fine


class CheckpointPlan:
    """Singular / near-singular evaluation on a fixed patch surface by check-point
    extrapolation (Sec. 3.1).  The fine discretisation (fine_pts, fine_nrm,
    fine_w, fine_h; 4^eta sub-patches per patch, see include/stokesgpu.h for the
    node order) and the targets with their closest points y and normals n are
    fixed; calls take the densities on the coarse nodes.  Defaults: q = 10,
    eta = 2 (16 sub-patches), p = 4, R = 3 h_c, r = h_c with h_c the caller's
    coarse node spacing."""

    def __init__(self, npatch, fine_pts, fine_nrm, fine_w, fine_h, trg, y, n, R, r, p=4, q=10,
                 eta=2, kernels=2, precision="mixed", near_ratio=1.0):
        self.npatch, self.q, self.eta, self.p = int(npatch), int(q), int(eta), int(p)
        self.R, self.r, self.kernels = float(R), float(r), int(kernels)
        m = 1 << self.eta
        nf = self.npatch * m * m * (self.q + 1) ** 2
        self.fine = (A.vec3(fine_pts, "fine_pts", nf), A.vec3(fine_nrm, "fine_nrm", nf),
                     A.vec1(fine_w, "fine_w", nf), A.vec1(fine_h, "fine_h", nf))
        self.nt = trg.shape[0]
        self.trg, self.y, self.n = (A.vec3(trg, "trg", self.nt), A.vec3(y, "y", self.nt),
                                    A.vec3(n, "n", self.nt))
        self.opts = A.make_opts(precision, near_ratio)
        self.device = trg.device
        nb = ctypes.c_size_t(0)
        with torch.cuda.device(self.device):
            A.check(A.lib().stokes_checkpoint_workspace_size(
                self.kernels, self.npatch, self.q, self.eta, self.nt, self.p,
                ctypes.byref(self.opts), ctypes.byref(nb)))
        self.ws = A.workspace(nb.value, self.device)

    def __call__(self, f=None, phi=None, mu=1.0, out=None, accumulate=False):
        nc = self.npatch * (self.q + 1) ** 2
        f = A.vec3(f, "f", nc) if f is not None else None
        phi = A.vec3(phi, "phi", nc) if phi is not None else None
        if out is None:
            out = torch.zeros((self.nt, 3), dtype=torch.float64, device=self.device)
        self.opts.accumulate = 1 if accumulate else 0
        fp, fn, fw, fh = self.fine
        with torch.cuda.device(self.device):
            A.check(A.lib().stokes_checkpoint_eval(
                self.kernels, A.ptr(f), A.ptr(phi), self.npatch, self.q, self.eta, A.ptr(fp),
                A.ptr(fn), A.ptr(fw), A.ptr(fh), A.ptr(self.trg), A.ptr(self.y), A.ptr(self.n),
                self.nt, self.R, self.r, self.p, float(mu), A.ptr(out), ctypes.byref(self.opts),
                A.ptr(self.ws), self.ws.numel(), A.stream_ptr(self.device)))
        return out


class BIEPlan:
    """The boundary-integral operator (D - I/2 + N) of a fixed patch surface
    (Eq. "double_layer_int_eq", discretised as Eq. "int_eq_disc"), applied by
    matvec(phi) to double-layer densities on the coarse nodes; D - I/2 is the
    fluid-side limit taken by check points (see CheckpointPlan), N the
    rank-completing term.  Sign convention: n points out of the fluid."""

    def __init__(self, npatch, nodes, nodes_n, nodes_w, fine_pts, fine_nrm, fine_w, fine_h, R, r,
                 p=4, q=10, eta=2, precision="mixed", near_ratio=1.0):
        self.npatch, self.q, self.eta, self.p = int(npatch), int(q), int(eta), int(p)
        self.R, self.r = float(R), float(r)
        nc = self.npatch * (self.q + 1) ** 2
        m = 1 << self.eta
        nf = self.npatch * m * m * (self.q + 1) ** 2
        self.nodes = (A.vec3(nodes, "nodes", nc), A.vec3(nodes_n, "nodes_n", nc),
                      A.vec1(nodes_w, "nodes_w", nc))
        self.fine = (A.vec3(fine_pts, "fine_pts", nf), A.vec3(fine_nrm, "fine_nrm", nf),
                     A.vec1(fine_w, "fine_w", nf), A.vec1(fine_h, "fine_h", nf))
        self.nc = nc
        self.device = nodes.device
        self.opts = A.make_opts(precision, near_ratio)
        nb = ctypes.c_size_t(0)
        with torch.cuda.device(self.device):
            A.check(A.lib().stokes_bie_workspace_size(self.npatch, self.q, self.eta, self.p,
                                                      ctypes.byref(self.opts), ctypes.byref(nb)))
        self.ws = A.workspace(nb.value, self.device)

    def matvec(self, phi, out=None, accumulate=False):
        phi = A.vec3(phi, "phi", self.nc)
        if out is None:
            out = torch.zeros((self.nc, 3), dtype=torch.float64, device=self.device)
        self.opts.accumulate = 1 if accumulate else 0
        x, xn, xw = self.nodes
        fp, fn, fw, fh = self.fine
        with torch.cuda.device(self.device):
            A.check(A.lib().stokes_bie_matvec(
                A.ptr(phi), self.npatch, self.q, self.eta, A.ptr(x), A.ptr(xn), A.ptr(xw),
                A.ptr(fp), A.ptr(fn), A.ptr(fw), A.ptr(fh), self.R, self.r, self.p, A.ptr(out),
                ctypes.byref(self.opts), A.ptr(self.ws), self.ws.numel(),
                A.stream_ptr(self.device)))
        return out


def near_patch_search(nodes, npatch, trg, d_eps, q=10):
    """Closest patch and point for every target within d_eps of a patch surface
    (Sec. 3.2): returns (patch [nt] int32, -1 for none; uv [nt, 2]; y [nt, 3];
    n [nt, 3]; dist [nt], -1 for none)."""
    nc = int(npatch) * (q + 1) ** 2
    nodes = A.vec3(nodes, "nodes", nc)
    trg = A.vec3(trg, "trg")
    nt = trg.shape[0]
    dev = trg.device
    patch = torch.empty(nt, dtype=torch.int32, device=dev)
    uv = torch.empty((nt, 2), dtype=torch.float64, device=dev)
    y = torch.empty((nt, 3), dtype=torch.float64, device=dev)
    n = torch.empty((nt, 3), dtype=torch.float64, device=dev)
    dist = torch.empty(nt, dtype=torch.float64, device=dev)
    nb = ctypes.c_size_t(0)
    A.check(A.lib().stokes_near_search_workspace_size(int(npatch), int(q), nt, ctypes.byref(nb)))
    ws = A.workspace(nb.value, dev)
    with torch.cuda.device(dev):
        A.check(A.lib().stokes_near_patch_search(
            A.ptr(nodes), int(npatch), int(q), A.ptr(trg), nt, float(d_eps), A.ptr(patch),
            A.ptr(uv), A.ptr(y), A.ptr(n), A.ptr(dist), A.ptr(ws), ws.numel(),
            A.stream_ptr(dev)))
    return patch, uv, y, n, dist


def octree(pts, max_leaf=256):
    """Octree and interaction lists of a point set (host, stokes_octree_build).
    pts: [n, 3] float64 (numpy or a tensor on any device).  Returns a dict of
    numpy arrays: perm (leaf-sorted position -> caller index), leaf_ptr,
    ulist_ptr / ulist_idx (the U-lists of P2PPlan), box_depth, box_anchor,
    box_parent, box_leaf, the V, W, X lists and each box's 27 same-depth
    neighbours (colleague), with root_lo, root_size and max_depth;
    ops.fmm_tree_arrays(**fmm_tree_args(t)) gives the far field's tree."""
    import numpy as np
    if isinstance(pts, torch.Tensor):
        pts = pts.detach().cpu().numpy()
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != 3:
        raise ValueError("pts must have shape [n, 3]")
    L = A.lib()
    h = ctypes.c_void_p()
    A.check(L.stokes_octree_build(pts.ctypes.data, pts.shape[0], int(max_leaf), ctypes.byref(h)))
    try:
        info = A.StkOctreeInfo()
        A.check(L.stokes_octree_info(h, ctypes.byref(info)))
        n, nl, nb = int(info.n), int(info.nleaf), int(info.nbox)
        out = {"perm": np.empty(n, np.int64), "leaf_ptr": np.empty(nl + 1, np.int32),
               "ulist_ptr": np.empty(nl + 1, np.int32),
               "ulist_idx": np.empty(int(info.nulist), np.int32),
               "box_depth": np.empty(nb, np.int32), "box_anchor": np.empty((nb, 3), np.int32),
               "box_parent": np.empty(nb, np.int32), "box_leaf": np.empty(nb, np.int32),
               "v_ptr": np.empty(nb + 1, np.int32), "v_idx": np.empty(int(info.nv), np.int32),
               "w_ptr": np.empty(nb + 1, np.int32), "w_idx": np.empty(int(info.nw), np.int32),
               "x_ptr": np.empty(nb + 1, np.int32), "x_idx": np.empty(int(info.nx), np.int32),
               "colleague": np.empty((nb, 27), np.int32)}
        keys = ("perm", "leaf_ptr", "ulist_ptr", "ulist_idx", "box_depth", "box_anchor",
                "box_parent", "box_leaf", "v_ptr", "v_idx", "w_ptr", "w_idx", "x_ptr", "x_idx",
                "colleague")
        A.check(L.stokes_octree_export(h, *[ctypes.c_void_p(out[k].ctypes.data) for k in keys]))
    finally:
        L.stokes_octree_destroy(h)
    out["root_lo"] = np.array(info.root_lo[:], dtype=np.float64)
    out["root_size"] = float(info.root_size)
    out["max_depth"] = int(info.max_depth)
    return out


def fmm_tree_args(t):
    """The arguments of fmm_tree_arrays from an octree() result (its colleague
    table is checked against the derived one)."""
    return dict(depth=t["box_depth"], anchor=t["box_anchor"], parent=t["box_parent"],
                box_leaf=t["box_leaf"], leaf_ptr=t["leaf_ptr"], v_ptr=t["v_ptr"],
                v_idx=t["v_idx"], w_ptr=t["w_ptr"], w_idx=t["w_idx"], x_ptr=t["x_ptr"],
                x_idx=t["x_idx"], root_lo=t["root_lo"], root_size=t["root_size"],
                colleague=t.get("colleague"))


_FMM_DEVICE_KEYS = ("depth", "anchor", "parent", "child_ptr", "box_leaf", "leaf_box", "leaf_ptr",
                    "v_ptr", "v_idx", "w_ptr", "w_idx", "x_ptr", "x_idx", "colleague")


def fmm_tree_arrays(depth, anchor, parent, box_leaf, leaf_ptr, v_ptr, v_idx, w_ptr, w_idx, x_ptr,
                    x_idx, root_lo, root_size, colleague=None):
    """Host arrays of the far field's tree (stk_fmm_tree, include/stokesgpu.h)
    from each box's depth, integer anchor, parent and leaf number, the leaves'
    point ranges and the V, W and X lists.  The library derives depth_ptr,
    child_ptr, leaf_box and the same-depth neighbours (colleague) and checks
    the order the passes rely on (stokes_fmm_tree_complete); this function
    marshals the arrays and checks that the lists are CSR lists over the boxes."""
    import numpy as np
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    depth, anchor, parent, box_leaf = i32(depth), i32(anchor), i32(parent), i32(box_leaf)
    leaf_ptr = i32(leaf_ptr)
    M = depth.size
    if anchor.shape != (M, 3) or parent.size != M or box_leaf.size != M:
        raise ValueError("anchor must have shape [nbox, 3] and parent, box_leaf [nbox]")
    nleaf = leaf_ptr.size - 1
    if nleaf < 1:
        raise ValueError("leaf_ptr must hold at least one leaf")
    md = ctypes.c_int32(0)
    depth_ptr = np.zeros(23, dtype=np.int32)
    child_ptr = np.zeros(M + 1, dtype=np.int32)
    leaf_box = np.zeros(nleaf, dtype=np.int32)
    coll = np.zeros((M, 27), dtype=np.int32)
    s = A.lib().stokes_fmm_tree_complete(M, nleaf, depth.ctypes.data, anchor.ctypes.data,
                                         parent.ctypes.data, box_leaf.ctypes.data, ctypes.byref(md),
                                         depth_ptr.ctypes.data, child_ptr.ctypes.data,
                                         leaf_box.ctypes.data, coll.ctypes.data)
    if s != A.STK_OK:
        raise ValueError(A.lib().stokes_last_error().decode())
    max_depth = int(md.value)
    if colleague is not None and not np.array_equal(i32(colleague), coll):
        raise ValueError("colleague does not match the tree")
    t = {"depth_ptr": depth_ptr[:max_depth + 2].copy(), "depth": depth, "anchor": anchor,
         "parent": parent, "child_ptr": child_ptr, "box_leaf": box_leaf, "leaf_box": leaf_box,
         "leaf_ptr": leaf_ptr, "v_ptr": i32(v_ptr), "v_idx": i32(v_idx), "w_ptr": i32(w_ptr),
         "w_idx": i32(w_idx), "x_ptr": i32(x_ptr), "x_idx": i32(x_idx),
         "root_lo": np.asarray(root_lo, dtype=np.float64).reshape(3).copy(),
         "root_size": float(root_size), "max_depth": max_depth, "colleague": coll}
    for k in ("v", "w", "x"):
        ptr, idx = t[k + "_ptr"], t[k + "_idx"]
        if ptr.size != M + 1 or ptr[0] != 0 or np.any(np.diff(ptr) < 0) or ptr[-1] != idx.size \
                or np.any(idx < 0) or np.any(idx >= M):
            raise ValueError(f"{k.upper()} list is not a CSR list over the boxes")
    if np.any(box_leaf[t["x_idx"]] < 0):
        raise ValueError("X lists hold leaves only")
    if leaf_ptr[0] != 0 or np.any(np.diff(leaf_ptr) < 0):
        raise ValueError("leaf_ptr must be non-decreasing from 0")
    return t


def fmm_operators(p, root_size, max_depth, mu=1.0, flux=True, rcond=1e-13, upward="per_depth"):
    """Check-to-equivalent operators of depths 2..max_depth (host, FP64,
    stokes_fmm_operators): uc2e [max_depth - 1][(flux ? 4 : 3) ns][3 ns],
    dc2e [max_depth - 1][3 ns][3 ns].  upward = "per_depth" decomposes the
    upward operator with point sources at every depth (minimum-norm densities),
    "scaled" derives every depth's from the one of half-width 1, source
    strengths in units of the half-width (exact, one decomposition; at p = 6
    one instead of one per depth at ~8 s each), a far field within the
    truncation error of the per-depth one."""
    if upward not in ("per_depth", "scaled"):
        raise ValueError('upward must be "per_depth" or "scaled"')
    import numpy as np
    ns = p ** 3 - (p - 2) ** 3
    nc = 4 if flux else 3
    D = max(int(max_depth) - 1, 0)
    uc = np.zeros((D, nc * ns, 3 * ns))
    dc = np.zeros((D, 3 * ns, 3 * ns))
    if D == 0:
        return uc, dc
    A.check(A.lib().stokes_fmm_operators(int(p), float(root_size), int(max_depth), float(mu),
                                         int(bool(flux)), float(rcond), int(upward == "scaled"),
                                         uc.ctypes.data, dc.ctypes.data))
    return uc, dc


def fmm_m2l_spectra(p, mu=1.0, flux=True):
    """Kernel spectra of Fourier-space M2L at half-width 1 (host, FP64):
    [343, 2p, 2p, p + 1, 3, nc, 2] (see stokes_fmm_m2l_spectra)."""
    import numpy as np
    nc = 4 if flux else 3
    out = np.zeros((343, 2 * p, 2 * p, p + 1, 3, nc, 2))
    A.check(A.lib().stokes_fmm_m2l_spectra(int(p), float(mu), int(bool(flux)), out.ctypes.data))
    return out


class FmmFarPlan:
    """Far field of the FMM (stokes_fmm_far_eval) on a fixed tree: device
    copies of the tree arrays (from fmm_tree_arrays), the per-depth operators
    (fmm_operators unless given) and a workspace.  Calls take the densities of
    the leaf-sorted points and return the far field [n, 3]; adding the U-list
    P2P sum over the same leaves gives the FMM velocity.  m2l = "dense"
    evaluates M2L kernel by kernel, "fft" in Fourier space (fmm_m2l_spectra);
    precision = "fp64" runs every pass in FP64, "mixed" the evaluations in FP32
    on local coordinates with double-FP32 check-to-equivalent products.  The operators'
    cut-off (rcond) defaults to 1e-13, and to 1e-7 (FP32's resolution) for the
    mixed form at p >= 6, where FP32 rounding of densities fitted beyond it
    would exceed the truncation error.  upward = "scaled" derives every
    depth's upward operator from one decomposition (see fmm_operators)."""

    def __init__(self, tree, p=4, mu=1.0, flux=True, uc2e=None, dc2e=None, rcond=None,
                 device=None, m2l="dense", precision="fp64", upward="per_depth"):
        import numpy as np
        self.device = device or torch.device("cuda")
        self.p, self.mu, self.flux = int(p), float(mu), bool(flux)
        self.depth_ptr = np.ascontiguousarray(tree["depth_ptr"], dtype=np.int32)
        self._arrays = {k: torch.as_tensor(np.asarray(tree[k], dtype=np.int32)).to(
            self.device).contiguous() for k in _FMM_DEVICE_KEYS}
        self.n = int(tree["leaf_ptr"][-1])
        if rcond is None:
            rcond = 1e-7 if (precision == "mixed" and self.p >= 6) else 1e-13
        if uc2e is None or dc2e is None:
            uc2e, dc2e = fmm_operators(self.p, tree["root_size"], tree["max_depth"], self.mu,
                                       self.flux, rcond, upward)
        ns, nc, D = self.p ** 3 - (self.p - 2) ** 3, 4 if self.flux else 3, max(
            int(tree["max_depth"]) - 1, 0)
        uc2e, dc2e = np.asarray(uc2e, dtype=np.float64), np.asarray(dc2e, dtype=np.float64)
        if D and (uc2e.shape != (D, nc * ns, 3 * ns) or dc2e.shape != (D, 3 * ns, 3 * ns)):
            raise ValueError(f"operators must be [{D}, {nc * ns}, {3 * ns}] and "
                             f"[{D}, {3 * ns}, {3 * ns}] for p = {self.p}, flux = {self.flux}")
        self.uc2e = torch.as_tensor(uc2e).to(self.device).contiguous()
        self.dc2e = torch.as_tensor(dc2e).to(self.device).contiguous()
        if m2l not in ("dense", "fft"):
            raise ValueError('m2l must be "dense" or "fft"')
        if precision not in ("fp64", "mixed"):
            raise ValueError('precision must be "fp64" or "mixed"')
        self.precision = A.STK_MIXED if precision == "mixed" else A.STK_FP64
        self.spec = None
        if m2l == "fft":
            self.spec = torch.as_tensor(fmm_m2l_spectra(self.p, self.mu, self.flux)).to(
                self.device).contiguous()
        t = A.StkFmmTree()
        t.nbox = int(tree["depth"].size)
        t.nleaf = int(tree["leaf_box"].size)
        t.max_depth = int(tree["max_depth"])
        t.depth_ptr = self.depth_ptr.ctypes.data
        for k in _FMM_DEVICE_KEYS:
            setattr(t, k, self._arrays[k].data_ptr() if self._arrays[k].numel() else None)
        for q in range(3):
            t.root_lo[q] = float(tree["root_lo"][q])
        t.root_size = float(tree["root_size"])
        self.tree = t
        nb = ctypes.c_size_t(0)
        A.check(A.lib().stokes_fmm_far_workspace_size(self.p, int(self.flux),
                                                      int(self.spec is not None), self.precision,
                                                      self.n, ctypes.byref(t), ctypes.byref(nb)))
        self.ws = A.workspace(nb.value, self.device)

    def __call__(self, pts, f=None, phi=None, nrm=None, w=None, out=None, accumulate=False):
        n = self.n
        pts = A.vec3(pts, "pts", n)
        f, phi, nrm = A.vec3(f, "f", n), A.vec3(phi, "phi", n), A.vec3(nrm, "nrm", n)
        w = A.vec1(w, "w", n)
        if out is None:
            out = torch.zeros((n, 3), dtype=torch.float64, device=self.device)
        else:
            out = A.vec3(out, "out", n)
        ops = self.uc2e.numel() > 0
        with torch.cuda.device(self.device):
            A.check(A.lib().stokes_fmm_far_eval(
                A.ptr(pts), A.ptr(f), A.ptr(phi), A.ptr(nrm), A.ptr(w), n, ctypes.byref(self.tree),
                self.p, int(self.flux), A.ptr(self.uc2e) if ops else None,
                A.ptr(self.dc2e) if ops else None, A.ptr(self.spec), self.precision, self.mu,
                A.ptr(out),
                int(bool(accumulate)),
                A.ptr(self.ws), self.ws.numel(), A.stream_ptr(self.device)))
        return out


class FmmPlan:
    """The FMM velocity of one point set (Sec. 3.1, "Far evaluation"): the
    library's octree built once from the points, the U-list near field
    (P2PPlan) and the far field on the same tree (FmmFarPlan).  Calls take
    positions and densities in the tree's leaf order (perm[i] is the caller's
    index of leaf-ordered point i) and return the velocity in that order.
    kernels: 1 single layer (f), 2 double layer (phi, nrm), 3 both; the far
    field's upward densities carry point sources whenever the double layer is
    on."""

    def __init__(self, pts, max_leaf=256, p=4, mu=1.0, kernels=3, near_precision="mixed",
                 near_ratio=1.0, far_precision="fp64", m2l="dense", device=None):
        self.tree = octree(pts, max_leaf)
        self.perm = self.tree["perm"]
        self.n = int(self.perm.size)
        self.mu, self.kernels = float(mu), int(kernels)
        if self.kernels not in (1, 2, 3):
            raise ValueError("kernels must be 1, 2 or 3")
        t = fmm_tree_arrays(**fmm_tree_args(self.tree))
        self.near = P2PPlan(self.n, t["leaf_ptr"], self.tree["ulist_ptr"], self.tree["ulist_idx"],
                            self.kernels, near_precision, near_ratio, device)
        self.far = FmmFarPlan(t, p=p, mu=mu, flux=bool(self.kernels & 2), m2l=m2l,
                              precision=far_precision, device=device)

    def __call__(self, pts, f=None, phi=None, nrm=None, w=None, h=None, out=None):
        if self.kernels & 1 and f is None:
            raise ValueError("the single layer needs f")
        if self.kernels & 2 and (phi is None or nrm is None):
            raise ValueError("the double layer needs phi and nrm")
        f = f if self.kernels & 1 else None
        phi, nrm = (phi, nrm) if self.kernels & 2 else (None, None)
        u = self.far(pts, f, phi, nrm, w, out=out)
        return self.near(pts, f, phi, nrm, w, h, self.mu, out=u, accumulate=True)
