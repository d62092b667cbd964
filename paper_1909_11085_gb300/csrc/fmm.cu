// fmm.cu -- the far field of the kernel-independent FMM on the GPU (Sec. 3.1,
// "Far evaluation"): the passes of fmm_passes.cuh, one grid-stride launch per
// pass and depth on the caller's stream, in FP64 or in the mixed form (FP32
// evaluations and spectra, double-FP32 check-to-equivalent products), with M2L
// dense or in Fourier space.  The near field is the U-list P2P sum
// (stokes_p2p_leaflists); the two together are the FMM.
#include <cmath>

#include "../../include/stokesgpu.h"
#include "fmm_fast.cuh"
#include "prep.cuh"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

using stk::fmm::Pass;

// Per-launch timing hooks of this thread's later far-field calls
// (stokes_fmm_set_pass_events).
thread_local stk::fmm::FastHooks g_hooks;

template <class F>
__global__ void __launch_bounds__(256) k_fmm_pass(Pass P, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) F()(P, e);
}

__global__ void k_fmm_setup(Pass P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) stk::fmm::fill_setup(P);
}

struct DeviceExec {
  cudaStream_t st;
  int64_t max_blocks;
  cudaError_t err = cudaSuccess;
  template <class F>
  void run(const Pass &P, int64_t n) {
    if (n <= 0 || err != cudaSuccess) return;
    int64_t g = (n + 255) / 256;
    if (g > max_blocks) g = max_blocks;
    k_fmm_pass<F><<<(unsigned)g, 256, 0, st>>>(P, n);
    err = cudaGetLastError();
    stk::count_launches(1);
  }
};

stk_status check_tree(const stk_fmm_tree *t) {
  using stk::report_error;
  if (!t) return report_error(STK_EINVAL, "tree is NULL");
  if (t->nbox < 1 || t->nleaf < 1 || t->nleaf > t->nbox)
    return report_error(STK_EINVAL, "tree needs 1 <= nleaf <= nbox");
  if (t->max_depth < 0 || t->max_depth > stk::fmm::kMaxTreeDepth)
    return report_error(STK_EINVAL, "tree max_depth must be in [0, 21]");
  if (!t->depth_ptr) return report_error(STK_EINVAL, "tree depth_ptr is NULL");
  if (t->depth_ptr[0] != 0 || t->depth_ptr[t->max_depth + 1] != t->nbox)
    return report_error(STK_EINVAL, "tree depth_ptr must run from 0 to nbox");
  for (int d = 0; d <= t->max_depth; ++d)
    if (t->depth_ptr[d + 1] < t->depth_ptr[d])
      return report_error(STK_EINVAL, "tree depth_ptr must be non-decreasing");
  if (!t->depth || !t->anchor || !t->parent || !t->child_ptr || !t->box_leaf || !t->leaf_box ||
      !t->leaf_ptr || !t->v_ptr || !t->w_ptr || !t->x_ptr)
    return report_error(STK_EINVAL, "a tree array is NULL");
  if (!(t->root_size > 0.0) || !std::isfinite(t->root_size))
    return report_error(STK_EINVAL, "tree root_size must be finite and > 0");
  for (int q = 0; q < 3; ++q)
    if (!std::isfinite(t->root_lo[q])) return report_error(STK_EINVAL, "tree root_lo is not finite");
  return STK_OK;
}

stk::fmm::Tree device_tree(const stk_fmm_tree *t) {
  stk::fmm::Tree T;
  T.nbox = t->nbox;
  T.nleaf = t->nleaf;
  T.depth = t->depth;
  T.anchor = t->anchor;
  T.parent = t->parent;
  T.child_ptr = t->child_ptr;
  T.leaf_box = t->leaf_box;
  T.leaf_ptr = t->leaf_ptr;
  T.v_ptr = t->v_ptr;
  T.v_idx = t->v_idx;
  T.w_ptr = t->w_ptr;
  T.w_idx = t->w_idx;
  T.x_ptr = t->x_ptr;
  T.x_idx = t->x_idx;
  T.box_leaf = t->box_leaf;
  T.colleague = t->colleague;
  for (int q = 0; q < 3; ++q) T.root_lo[q] = t->root_lo[q];
  T.root_size = t->root_size;
  return T;
}

}  // namespace

extern "C" {

stk_status stokes_fmm_far_workspace_size(int32_t p, int32_t flux, int32_t fft_m2l,
                                         int32_t precision, int64_t n,
                                         const stk_fmm_tree *tree, size_t *bytes) {
  if (p < 2 || p > 12) return stk::report_error(STK_EINVAL, "p must be in [2, 12]");
  if (precision != STK_FP64 && precision != STK_MIXED)
    return stk::report_error(STK_EINVAL, "precision must be STK_FP64 or STK_MIXED");
  if (n < 0 || n > 0x7fffffffLL) return stk::report_error(STK_EINVAL, "n must be in [0, 2^31-1]");
  if (!bytes) return stk::report_error(STK_EINVAL, "bytes is NULL");
  const stk_status s = check_tree(tree);
  if (s != STK_OK) return s;
  *bytes = stk::fmm::layout(tree->nbox, p, flux ? 4 : 3, fft_m2l != 0, precision == STK_MIXED, n,
                            tree->max_depth, tree->depth_ptr)
               .total;
  return STK_OK;
}

stk_status stokes_fmm_far_eval(const double *pts, const double *f, const double *phi,
                               const double *nrm, const double *w, int64_t n,
                               const stk_fmm_tree *tree, int32_t p, int32_t flux,
                               const double *uc2e, const double *dc2e,
                               const double *m2l_spectra, int32_t precision, double mu,
                               double *out,
                               int32_t accumulate, void *workspace, size_t workspace_bytes,
                               void *stream) {
  using stk::report_error;
  if (p < 2 || p > 12) return report_error(STK_EINVAL, "p must be in [2, 12]");
  if (n < 0 || n > 0x7fffffffLL) return report_error(STK_EINVAL, "n must be in [0, 2^31-1]");
  if (precision != STK_FP64 && precision != STK_MIXED)
    return report_error(STK_EINVAL, "precision must be STK_FP64 or STK_MIXED");
  stk_status s = check_tree(tree);
  if (s != STK_OK) return s;
  if (n == 0) return STK_OK;
  if (!pts || !w || !out) return report_error(STK_EINVAL, "pts/w/out is NULL");
  if (!f && !phi) return report_error(STK_EINVAL, "f and phi are both NULL");
  if (phi && !nrm) return report_error(STK_EINVAL, "nrm is NULL");
  // the equivalent forces carry the Stokeslet of the operators' viscosity, also
  // without a single layer
  if (!(mu > 0.0 && std::isfinite(mu))) return report_error(STK_EINVAL, "mu must be finite and > 0");
  if (tree->max_depth >= stk::fmm::kFirstDepth && (!uc2e || !dc2e))
    return report_error(STK_EINVAL, "uc2e/dc2e is NULL");
  const int ns = stk::fmm::surface_count(p), nc = flux ? 4 : 3;
  const bool fft = m2l_spectra != nullptr, mixed = precision == STK_MIXED;
  const stk::fmm::Layout L =
      stk::fmm::layout(tree->nbox, p, nc, fft, mixed, n, tree->max_depth, tree->depth_ptr);
  if (!workspace || workspace_bytes < L.total) return report_error(STK_ENOMEM, "workspace too small");
  char *ws = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~(uintptr_t)255);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return report_error(STK_ECUDA, "cannot query the device");

  Pass P;
  P.t = device_tree(tree);
  P.pts = pts;
  P.f = f;
  P.phi = phi;
  P.nrm = nrm;
  P.w = w;
  P.n = n;
  P.csl = 1.0 / (8.0 * stk::fmm::kPi * mu);
  P.cdl = 6.0 / (8.0 * stk::fmm::kPi);
  P.csrc = 1.0 / (4.0 * stk::fmm::kPi);
  P.ns = ns;
  P.nc = nc;
  P.uc2e = uc2e;
  P.dc2e = dc2e;
  P.out = out;
  P.accumulate = accumulate ? 1 : 0;
  P.depth = 0;
  P.box0 = P.box1 = 0;
  P.p = p;
  P.spec = m2l_spectra;
  P.n_uc2e = stk::fmm::op_entries(p, nc, tree->max_depth, true);
  P.n_dc2e = stk::fmm::op_entries(p, nc, tree->max_depth, false);
  stk::fmm::bind(P, ws, L, fft, mixed);

  if (cudaMemsetAsync(ws + L.counters, 0, sizeof(int32_t) * 4, st) != cudaSuccess)
    return report_error(STK_ECUDA, "cannot clear the error word");
  k_fmm_setup<<<1, 32, 0, st>>>(P);
  if (cudaGetLastError() != cudaSuccess) return report_error(STK_ECUDA, "set-up launch failed");
  stk::count_launches(1);
  // the CTA-blocked mixed kernels (their spectral products need the colleague table)
  if (mixed && p <= stk::fmm::kFastMaxP && (!fft || tree->colleague)) {
    const cudaError_t e = stk::fmm::far_field_fast(P, tree->depth_ptr, tree->max_depth, sms, st,
                                                   g_hooks);
    if (e != cudaSuccess) return report_error(STK_ECUDA, cudaGetErrorString(e));
    return STK_OK;
  }
  DeviceExec ex{st, (int64_t)sms * 8};
  stk::fmm::far_field(ex, P, tree->depth_ptr, tree->max_depth);
  if (ex.err != cudaSuccess) return report_error(STK_ECUDA, cudaGetErrorString(ex.err));
  return STK_OK;
}

stk_status stokes_fmm_set_pass_events(void **events, int32_t capacity, const char **names,
                                      int32_t *count) {
  if (events && capacity < 2) return stk::report_error(STK_EINVAL, "capacity must be >= 2");
  g_hooks.events = reinterpret_cast<cudaEvent_t *>(events);
  g_hooks.capacity = events ? capacity : 0;
  g_hooks.names = events ? names : nullptr;
  g_hooks.count = events ? count : nullptr;
  if (count) *count = 0;
  return STK_OK;
}

}  // extern "C"
