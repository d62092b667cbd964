// noalloc.cu -- a single-layer direct sum for callers that cannot allocate
// device memory.
//
// Some callers may not call cudaMalloc at the moment they need a velocity:
// code that runs inside a host application which owns every device
// allocation (a solver framework or plugin host that hands out no scratch),
// real-time pipelines that forbid allocation after start-up because
// cudaMalloc can synchronise the device and its latency is unbounded, and
// processes running under a fixed device-memory budget.  For them this file
// keeps one fixed scratch buffer in device memory, declared at file scope, and
// stokes_sl_eval_noalloc() evaluates the single layer with it in place of a
// caller workspace.
//
// The buffer is kNoAllocScratchBytes (32 MiB); every GPU that loads the
// library holds it until the process exits.  It is shared by all calls and
// keeps the last call's contents; each call zeroes what must start at zero
// (the work-queue counters) and writes every other word before reading it.
// Calls whose kernels overlap on the GPU (for example on two streams) race on
// the buffer and must be serialised by the caller.
#include <mutex>

#include "../../include/stokesgpu.h"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr int64_t kNoAllocMaxPoints = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// The host-side name of g_noalloc_scratch is not a device address.  The
// device address is looked up on the first call on each device, with that
// device current, and kept.
stk_status scratch_address(void **addr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return stk::report_error(STK_ECUDA, "stokes_sl_eval_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return stk::report_error(STK_ECUDA,
                               "stokes_sl_eval_noalloc: cudaGetSymbolAddress of the scratch failed");
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  return STK_OK;
}

}  // namespace

extern "C" stk_status stokes_sl_eval_noalloc(const double *src, const double *f, const double *w,
                                             const double *h, int64_t ns, const double *trg,
                                             int64_t nt, double mu, double *out,
                                             const stk_opts *opts, void *stream) {
  if (!opts) return stk::report_error(STK_EINVAL, "opts is NULL");
  if (ns > kNoAllocMaxPoints || nt > kNoAllocMaxPoints)
    return stk::report_error(STK_EUNSUPPORTED,
                             "stokes_sl_eval_noalloc: ns and nt must not exceed 65536");
  void *scratch = nullptr;
  stk_status s = scratch_address(&scratch);
  if (s != STK_OK) return s;
  // Use the requested source splits, or fewer until the workspace fits the buffer.
  stk_opts o = *opts;
  size_t need = 0;
  s = stokes_direct_workspace_size(ns < 0 ? 0 : ns, nt < 0 ? 0 : nt, 1, &o, &need);
  if (s != STK_OK) return s;
  const int32_t fewer[] = {8, 4, 2, 1};
  for (int i = 0; i < 4 && need > kNoAllocScratchBytes; ++i) {
    if (o.source_splits != 0 && o.source_splits <= fewer[i]) continue;
    o.source_splits = fewer[i];
    s = stokes_direct_workspace_size(ns, nt, 1, &o, &need);
    if (s != STK_OK) return s;
  }
  if (need > kNoAllocScratchBytes)
    return stk::report_error(STK_EUNSUPPORTED,
                             "stokes_sl_eval_noalloc: problem does not fit the 32 MiB scratch");
  return stokes_sl_eval(src, f, w, h, ns, trg, nt, mu, out, &o, scratch, kNoAllocScratchBytes,
                        stream);
}
