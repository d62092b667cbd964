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
#include <cuda.h>  // driver API types only; the functions are reached through the runtime

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

// The host-side name of g_noalloc_scratch is not a device address.  Its device
// address belongs to the module loaded into one CUDA context: after
// cudaDeviceReset, or when the primary context is released and created again,
// the module is loaded anew and the buffer may sit elsewhere.  So the address
// is looked up with the device current and cached per device together with
// the identity of the context it was looked up in (cuCtxGetId: unique for the
// life of the process); a call in another context looks it up again.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

struct ScratchCache {
  unsigned long long ctx_id = 0;
  void *addr = nullptr;
};

std::mutex g_mu;
ScratchCache g_cache[kMaxDevices];
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_driver_looked_up = false;

// Identity of the calling thread's current context (0 when it cannot be
// read; the cache is then bypassed and the address looked up on every call).
unsigned long long current_context_id() {
  if (!g_driver_looked_up) {
    g_driver_looked_up = true;
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
            cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
            cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
      g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the buffer in the current context.  With lookup == false
// only an address already looked up in this context is returned (NULL
// otherwise).  cudaGetSymbolAddress makes the device's primary context current
// on this thread if none was, so the context is read again after it.
stk_status scratch_address(void **addr, bool lookup) {
  *addr = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return stk::report_error(STK_ECUDA, "stokes_sl_eval_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  ScratchCache &c = g_cache[dev];
  const unsigned long long id = current_context_id();
  if (id != 0 && c.addr && c.ctx_id == id) {
    *addr = c.addr;
    return STK_OK;
  }
  if (!lookup) return STK_OK;
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return stk::report_error(STK_ECUDA,
                             "stokes_sl_eval_noalloc: cudaGetSymbolAddress of the scratch failed");
  const unsigned long long id_now = current_context_id();
  c.ctx_id = id_now;
  c.addr = id_now != 0 ? p : nullptr;
  *addr = p;
  return STK_OK;
}

}  // namespace

namespace stk {
// Identity of the calling thread's current CUDA context (0 if it cannot be
// read), for caches of per-context handles elsewhere in the library.
unsigned long long context_id() {
  std::lock_guard<std::mutex> lock(g_mu);
  return current_context_id();
}

// The buffer's address in the current context if stokes_sl_eval_noalloc has
// run there (its error word is read by stokes_device_status(NULL, 0)).
stk_status noalloc_scratch(void **addr, size_t *bytes) {
  *bytes = kNoAllocScratchBytes;
  const stk_status s = scratch_address(addr, false);
  if (s != STK_OK) return s;
  if (!*addr)
    return report_error(STK_EINVAL,
                        "stokes_device_status: stokes_sl_eval_noalloc has not run in this context");
  return STK_OK;
}
}  // namespace stk

extern "C" stk_status stokes_sl_eval_noalloc(const double *src, const double *f, const double *w,
                                             const double *h, int64_t ns, const double *trg,
                                             int64_t nt, double mu, double *out,
                                             const stk_opts *opts, void *stream) {
  if (!opts) return stk::report_error(STK_EINVAL, "opts is NULL");
  if (ns > kNoAllocMaxPoints || nt > kNoAllocMaxPoints)
    return stk::report_error(STK_EUNSUPPORTED,
                             "stokes_sl_eval_noalloc: ns and nt must not exceed 65536");
  void *scratch = nullptr;
  stk_status s = scratch_address(&scratch, true);
  if (s != STK_OK) return s;
  // Use the requested source splits, or fewer until the workspace fits the buffer.
  // The default work-item shape is named explicitly: this entry point keeps the
  // engine form (bounded waits, device status) at every size.
  stk_opts o = *opts;
  if (o.tile_config < 0) o.tile_config = 0;
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
