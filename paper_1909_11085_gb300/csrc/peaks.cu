// peaks.cu -- throughput probes of the arithmetic pipes the summation kernels
// are bound by, so that their rooflines use rates measured on the GPU at hand
// (FP32 FMA, packed two-wide FP32 FMA, FP64 FMA, the MUFU reciprocal square
// root).  Each thread runs kChains independent dependent chains of one
// operation; a grid of resident CTAs on every SM keeps the pipe full.  The
// caller times the launch with events on the stream and divides the returned
// operation count by that time.
#include "../../include/stokesgpu.h"
#include "prep.cuh"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

__device__ __forceinline__ float probe_rsqrt(float x) {
  float r;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// op 0: FFMA, 1: packed FFMA2, 2: DFMA, 3: MUFU rsqrt.  a = a * b + c keeps
// every chain at its fixed point near 1 (b < 1, c = 1 - b), so no value
// overflows or becomes subnormal.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_pipe_probe(int32_t iters, float bf, double bd,
                                                              void *sink) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (OP == 0) {
    float a[kChains];
    const float c = 1.0f - bf;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (float)(k + (int)(tid & 7));
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], bf, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    reinterpret_cast<float *>(sink)[tid] = s;
  } else if (OP == 1) {
    float2 a[kChains];
    const float2 b2 = make_float2(bf, bf), c2 = make_float2(1.0f - bf, 1.0f - bf);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(1.0f + 1e-3f * k, 1.0f - 1e-3f * k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    reinterpret_cast<float *>(sink)[tid] = s;
  } else if (OP == 2) {
    double a[kChains];
    const double c = 1.0 - bd;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(k + (int)(tid & 7));
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], bd, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    reinterpret_cast<float *>(sink)[tid] = (float)s;
  } else {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = bf + 1e-3f * (float)(k + (int)(tid & 7));
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = probe_rsqrt(a[k]);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    reinterpret_cast<float *>(sink)[tid] = s;
  }
}

template <int OP>
cudaError_t launch_probe(int blocks, int32_t iters, void *sink, cudaStream_t st) {
  k_pipe_probe<OP><<<blocks, kProbeThreads, 0, st>>>(iters, 0.999999f, 0.999999, sink);
  stk::count_launches(1);
  return cudaGetLastError();
}

// The library's integer-pipe conversions beside CUDA's (stokes_convert_check).
__global__ void k_convert_check(const double *in, int64_t n, float *narrow_own,
                                float *narrow_cuda, double *widen_own, double *widen_cuda) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = in[i];
  const float c = __double2float_rn(v);
  narrow_own[i] = stk::f64_to_f32_rn(v);
  narrow_cuda[i] = c;
  widen_own[i] = stk::f32_to_f64(c);
  widen_cuda[i] = (double)c;
}

}  // namespace

extern "C" {

stk_status stokes_pipe_probe_size(size_t *sink_bytes) {
  if (!sink_bytes) return stk::report_error(STK_EINVAL, "sink_bytes is NULL");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return stk::report_error(STK_ECUDA, "cannot query the device");
  *sink_bytes = sizeof(float) * (size_t)sms * kProbeBlocksPerSm * kProbeThreads;
  return STK_OK;
}

stk_status stokes_pipe_probe(int32_t op, int32_t iters, void *sink, size_t sink_bytes,
                             double *ops, void *stream) {
  if (op < 0 || op > 3) return stk::report_error(STK_EINVAL, "op must be 0..3");
  if (iters < 1) return stk::report_error(STK_EINVAL, "iters must be >= 1");
  if (!sink || !ops) return stk::report_error(STK_EINVAL, "sink/ops is NULL");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return stk::report_error(STK_ECUDA, "cannot query the device");
  const int blocks = sms * kProbeBlocksPerSm;
  if (sink_bytes < sizeof(float) * (size_t)blocks * kProbeThreads)
    return stk::report_error(STK_ENOMEM, "sink smaller than stokes_pipe_probe_size");
  const double threads = (double)blocks * kProbeThreads;
  // flops for the FMA forms (2 per FMA, 4 per packed FMA), evaluations for rsqrt
  const double per = op == 1 ? 4.0 : (op == 3 ? 1.0 : 2.0);
  *ops = threads * (double)iters * kChains * per;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (op) {
    case 0: e = launch_probe<0>(blocks, iters, sink, st); break;
    case 1: e = launch_probe<1>(blocks, iters, sink, st); break;
    case 2: e = launch_probe<2>(blocks, iters, sink, st); break;
    default: e = launch_probe<3>(blocks, iters, sink, st); break;
  }
  if (e != cudaSuccess) return stk::report_error(STK_ECUDA, cudaGetErrorString(e));
  return STK_OK;
}

stk_status stokes_convert_check(const double *in, int64_t n, float *narrow_own,
                                float *narrow_cuda, double *widen_own, double *widen_cuda,
                                void *stream) {
  if (n < 0) return stk::report_error(STK_EINVAL, "n must be >= 0");
  if (n == 0) return STK_OK;
  if (!in || !narrow_own || !narrow_cuda || !widen_own || !widen_cuda)
    return stk::report_error(STK_EINVAL, "a pointer is NULL");
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffff) return stk::report_error(STK_EINVAL, "n too large");
  k_convert_check<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      in, n, narrow_own, narrow_cuda, widen_own, widen_cuda);
  stk::count_launches(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return stk::report_error(STK_ECUDA, cudaGetErrorString(e));
  return STK_OK;
}

}  // extern "C"
