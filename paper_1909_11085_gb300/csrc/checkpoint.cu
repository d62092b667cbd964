// checkpoint.cu -- singular and near-singular evaluation on patch surfaces by
// check-point extrapolation (Sec. 3.1, "Singular and near-singular integral
// quadrature").
//
// Per call, for targets x with closest surface points y and unit normals n:
//  1. k_upsample: the density on each patch's (q+1) x (q+1) Clenshaw-Curtis
//     nodes is interpolated (tensor-product, degree q) to the fine
//     discretisation, m x m sub-patches (m = 2^eta) with the same node set;
//     one CTA per patch, the 1-D interpolation matrix built in shared memory
//     by the barycentric formula, applied along u and then along v (FP64);
//  2. k_check_points: c_i = y - (R + i r) n, i = 0..p;
//  3. the smooth quadrature sum on the fine nodes at the check points: the
//     library's own direct sums (mixed FP32/FP64 engine or FP64);
//  4. k_extrapolate: u(x) = sum_i e_i u(c_i), with e_i the Lagrange weights
//     of the nodes t_i = R + i r at the target's t = (y - x) . n (FP64).
// Node orderings: coarse nodes i-major per patch; fine nodes by patch, then
// sub-patch (su-major), then node (i-major).
#include <cmath>

#include "../../include/stokesgpu.h"
#include "common.cuh"
#include "prep.cuh"

namespace stk {
stk_status report_error(stk_status s, const char *msg);
}

namespace {

using namespace stk;

constexpr int kMaxQ = 12;    // nodes per patch side q + 1 <= 13
constexpr int kMaxEta = 3;   // m = 2^eta <= 8 sub-patches per side
constexpr int kMaxP = 15;    // check points p + 1 <= 16
constexpr int kUpThreads = 128;

size_t up_smem_bytes(int q, int m, int ncomp) {
  const size_t n1 = (size_t)q + 1, nf = (size_t)m * n1;
  return sizeof(double) * (nf * n1 + n1 * n1 * ncomp + nf * n1 * ncomp);
}

// coarse [npatch][(q+1)^2][ncomp] -> fine [npatch][m^2][(q+1)^2][ncomp]
__global__ void __launch_bounds__(kUpThreads) k_upsample(const double *__restrict__ coarse,
                                                         int q, int m, int ncomp,
                                                         double *__restrict__ fine) {
  extern __shared__ double sh[];
  const int n1 = q + 1, nf = m * n1;
  double *U1 = sh;                     // [nf][n1]
  double *C = U1 + nf * n1;            // [n1][n1][ncomp]
  double *T1 = C + n1 * n1 * ncomp;    // [nf][n1][ncomp]: interpolated along u
  const int patch = blockIdx.x;
  const double *src = coarse + (size_t)patch * n1 * n1 * ncomp;
  for (int e = threadIdx.x; e < n1 * n1 * ncomp; e += blockDim.x) C[e] = src[e];
  // U1[a][j]: degree-q interpolant through the CC nodes x_j = cos(j pi / q),
  // second barycentric form with weights (-1)^j, halved at both ends
  const double pi = 3.14159265358979323846;
  for (int a = threadIdx.x; a < nf; a += blockDim.x) {
    const int s = a / n1, i = a % n1;
    const double t = -1.0 + 2.0 * s / m + (cos(pi * i / q) + 1.0) / m;
    int hit = -1;
    double den = 0.0;
    for (int j = 0; j < n1; ++j) {
      const double d = t - cos(pi * j / q);
      if (d == 0.0) hit = j;
    }
    for (int j = 0; j < n1; ++j) {
      double c;
      if (hit >= 0) {
        c = j == hit ? 1.0 : 0.0;
      } else {
        const double wj = ((j & 1) ? -1.0 : 1.0) * ((j == 0 || j == q) ? 0.5 : 1.0);
        c = wj / (t - cos(pi * j / q));
      }
      U1[a * n1 + j] = c;
      den += c;
    }
    for (int j = 0; j < n1; ++j) U1[a * n1 + j] /= den;
  }
  __syncthreads();
  // along u: T1[a][j][c] = sum_i U1[a][i] C[i][j][c]
  for (int e = threadIdx.x; e < nf * n1 * ncomp; e += blockDim.x) {
    const int c = e % ncomp, j = (e / ncomp) % n1, a = e / (ncomp * n1);
    double acc = 0.0;
    for (int i = 0; i < n1; ++i) acc = fma(U1[a * n1 + i], C[(i * n1 + j) * ncomp + c], acc);
    T1[e] = acc;
  }
  __syncthreads();
  // along v, written in the fine order (sub-patch su-major, node i-major)
  double *dst = fine + (size_t)patch * nf * nf * ncomp;
  for (int e = threadIdx.x; e < nf * nf * ncomp; e += blockDim.x) {
    const int c = e % ncomp, b = (e / ncomp) % nf, a = e / (ncomp * nf);
    double acc = 0.0;
    for (int j = 0; j < n1; ++j) acc = fma(U1[b * n1 + j], T1[(a * n1 + j) * ncomp + c], acc);
    const int su = a / n1, i = a % n1, sv = b / n1, jj = b % n1;
    const size_t o = ((size_t)(su * m + sv) * n1 * n1 + (size_t)i * n1 + jj) * ncomp + c;
    dst[o] = acc;
  }
}

// c[t][i] = y[t] - (R + i r) n[t]
__global__ void k_check_points(int64_t nt, int p, double R, double r,
                               const double *__restrict__ y, const double *__restrict__ n,
                               double *__restrict__ c) {
  const int64_t total = nt * (p + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / (p + 1);
    const int i = (int)(e % (p + 1));
    const double d = R + i * r;
#pragma unroll
    for (int k = 0; k < 3; ++k) c[3 * e + k] = y[3 * t + k] - d * n[3 * t + k];
  }
}

// out[t] (+)= sum_i e_i(t_x) uc[t][i], t_x = (y - x) . n
__global__ void k_extrapolate(int64_t nt, int p, double R, double r, const double *__restrict__ x,
                              const double *__restrict__ y, const double *__restrict__ n,
                              const double *__restrict__ uc, int accumulate,
                              double *__restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt;
       t += (int64_t)gridDim.x * blockDim.x) {
    double tx = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) tx = fma(y[3 * t + k] - x[3 * t + k], n[3 * t + k], tx);
    double u[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i <= p; ++i) {
      const double ti = R + i * r;
      double e = 1.0;
      for (int j = 0; j <= p; ++j)
        if (j != i) e *= (tx - (R + j * r)) / (ti - (R + j * r));
      const double *v = uc + 3 * ((size_t)t * (p + 1) + i);
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] = fma(e, v[k], u[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) out[3 * t + k] = accumulate ? out[3 * t + k] + u[k] : u[k];
  }
}

// Rank-completing term of the boundary-integral equation: M = sum_m w_m n_m
// phi_m^T over the coarse nodes, in two fixed-order stages (per-block partial
// sums, then every apply block adds the partials in block order), and
// out[t] += M n[t].
constexpr int kNullBlocks = 128;
constexpr int kNullThreads = 256;

__global__ void __launch_bounds__(kNullThreads) k_null_partial(int64_t n, const double *__restrict__ nn,
                                                               const double *__restrict__ w,
                                                               const double *__restrict__ phi,
                                                               double *__restrict__ part) {
  __shared__ double s[9][kNullThreads];
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  for (int64_t m = b0 + threadIdx.x; m < b1; m += blockDim.x) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) acc[3 * i + j] = fma(w[m] * nn[3 * m + i], phi[3 * m + j], acc[3 * i + j]);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int k = 0; k < 9; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 9) part[9 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNullThreads) k_null_apply(int64_t nt, int nparts,
                                                             const double *__restrict__ part,
                                                             const double *__restrict__ tn,
                                                             double *__restrict__ out) {
  __shared__ double M[9];
  if (threadIdx.x < 9) {
    double v = 0.0;
    for (int b = 0; b < nparts; ++b) v += part[9 * b + threadIdx.x];
    M[threadIdx.x] = v;
  }
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt;
       t += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
      out[3 * t + i] += M[3 * i] * tn[3 * t] + M[3 * i + 1] * tn[3 * t + 1] + M[3 * i + 2] * tn[3 * t + 2];
  }
}

int grid_1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 65535) g = 65535;
  return (int)g;
}

stk_status check_shape(int32_t npatch, int32_t q, int32_t eta) {
  if (npatch < 0) return report_error(STK_EINVAL, "npatch must be >= 0");
  if (q < 2 || q > kMaxQ) return report_error(STK_EUNSUPPORTED, "q must be in [2, 12]");
  if (eta < 0 || eta > kMaxEta) return report_error(STK_EUNSUPPORTED, "eta must be in [0, 3]");
  return STK_OK;
}

struct CpLayout {
  size_t f_up = 0, phi_up = 0, chk, uc, direct, total;
  size_t direct_bytes;
};

size_t take(size_t &off, size_t bytes) {
  const size_t o = off;
  off += (bytes + 255) & ~(size_t)255;
  return o;
}

stk_status cp_layout(int32_t kernels, int32_t npatch, int32_t q, int32_t eta, int64_t nt,
                     int32_t p, const stk_opts *opts, CpLayout &L) {
  const int64_t m = (int64_t)1 << eta;
  const int64_t nf = (int64_t)npatch * m * m * (q + 1) * (q + 1);
  const int64_t nc = nt * (p + 1);
  size_t off = 0;
  if (kernels & 1) L.f_up = take(off, sizeof(double) * 3 * (size_t)nf);
  if (kernels & 2) L.phi_up = take(off, sizeof(double) * 3 * (size_t)nf);
  L.chk = take(off, sizeof(double) * 3 * (size_t)nc);
  L.uc = take(off, sizeof(double) * 3 * (size_t)nc);
  stk_status s = stokes_direct_workspace_size(nf, nc, kernels, opts, &L.direct_bytes);
  if (s != STK_OK) return s;
  L.direct = take(off, L.direct_bytes);
  L.total = off + 256;
  return STK_OK;
}

}  // namespace

extern "C" {

stk_status stokes_upsample_patches(const double *coarse, int32_t npatch, int32_t q, int32_t eta,
                                   int32_t ncomp, double *fine, void *stream) {
  stk_status s = check_shape(npatch, q, eta);
  if (s != STK_OK) return s;
  if (ncomp < 1 || ncomp > 3) return report_error(STK_EINVAL, "ncomp must be 1, 2 or 3");
  if (npatch == 0) return STK_OK;
  if (!coarse || !fine) return report_error(STK_EINVAL, "coarse/fine is NULL");
  const int m = 1 << eta;
  k_upsample<<<npatch, kUpThreads, up_smem_bytes(q, m, ncomp),
               reinterpret_cast<cudaStream_t>(stream)>>>(coarse, q, m, ncomp, fine);
  count_launches(1);
  if (cudaGetLastError() != cudaSuccess) return report_error(STK_ECUDA, "k_upsample launch failed");
  return STK_OK;
}

stk_status stokes_checkpoint_workspace_size(int32_t kernels, int32_t npatch, int32_t q,
                                            int32_t eta, int64_t nt, int32_t p,
                                            const stk_opts *opts, size_t *bytes) {
  if (!bytes) return report_error(STK_EINVAL, "bytes is NULL");
  if (kernels < 1 || kernels > 3) return report_error(STK_EINVAL, "kernels must be 1, 2 or 3");
  stk_status s = check_shape(npatch, q, eta);
  if (s != STK_OK) return s;
  if (nt < 0 || p < 0 || p > kMaxP) return report_error(STK_EINVAL, "nt >= 0 and p in [0, 15]");
  CpLayout L;
  s = cp_layout(kernels, npatch, q, eta, nt, p, opts, L);
  if (s != STK_OK) return s;
  *bytes = L.total;
  return STK_OK;
}

stk_status stokes_checkpoint_eval(int32_t kernels, const double *f, const double *phi,
                                  int32_t npatch, int32_t q, int32_t eta, const double *fine_pts,
                                  const double *fine_nrm, const double *fine_w,
                                  const double *fine_h, const double *trg, const double *cp_y,
                                  const double *cp_n, int64_t nt, double R, double r, int32_t p,
                                  double mu, double *out, const stk_opts *opts, void *workspace,
                                  size_t workspace_bytes, void *stream) {
  if (!opts) return report_error(STK_EINVAL, "opts is NULL");
  size_t need = 0;
  stk_status s = stokes_checkpoint_workspace_size(kernels, npatch, q, eta, nt, p, opts, &need);
  if (s != STK_OK) return s;
  if (!(R > 0.0) || !(r > 0.0) || !std::isfinite(R) || !std::isfinite(r))
    return report_error(STK_EINVAL, "R and r must be finite and > 0");
  if (nt == 0) return STK_OK;
  if (!trg || !cp_y || !cp_n || !out) return report_error(STK_EINVAL, "trg/cp_y/cp_n/out is NULL");
  if (npatch > 0 && (!fine_pts || !fine_w || ((kernels & 1) && !f) ||
                     ((kernels & 2) && (!phi || !fine_nrm))))
    return report_error(STK_EINVAL, "a density or fine-geometry array is NULL");
  if (!workspace || workspace_bytes < need) return report_error(STK_ENOMEM, "workspace too small");
  CpLayout L;
  s = cp_layout(kernels, npatch, q, eta, nt, p, opts, L);
  if (s != STK_OK) return s;
  const uintptr_t u = reinterpret_cast<uintptr_t>(workspace);
  char *ws = reinterpret_cast<char *>((u + 255) & ~(uintptr_t)255);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int m = 1 << eta;
  const int64_t nf = (int64_t)npatch * m * m * (q + 1) * (q + 1);
  const int64_t nc = nt * (p + 1);
  double *f_up = (kernels & 1) ? reinterpret_cast<double *>(ws + L.f_up) : nullptr;
  double *phi_up = (kernels & 2) ? reinterpret_cast<double *>(ws + L.phi_up) : nullptr;
  double *chk = reinterpret_cast<double *>(ws + L.chk);
  double *uc = reinterpret_cast<double *>(ws + L.uc);
  void *dws = ws + L.direct;
  // 1. upsampled densities
  if (f_up && (s = stokes_upsample_patches(f, npatch, q, eta, 3, f_up, stream)) != STK_OK)
    return s;
  if (phi_up && (s = stokes_upsample_patches(phi, npatch, q, eta, 3, phi_up, stream)) != STK_OK)
    return s;
  // 2. check points
  k_check_points<<<grid_1d(nc, 256), 256, 0, st>>>(nt, p, R, r, cp_y, cp_n, chk);
  count_launches(1);
  if (cudaGetLastError() != cudaSuccess)
    return report_error(STK_ECUDA, "k_check_points launch failed");
  // 3. smooth quadrature on the fine nodes at the check points
  stk_opts o = *opts;
  o.accumulate = 0;
  if (kernels == 1)
    s = stokes_sl_eval(fine_pts, f_up, fine_w, fine_h, nf, chk, nc, mu, uc, &o, dws,
                       L.direct_bytes, stream);
  else if (kernels == 2)
    s = stokes_dl_eval(fine_pts, fine_nrm, phi_up, fine_w, fine_h, nf, chk, nc, uc, &o, dws,
                       L.direct_bytes, stream);
  else
    s = stokes_sldl_eval(fine_pts, f_up, fine_nrm, phi_up, fine_w, fine_h, nf, chk, nc, mu, uc,
                         &o, dws, L.direct_bytes, stream);
  if (s != STK_OK) return s;
  // 4. extrapolation to the targets
  k_extrapolate<<<grid_1d(nt, 256), 256, 0, st>>>(nt, p, R, r, trg, cp_y, cp_n, uc,
                                                  opts->accumulate, out);
  count_launches(1);
  if (cudaGetLastError() != cudaSuccess)
    return report_error(STK_ECUDA, "k_extrapolate launch failed");
  return STK_OK;
}

stk_status stokes_bie_workspace_size(int32_t npatch, int32_t q, int32_t eta, int32_t p,
                                     const stk_opts *opts, size_t *bytes) {
  const int64_t nc = (int64_t)npatch * (q + 1) * (q + 1);
  stk_status s = stokes_checkpoint_workspace_size(2, npatch, q, eta, nc, p, opts, bytes);
  if (s != STK_OK) return s;
  *bytes += sizeof(double) * 9 * kNullBlocks + 256;
  return STK_OK;
}

stk_status stokes_bie_matvec(const double *phi, int32_t npatch, int32_t q, int32_t eta,
                             const double *nodes, const double *nodes_n, const double *nodes_w,
                             const double *fine_pts, const double *fine_nrm, const double *fine_w,
                             const double *fine_h, double R, double r, int32_t p, double *out,
                             const stk_opts *opts, void *workspace, size_t workspace_bytes,
                             void *stream) {
  if (!opts) return report_error(STK_EINVAL, "opts is NULL");
  size_t need = 0;
  stk_status s = stokes_bie_workspace_size(npatch, q, eta, p, opts, &need);
  if (s != STK_OK) return s;
  const int64_t nc = (int64_t)npatch * (q + 1) * (q + 1);
  if (nc == 0) return STK_OK;
  if (!phi || !nodes || !nodes_n || !nodes_w || !out)
    return report_error(STK_EINVAL, "phi/nodes/nodes_n/nodes_w/out is NULL");
  if (!workspace || workspace_bytes < need) return report_error(STK_ENOMEM, "workspace too small");
  const size_t cp_bytes = need - sizeof(double) * 9 * kNullBlocks - 256;
  s = stokes_checkpoint_eval(2, nullptr, phi, npatch, q, eta, fine_pts, fine_nrm, fine_w, fine_h,
                             nodes, nodes, nodes_n, nc, R, r, p, 1.0, out, opts, workspace,
                             cp_bytes, stream);
  if (s != STK_OK) return s;
  const uintptr_t u = reinterpret_cast<uintptr_t>(workspace) + cp_bytes;
  double *part = reinterpret_cast<double *>((u + 255) & ~(uintptr_t)255);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_null_partial<<<kNullBlocks, kNullThreads, 0, st>>>(nc, nodes_n, nodes_w, phi, part);
  k_null_apply<<<grid_1d(nc, kNullThreads), kNullThreads, 0, st>>>(nc, kNullBlocks, part, nodes_n,
                                                                   out);
  count_launches(2);
  if (cudaGetLastError() != cudaSuccess) return report_error(STK_ECUDA, "null-space term launch failed");
  return STK_OK;
}

}  // extern "C"
