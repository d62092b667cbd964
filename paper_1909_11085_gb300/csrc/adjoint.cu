// adjoint.cu -- gradients of L = sum_i g_i . u(x_i), u = SL[f] + DL[phi], with
// respect to the densities, the source positions and normals and the target
// positions.  The pair terms are the derivatives of the two kernels (the
// single layer of Eq. "sl_stokes", the double layer of Sec. 2.1), with d = x - y,
// q = w f / (8 pi mu), psi = 6 w phi / (8 pi):
//   s = g.q/r + (d.g)(d.q)/r^3
//     ds/dq   = g/r + d (d.g)/r^3
//     ds/dd   = [g (d.q) + q (d.g) - (g.q) d]/r^3 - 3 (d.g)(d.q) d/r^5
//   t = (d.g)(d.psi)(d.n)/r^5
//     dt/dpsi = (d.g)(d.n) d/r^5,   dt/dn = (d.g)(d.psi) d/r^5
//     dt/dd   = [g (d.psi)(d.n) + psi (d.g)(d.n) + n (d.g)(d.psi)]/r^5 - 5 t d/r^2
// dL/dx_i = sum_j d(s + t)/dd,  dL/dy_j = -sum_i d(s + t)/dd.  Nothing O(N^2) is
// stored: two passes recompute the pair terms.  The source-major pass gives,
// per source, dL/df, dL/dphi, dL/dn and dL/dy (a sum over targets); the
// target-major pass gives dL/dx (a sum over sources).
//
// Both passes tile their inputs through shared memory in CTAs of 128 output
// points (Morton-sorted, so a CTA is spatially compact) and split the inputs
// over blockIdx.y for occupancy.  The mixed form works in FP32 in the CTA's
// local frame (positions split hi/lo as in the forward records) with a
// two-sum per tile; a pair with |r| < alpha h_j is left out of the FP32 sum
// and listed for its output point (up to kAdjNearCap); k_adj_near then
// evaluates the listed pairs in FP64 (difference, 1/|r| and the pair terms) in
// input order and adds them to the point's partial.  Keeping FP64 out of the
// FP32 pass keeps its registers, and so its occupancy, those of FP32 code.
// An output point with more near pairs than the list holds is rescanned by
// k_adj_near with the FP32 pass's own frame and test.  The FP64 form does all
// of it in double.
#include <cfloat>

#include "common.cuh"
#include "prep.cuh"

namespace stk {

constexpr int kAdjThreads = 128;

// Pair terms.  For the source-major pass the own point is the source (q, psi,
// n fixed) and g comes from the input; for the target-major pass the own
// point is the target (g fixed).  acc layout (source-major): 0..2 ds/dq,
// 3..5 dt/dpsi / psi-scale, 6..8 dt/dn, 9..11 -d(s+t)/dd; (target-major):
// 0..2 d(s+t)/dd.
template <typename R, bool SRC>
__device__ __forceinline__ void adj_pair(R dx, R dy, R dz, R ri, const R (&g)[3], const R (&q)[3],
                                         const R (&p)[3], const R (&n)[3], int has_sl, int has_dl,
                                         R *acc) {
  const R ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2;
  const R dg = dx * g[0] + dy * g[1] + dz * g[2];
  R gx = 0, gy = 0, gz = 0;
  if (has_sl) {
    const R dq = dx * q[0] + dy * q[1] + dz * q[2];
    const R gq = g[0] * q[0] + g[1] * q[1] + g[2] * q[2];
    if (SRC) {
      const R c = dg * ri3;
      acc[0] += g[0] * ri + dx * c;
      acc[1] += g[1] * ri + dy * c;
      acc[2] += g[2] * ri + dz * c;
    }
    const R a = dq * ri3, b = dg * ri3, cd = -gq * ri3 - R(3) * dg * dq * ri5;
    gx += g[0] * a + q[0] * b + dx * cd;
    gy += g[1] * a + q[1] * b + dy * cd;
    gz += g[2] * a + q[2] * b + dz * cd;
  }
  if (has_dl) {
    const R dp = dx * p[0] + dy * p[1] + dz * p[2];
    const R dn = dx * n[0] + dy * n[1] + dz * n[2];
    const R a = dg * dn * ri5, b = dg * dp * ri5;
    if (SRC) {
      acc[3] += dx * a;
      acc[4] += dy * a;
      acc[5] += dz * a;
      acc[6] += dx * b;
      acc[7] += dy * b;
      acc[8] += dz * b;
    }
    const R e = dp * dn * ri5, t5 = R(5) * b * dn * ri2;  // 5 t / r^2, t = (d.g)(d.psi)(d.n)/r^5
    gx += g[0] * e + p[0] * a + n[0] * b - dx * t5;
    gy += g[1] * e + p[1] * a + n[1] * b - dy * t5;
    gz += g[2] * e + p[2] * a + n[2] * b - dz * t5;
  }
  if (SRC) {
    acc[9] -= gx;
    acc[10] -= gy;
    acc[11] -= gz;
  } else {
    acc[0] += gx;
    acc[1] += gy;
    acc[2] += gz;
  }
}

template <bool SRC>
struct NAcc {
  static constexpr int value = SRC ? 12 : 3;
};

// ---------------------------------------------------------------- FP32 pass
template <bool SRC>
__global__ void __launch_bounds__(kAdjThreads) k_adj_mixed(AdjParams A) {
  constexpr int NA = NAcc<SRC>::value;
  __shared__ float4 sP[kAdjThreads];   // local position, hh
  __shared__ float4 sG[kAdjThreads];   // g (src-major) or q (trg-major)
  __shared__ float4 sN[kAdjThreads];   // n (trg-major)
  __shared__ float4 sPs[kAdjThreads];  // psi (trg-major)
  __shared__ int32_t sI[kAdjThreads];  // caller index
  __shared__ float red[6][kAdjThreads];
  const SrcRec *orec = reinterpret_cast<const SrcRec *>(A.out_rec);
  const SrcRec *irec = reinterpret_cast<const SrcRec *>(A.in_rec);
  const int tid = threadIdx.x;
  const int64_t o_sorted = (int64_t)blockIdx.x * kAdjThreads + tid;
  const bool valid = o_sorted < A.nout;
  const int64_t oc = valid ? A.operm[o_sorted] : A.operm[(int64_t)blockIdx.x * kAdjThreads];

  // CTA origin: centre of the output points' bounding box, as hi/lo splits
  const SrcRec Ro = orec[oc];
  const SrcRec R0 = orec[A.operm[(int64_t)blockIdx.x * kAdjThreads]];
  {
    const float r[3] = {(Ro.yh.x - R0.yh.x) + (Ro.q.w - R0.q.w),
                        (Ro.yh.y - R0.yh.y) + (Ro.n.w - R0.n.w),
                        (Ro.yh.z - R0.yh.z) + (Ro.p.w - R0.p.w)};
    for (int k = 0; k < 3; ++k) {
      red[k][tid] = valid ? r[k] : INFINITY;
      red[3 + k][tid] = valid ? r[k] : -INFINITY;
    }
  }
  __syncthreads();
  for (int s = kAdjThreads / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int k = 0; k < 3; ++k) {
        red[k][tid] = fminf(red[k][tid], red[k][tid + s]);
        red[3 + k][tid] = fmaxf(red[3 + k][tid], red[3 + k][tid + s]);
      }
    __syncthreads();
  }
  float oh[3], ol[3];
  {
    const double o[3] = {(double)R0.yh.x + (double)R0.q.w + 0.5 * ((double)red[0][0] + red[3][0]),
                         (double)R0.yh.y + (double)R0.n.w + 0.5 * ((double)red[1][0] + red[4][0]),
                         (double)R0.yh.z + (double)R0.p.w + 0.5 * ((double)red[2][0] + red[5][0])};
    for (int k = 0; k < 3; ++k) split_hl(o[k], oh[k], ol[k]);
  }
  __syncthreads();
  const float ox = to_local(Ro.yh.x, Ro.q.w, oh[0], ol[0]);
  const float oy = to_local(Ro.yh.y, Ro.n.w, oh[1], ol[1]);
  const float oz = to_local(Ro.yh.z, Ro.p.w, oh[2], ol[2]);
  const float own_hh = Ro.yh.w;
  if (valid && blockIdx.y == 0) {  // the frame, for a rescan of an overflowing list
    float *fr = A.oframe + 9 * (size_t)oc;
    fr[0] = ox; fr[1] = oy; fr[2] = oz;
    fr[3] = oh[0]; fr[4] = oh[1]; fr[5] = oh[2];
    fr[6] = ol[0]; fr[7] = ol[1]; fr[8] = ol[2];
  }
  const float ov1[3] = {Ro.q.x, Ro.q.y, Ro.q.z};  // g (trg-major) or q (src-major)
  const float on[3] = {Ro.n.x, Ro.n.y, Ro.n.z};
  const float op[3] = {Ro.p.x, Ro.p.y, Ro.p.z};

  float hi[NA], lo[NA], ps[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) hi[a] = lo[a] = ps[a] = 0.f;

  const int64_t i0 = A.nin * blockIdx.y / A.nsplit, i1 = A.nin * (blockIdx.y + 1) / A.nsplit;
  for (int64_t tb = i0; tb < i1; tb += kAdjThreads) {
    const int64_t k = tb + tid;
    if (k < i1) {
      const int32_t ic = A.iperm[k];
      const SrcRec R = irec[ic];
      sP[tid] = make_float4(to_local(R.yh.x, R.q.w, oh[0], ol[0]),
                            to_local(R.yh.y, R.n.w, oh[1], ol[1]),
                            to_local(R.yh.z, R.p.w, oh[2], ol[2]), R.yh.w);
      sG[tid] = make_float4(R.q.x, R.q.y, R.q.z, 0.f);
      sN[tid] = make_float4(R.n.x, R.n.y, R.n.z, 0.f);
      sPs[tid] = make_float4(R.p.x, R.p.y, R.p.z, 0.f);
      sI[tid] = ic;
    }
    __syncthreads();
    const int m = (int)min((int64_t)kAdjThreads, i1 - tb);
    if (valid) {
      for (int kk = 0; kk < m; ++kk) {
        const float4 P = sP[kk];
        // d = x - y: source-major: x = input, y = own; target-major: x = own, y = input
        const float dx = SRC ? P.x - ox : ox - P.x, dy = SRC ? P.y - oy : oy - P.y,
                    dz = SRC ? P.z - oz : oz - P.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float hh = SRC ? own_hh : P.w;
        const bool near = r2 < hh;
        const float ri = near ? 0.f : rsqrt_ftz(r2);
        const float4 G = sG[kk];
        float g[3], q[3], pp[3], nn[3];
        if (SRC) {
          g[0] = G.x; g[1] = G.y; g[2] = G.z;
          q[0] = ov1[0]; q[1] = ov1[1]; q[2] = ov1[2];
          pp[0] = op[0]; pp[1] = op[1]; pp[2] = op[2];
          nn[0] = on[0]; nn[1] = on[1]; nn[2] = on[2];
        } else {
          const float4 N = sN[kk], Ps = sPs[kk];
          g[0] = ov1[0]; g[1] = ov1[1]; g[2] = ov1[2];
          q[0] = G.x; q[1] = G.y; q[2] = G.z;
          pp[0] = Ps.x; pp[1] = Ps.y; pp[2] = Ps.z;
          nn[0] = N.x; nn[1] = N.y; nn[2] = N.z;
        }
        adj_pair<float, SRC>(dx, dy, dz, ri, g, q, pp, nn, A.has_sl, A.has_dl, ps);
        if (near) {  // listed for the FP64 pass
          const int slot = atomicAdd(A.near_cnt + oc, 1);
          if (slot < A.near_cap) A.near_idx[(size_t)oc * A.near_cap + slot] = sI[kk];
        }
      }
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        two_sum_acc(hi[a], lo[a], ps[a]);
        ps[a] = 0.f;
      }
    }
    __syncthreads();
  }
  if (valid) {
    double *out = A.partial + ((size_t)blockIdx.y * (size_t)A.nout + (size_t)oc) * NA;
#pragma unroll
    for (int a = 0; a < NA; ++a) out[a] = (double)hi[a] + (double)lo[a];
  }
}

// ---------------------------------------------------------------- near pairs
// FP64 pair terms of output point oc with input ic (zero distance: nothing).
template <bool SRC>
__device__ __forceinline__ void adj_near_pair(const AdjParams &A, int64_t oc, int32_t ic,
                                              double (&ad)[NAcc<SRC>::value]) {
  const SrcRec *orec = reinterpret_cast<const SrcRec *>(A.out_rec);
  const SrcRec *irec = reinterpret_cast<const SrcRec *>(A.in_rec);
  const double *xa = SRC ? A.in64 + 3 * (size_t)ic : A.out64 + 3 * (size_t)oc;
  const double *ya = SRC ? A.out64 + 3 * (size_t)oc : A.in64 + 3 * (size_t)ic;
  const double ddx = xa[0] - ya[0], ddy = xa[1] - ya[1], ddz = xa[2] - ya[2];
  const double rr = ddx * ddx + ddy * ddy + ddz * ddz;
  if (!(rr > 0.0)) return;
  const SrcRec Ro = orec[oc], Ri = irec[ic];
  const double rid = 1.0 / sqrt(rr);
  // own values: g (target-major) or q, psi, n (source-major); the input's the others
  const SrcRec &S = SRC ? Ro : Ri, &Tg = SRC ? Ri : Ro;
  const double g[3] = {Tg.q.x, Tg.q.y, Tg.q.z}, q[3] = {S.q.x, S.q.y, S.q.z},
               p[3] = {S.p.x, S.p.y, S.p.z}, n[3] = {S.n.x, S.n.y, S.n.z};
  adj_pair<double, SRC>(ddx, ddy, ddz, rid, g, q, p, n, A.has_sl, A.has_dl, ad);
}

// One thread per output point: its listed near pairs, sorted by input index,
// in FP64, added to the point's first partial.  A point whose list overflowed
// is rescanned over all inputs (in index order) with the FP32 pass's frame
// and test, so the same pairs are found.
template <bool SRC>
__global__ void __launch_bounds__(kAdjThreads) k_adj_near(AdjParams A) {
  constexpr int NA = NAcc<SRC>::value;
  for (int64_t oc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; oc < A.nout;
       oc += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = A.near_cnt[oc];
    if (c == 0) continue;
    double ad[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) ad[a] = 0.0;
    if (c <= A.near_cap) {
      int32_t idx[kAdjNearCap];
      for (int k = 0; k < c; ++k) {  // insertion sort
        const int32_t v = A.near_idx[(size_t)oc * A.near_cap + k];
        int m = k;
        while (m > 0 && idx[m - 1] > v) {
          idx[m] = idx[m - 1];
          --m;
        }
        idx[m] = v;
      }
      for (int k = 0; k < c; ++k) adj_near_pair<SRC>(A, oc, idx[k], ad);
    } else {
      const SrcRec *orec = reinterpret_cast<const SrcRec *>(A.out_rec);
      const SrcRec *irec = reinterpret_cast<const SrcRec *>(A.in_rec);
      const float *fr = A.oframe + 9 * (size_t)oc;
      const float ox = fr[0], oy = fr[1], oz = fr[2];
      const float oh[3] = {fr[3], fr[4], fr[5]}, ol[3] = {fr[6], fr[7], fr[8]};
      const float own_hh = orec[oc].yh.w;
      for (int64_t ic = 0; ic < A.nin; ++ic) {
        const SrcRec R = irec[ic];
        const float px = to_local(R.yh.x, R.q.w, oh[0], ol[0]);
        const float py = to_local(R.yh.y, R.n.w, oh[1], ol[1]);
        const float pz = to_local(R.yh.z, R.p.w, oh[2], ol[2]);
        const float dx = SRC ? px - ox : ox - px, dy = SRC ? py - oy : oy - py,
                    dz = SRC ? pz - oz : oz - pz;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float hh = SRC ? own_hh : R.yh.w;
        if (r2 < hh) adj_near_pair<SRC>(A, oc, (int32_t)ic, ad);
      }
    }
    double *out = A.partial + (size_t)oc * NA;  // the first input split
#pragma unroll
    for (int a = 0; a < NA; ++a) out[a] += ad[a];
  }
}

// ---------------------------------------------------------------- FP64 pass
template <bool SRC>
__global__ void __launch_bounds__(kAdjThreads) k_adj_fp64(AdjParams A) {
  constexpr int NA = NAcc<SRC>::value;
  __shared__ double sP[kAdjThreads][3];
  __shared__ double sA[kAdjThreads][3];
  __shared__ double sN[kAdjThreads][3];
  __shared__ double sPs[kAdjThreads][3];
  const SrcRec64 *orec = reinterpret_cast<const SrcRec64 *>(A.out_rec);
  const SrcRec64 *irec = reinterpret_cast<const SrcRec64 *>(A.in_rec);
  const int tid = threadIdx.x;
  const int64_t o_sorted = (int64_t)blockIdx.x * kAdjThreads + tid;
  const bool valid = o_sorted < A.nout;
  const int64_t oc = valid ? A.operm[o_sorted] : 0;
  SrcRec64 Ro;
  if (valid) Ro = orec[oc];
  double acc[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) acc[a] = 0.0;
  const int64_t i0 = A.nin * blockIdx.y / A.nsplit, i1 = A.nin * (blockIdx.y + 1) / A.nsplit;
  for (int64_t tb = i0; tb < i1; tb += kAdjThreads) {
    const int64_t k = tb + tid;
    if (k < i1) {
      const SrcRec64 R = irec[A.iperm[k]];
      for (int c = 0; c < 3; ++c) {
        sP[tid][c] = R.y[c];
        sA[tid][c] = R.q[c];
        sN[tid][c] = R.n[c];
        sPs[tid][c] = R.p[c];
      }
    }
    __syncthreads();
    const int m = (int)min((int64_t)kAdjThreads, i1 - tb);
    if (valid) {
      for (int kk = 0; kk < m; ++kk) {
        const double dx = SRC ? sP[kk][0] - Ro.y[0] : Ro.y[0] - sP[kk][0];
        const double dy = SRC ? sP[kk][1] - Ro.y[1] : Ro.y[1] - sP[kk][1];
        const double dz = SRC ? sP[kk][2] - Ro.y[2] : Ro.y[2] - sP[kk][2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ri = r2 > 0.0 ? rsqrt(r2) : 0.0;
        double g[3], q[3], pp[3], nn[3];
        for (int c = 0; c < 3; ++c) {
          if (SRC) {
            g[c] = sA[kk][c];
            q[c] = Ro.q[c];
            pp[c] = Ro.p[c];
            nn[c] = Ro.n[c];
          } else {
            g[c] = Ro.q[c];
            q[c] = sA[kk][c];
            pp[c] = sPs[kk][c];
            nn[c] = sN[kk][c];
          }
        }
        adj_pair<double, SRC>(dx, dy, dz, ri, g, q, pp, nn, A.has_sl, A.has_dl, acc);
      }
    }
    __syncthreads();
  }
  if (valid) {
    double *out = A.partial + ((size_t)blockIdx.y * (size_t)A.nout + (size_t)oc) * NA;
#pragma unroll
    for (int a = 0; a < NA; ++a) out[a] = acc[a];
  }
}

// Sums the input splits in order and writes the caller's gradients.
__global__ void k_adj_finish_src(int64_t ns, int32_t nsplit, const double *__restrict__ part,
                                 const double *__restrict__ w, double csl, double cdl,
                                 double *grad_f, double *grad_phi, double *grad_n, double *grad_y) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns;
       j += (int64_t)gridDim.x * blockDim.x) {
    double a[12] = {0};
    for (int s = 0; s < nsplit; ++s)
      for (int k = 0; k < 12; ++k) a[k] += part[((size_t)s * ns + j) * 12 + k];
    const double wj = w[j];
    for (int k = 0; k < 3; ++k) {
      if (grad_f) grad_f[3 * j + k] = wj * csl * a[k];
      if (grad_phi) grad_phi[3 * j + k] = wj * cdl * a[3 + k];
      if (grad_n) grad_n[3 * j + k] = a[6 + k];
      if (grad_y) grad_y[3 * j + k] = a[9 + k];
    }
  }
}

__global__ void k_adj_finish_trg(int64_t nt, int32_t nsplit, const double *__restrict__ part,
                                 double *grad_x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
       i += (int64_t)gridDim.x * blockDim.x) {
    double a[3] = {0, 0, 0};
    for (int s = 0; s < nsplit; ++s)
      for (int k = 0; k < 3; ++k) a[k] += part[((size_t)s * nt + i) * 3 + k];
    for (int k = 0; k < 3; ++k) grad_x[3 * i + k] = a[k];
  }
}

cudaError_t launch_adjoint(bool mixed, bool src_major, const AdjParams &A, cudaStream_t st) {
  dim3 grid((unsigned)((A.nout + kAdjThreads - 1) / kAdjThreads), (unsigned)A.nsplit);
  if (mixed) {
    cudaMemsetAsync(A.near_cnt, 0, sizeof(int32_t) * (size_t)A.nout, st);
    int64_t gn = (A.nout + kAdjThreads - 1) / kAdjThreads;
    if (gn > 65535) gn = 65535;
    if (src_major) {
      k_adj_mixed<true><<<grid, kAdjThreads, 0, st>>>(A);
      k_adj_near<true><<<(int)gn, kAdjThreads, 0, st>>>(A);
    } else {
      k_adj_mixed<false><<<grid, kAdjThreads, 0, st>>>(A);
      k_adj_near<false><<<(int)gn, kAdjThreads, 0, st>>>(A);
    }
    count_launches(1);
  } else {
    if (src_major)
      k_adj_fp64<true><<<grid, kAdjThreads, 0, st>>>(A);
    else
      k_adj_fp64<false><<<grid, kAdjThreads, 0, st>>>(A);
  }
  count_launches(1);
  return cudaGetLastError();
}

void launch_adj_finish(bool src_major, int64_t n, int32_t nsplit, const double *part,
                       const double *w, double csl, double cdl, double *grad_f, double *grad_phi,
                       double *grad_n, double *grad_y, double *grad_x, cudaStream_t st) {
  const int threads = 256;
  int64_t g = (n + threads - 1) / threads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  if (src_major)
    k_adj_finish_src<<<(int)g, threads, 0, st>>>(n, nsplit, part, w, csl, cdl, grad_f, grad_phi,
                                                 grad_n, grad_y);
  else
    k_adj_finish_trg<<<(int)g, threads, 0, st>>>(n, nsplit, part, grad_x);
  count_launches(1);
}

}  // namespace stk
