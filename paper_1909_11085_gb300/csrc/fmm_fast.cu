// fmm_fast.cu -- the mixed-precision far field of the kernel-independent FMM
// (Sec. 3.1, "Far evaluation") as CTA-blocked kernels, for surfaces of order
// p <= 8.  The arithmetic is that of the per-output mixed passes in
// fmm_passes.cuh (FP32 kernel evaluations on local coordinates, one FP64
// difference of box centres per pair of boxes, double-FP32
// check-to-equivalent products, FP32 spectra); what changes is how the work
// is laid out on the GPU:
//   * kernel evaluations (S2M, M2M, the X and W lists, L2L, L2T, dense M2L):
//     one CTA per target box or leaf, one check point or target point per
//     thread, the source points or equivalent densities staged in shared
//     memory and read as broadcasts;
//   * check-to-equivalent products: a tile of 8 boxes per CTA, their check
//     velocities in shared memory, one operator row per thread, so that each
//     operator entry read from L2 serves 8 boxes;
//   * the lattice DFTs (UFFT, IFFT): dense products with tabulated twiddle
//     matrices, a tile of 8 boxes per CTA;
//   * the spectral M2L products: one thread per parent box and frequency, the
//     CTA's 128 parents sharing one frequency whose kernel spectra (all 343
//     offsets) sit in shared memory; a parent's 26 neighbours are walked by
//     child octant, so that every lane of a warp runs the same (neighbour,
//     source octant, target octant) sequence, reads the same kernel spectrum
//     (a broadcast) and only the loads of missing children are predicated off.
// Every box, leaf and point index read from a tree array is checked on the
// device before use; an index out of range is skipped and recorded as error
// 6 in the workspace's error word (stokes_device_status).
#include <algorithm>
#include <cmath>

#include "fmm_fast.cuh"
#include "prep.cuh"
#include "tc_gemm.cuh"

namespace stk {
namespace fmm {

namespace {

constexpr int kFastTile = 8;       // boxes per CTA of the products
constexpr int kErrIndex = 6;

__device__ __forceinline__ void bad_index(const Pass &P) {
  if (P.err) atomicCAS(P.err, 0, kErrIndex);
}
__device__ __forceinline__ bool in_range(const Pass &P, int64_t v, int64_t hi) {
  if (v >= 0 && v < hi) return true;
  bad_index(P);
  return false;
}

// Centre of box b of depth d (the box size is root_size 2^-d, exact).
__device__ __forceinline__ void centre(const Tree &t, int32_t b, int d, double c[3]) {
  const double s = ldexp(t.root_size, -d);
#pragma unroll
  for (int q = 0; q < 3; ++q) c[q] = t.root_lo[q] + ((double)t.anchor[3 * b + q] + 0.5) * s;
}
// centre(b) - centre(a), rounded to FP32 (one FP64 difference per pair of boxes)
__device__ __forceinline__ void offset_f(const Tree &t, int32_t b, int db, int32_t a, int da,
                                         float off[3]) {
  double cb[3], ca[3];
  centre(t, b, db, cb);
  centre(t, a, da, ca);
#pragma unroll
  for (int q = 0; q < 3; ++q) off[q] = (float)(cb[q] - ca[q]);
}
__device__ __forceinline__ float half_width(const Tree &t, int d) {
  return (float)ldexp(t.root_size, -d - 1);
}

// x rounded to TF32 (10 explicit mantissa bits, round to nearest, ties away),
// kept in an FP32 register.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// A source box of a batch of equivalent densities: its density [ns][nc], the
// radius of its surface and its centre's offset from the target box's centre.
struct EqSrc {
  const float *dens;
  int32_t nc;
  float rad;
  float off[3];  // centre(target box) - centre(source box), FP32
};

// ---------------------------------------------------------------- pair math
// Packed FP32 pairs: two staged sources per instruction (FFMA2 and friends);
// per half the operations are those of a scalar evaluation.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 p_hi(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 p_dup(float v) { return make_float2(v, v); }
// 1/sqrt per half (rsqrt.approx, relative error below 2^-22), 0 where r2 is 0
// (a coincident pair contributes nothing).
__device__ __forceinline__ float2 p_rsqrt(float2 r2) {
  float a, b;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(r2.x));
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(b) : "f"(r2.y));
  return make_float2(r2.x > 0.f ? a : 0.f, r2.y > 0.f ? b : 0.f);
}
constexpr float kFarAway = 1e18f;  // position of the missing half of a pair (zero strength)

// Source points staged two by two, the pair's halves interleaved, positions
// negated, in kSrcFields planes of cap float4 (lanes reading consecutive
// pairs touch consecutive words): plane 0 (-y.x, -y.y), 1 (-y.z, q.x),
// 2 (q.y, q.z), 3 (p.x, p.y), 4 (p.z, n.x), 5 (n.y, n.z), each entry a
// (first, second) pair.
constexpr int kSrcFields = 6;
// Stages points [i0, i0 + n) (n <= 2 blockDim, (n + 1) / 2 <= cap) as pairs.
__device__ __forceinline__ void stage_point_pairs(const Pass &P, float4 *S, int cap, int64_t i0,
                                                  int n) {
  const int t = threadIdx.x;
  if (2 * t >= n) return;
  float v[2][12];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t i = i0 + 2 * t + h;
    const bool ok = 2 * t + h < n;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      v[h][q] = ok ? -P.ploc[3 * i + q] : -kFarAway;
      v[h][3 + q] = ok && P.qf ? P.qf[3 * i + q] : 0.f;
      v[h][6 + q] = ok && P.pf ? P.pf[3 * i + q] : 0.f;
      v[h][9 + q] = ok && P.nf ? P.nf[3 * i + q] : 0.f;
    }
  }
#pragma unroll
  for (int f = 0; f < kSrcFields; ++f)
    S[(size_t)f * cap + t] = make_float4(v[0][2 * f], v[1][2 * f], v[0][2 * f + 1], v[1][2 * f + 1]);
}
// Adds the single and double layer of the staged pairs j0, j0 + js, ... < np
// at two targets (x: each coordinate duplicated into both halves; u: per-half
// sums).  SL: (q + d (d.q)/r^2)/r, DL: d (d.psi)(d.n)/r^5.
template <bool SL, bool DL>
__device__ __forceinline__ void eval_src_pairs(const float4 *S, int cap, int j0, int np, int js,
                                               const float2 (&x)[2][3], float2 (&u)[2][3]) {
  for (int j = j0; j < np; j += js) {
    const float4 a = S[j], b = S[cap + j];
    const float2 nyx = p_lo(a), nyy = p_hi(a), nyz = p_lo(b);
    float2 qx, qy, qz, px, py, pz, nx, ny, nz;
    if (SL) {
      const float4 c = S[2 * cap + j];
      qx = p_hi(b);
      qy = p_lo(c);
      qz = p_hi(c);
    }
    if (DL) {
      const float4 d = S[3 * cap + j], e = S[4 * cap + j], f = S[5 * cap + j];
      px = p_lo(d);
      py = p_hi(d);
      pz = p_lo(e);
      nx = p_hi(e);
      ny = p_lo(f);
      nz = p_hi(f);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float2 dx = p_add(x[t][0], nyx), dy = p_add(x[t][1], nyy), dz = p_add(x[t][2], nyz);
      const float2 r2 = p_fma(dx, dx, p_fma(dy, dy, p_mul(dz, dz)));
      const float2 ri = p_rsqrt(r2), ri2 = p_mul(ri, ri);
      if (SL && DL) {
        const float2 dq = p_fma(dx, qx, p_fma(dy, qy, p_mul(dz, qz)));
        const float2 dp = p_fma(dx, px, p_fma(dy, py, p_mul(dz, pz)));
        const float2 dn = p_fma(dx, nx, p_fma(dy, ny, p_mul(dz, nz)));
        const float2 c = p_mul(p_fma(p_mul(dp, dn), ri2, dq), ri2);
        u[t][0] = p_fma(p_fma(dx, c, qx), ri, u[t][0]);
        u[t][1] = p_fma(p_fma(dy, c, qy), ri, u[t][1]);
        u[t][2] = p_fma(p_fma(dz, c, qz), ri, u[t][2]);
      } else if (SL) {
        const float2 dq = p_fma(dx, qx, p_fma(dy, qy, p_mul(dz, qz)));
        const float2 c = p_mul(dq, ri2);
        u[t][0] = p_fma(p_fma(dx, c, qx), ri, u[t][0]);
        u[t][1] = p_fma(p_fma(dy, c, qy), ri, u[t][1]);
        u[t][2] = p_fma(p_fma(dz, c, qz), ri, u[t][2]);
      } else {
        const float2 dp = p_fma(dx, px, p_fma(dy, py, p_mul(dz, pz)));
        const float2 dn = p_fma(dx, nx, p_fma(dy, ny, p_mul(dz, nz)));
        const float2 c = p_mul(p_mul(dp, dn), p_mul(p_mul(ri2, ri2), ri));
        u[t][0] = p_fma(dx, c, u[t][0]);
        u[t][1] = p_fma(dy, c, u[t][1]);
        u[t][2] = p_fma(dz, c, u[t][2]);
      }
    }
  }
}
__device__ __forceinline__ void eval_src_pairs_any(const Pass &P, const float4 *S, int cap, int j0,
                                                   int np, int js, const float2 (&x)[2][3],
                                                   float2 (&u)[2][3]) {
  if (P.qf && P.pf) eval_src_pairs<true, true>(S, cap, j0, np, js, x, u);
  else if (P.qf) eval_src_pairs<true, false>(S, cap, j0, np, js, x, u);
  else eval_src_pairs<false, true>(S, cap, j0, np, js, x, u);
}

// Equivalent points staged two by two in kEqFields planes of cap float4:
// plane 0 (-y.x, -y.y), 1 (-y.z, e.x), 2 (e.y, e.z), 3 (e.w, unused), each
// entry a (first, second) pair; the positions already scaled by the radius
// and in the target box's frame.
constexpr int kEqFields = 4;
// Adds the field of the staged pairs j0, j0 + js, ... < np at T targets:
// Stokeslet (e + d (d.e)/r^2)/r into uf, point source d e.w/r^3 into uq.
template <bool FLUX, int T = 2>
__device__ __forceinline__ void eval_eq_pairs(const float4 *E, int cap, int j0, int np, int js,
                                              const float2 (&x)[T][3], float2 (&uf)[T][3],
                                              float2 (&uq)[T][3]) {
  for (int j = j0; j < np; j += js) {
    const float4 a = E[j], b = E[cap + j], c = E[2 * cap + j];
    const float2 nyx = p_lo(a), nyy = p_hi(a), nyz = p_lo(b);
    const float2 ex = p_hi(b), ey = p_lo(c), ez = p_hi(c);
    float2 ew;
    if (FLUX) ew = p_lo(E[3 * cap + j]);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const float2 dx = p_add(x[t][0], nyx), dy = p_add(x[t][1], nyy), dz = p_add(x[t][2], nyz);
      const float2 r2 = p_fma(dx, dx, p_fma(dy, dy, p_mul(dz, dz)));
      const float2 ri = p_rsqrt(r2), ri3 = p_mul(p_mul(ri, ri), ri);
      const float2 df = p_mul(p_fma(dx, ex, p_fma(dy, ey, p_mul(dz, ez))), ri3);
      uf[t][0] = p_fma(ex, ri, p_fma(dx, df, uf[t][0]));
      uf[t][1] = p_fma(ey, ri, p_fma(dy, df, uf[t][1]));
      uf[t][2] = p_fma(ez, ri, p_fma(dz, df, uf[t][2]));
      if (FLUX) {
        const float2 sv = p_mul(ew, ri3);
        uq[t][0] = p_fma(dx, sv, uq[t][0]);
        uq[t][1] = p_fma(dy, sv, uq[t][1]);
        uq[t][2] = p_fma(dz, sv, uq[t][2]);
      }
    }
  }
}

// Equivalent points staged per batch (shared memory budget of the batches).
constexpr int kEqBatchPoints = 512;
constexpr int kEqBatchMax = 64;  // source boxes per batch
__host__ __device__ inline int eq_batch_boxes(int ns) {
  const int b = kEqBatchPoints / ns;
  return b < 1 ? 1 : (b > kEqBatchMax ? kEqBatchMax : b);
}
// A batch entry that contributes nothing (an index that failed its check).
__device__ __forceinline__ EqSrc eq_none(const Pass &P) {
  EqSrc q;
  q.dens = P.surf32;
  q.nc = 0;
  q.rad = 0.f;
  q.off[0] = q.off[1] = q.off[2] = 0.f;
  return q;
}

// Stages the boxes src[0, nb) into E as (nb ns + 1) / 2 <= cap pairs, each
// surface point in the target box's frame: rad s_j - off (negated).
__device__ __forceinline__ void stage_eq_pairs(const Pass &P, float4 *E, int cap, const EqSrc *src,
                                               int nb) {
  const int total = nb * P.ns, npair = (total + 1) / 2;
  for (int e = threadIdx.x; e < npair; e += blockDim.x) {
    float v[2][7];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * e + h;
      if (i < total) {
        const int k = i / P.ns, j = i % P.ns;
        const EqSrc &S = src[k];
        const float *sp = P.surf32 + 3 * j;
        const float *d = S.dens + (size_t)S.nc * j;
#pragma unroll
        for (int q = 0; q < 3; ++q) v[h][q] = S.off[q] - S.rad * sp[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[h][3 + q] = q < S.nc ? d[q] : 0.f;
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) v[h][q] = -kFarAway;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[h][3 + q] = 0.f;
      }
    }
    E[e] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
    E[cap + e] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
    E[2 * cap + e] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
    E[3 * cap + e] = make_float4(v[0][6], v[1][6], 0.f, 0.f);
  }
}

// Targets of the pair-packed evaluations: two per thread, the coordinates
// duplicated into both halves of a pair.
__device__ __forceinline__ void dup_targets(const float (&x)[2][3], float2 (&x2)[2][3]) {
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) x2[t][q] = p_dup(x[t][q]);
}
// Sums u over the S adjacent lanes of a target pair (S a power of two <= 32),
// in a fixed order.
__device__ __forceinline__ void lane_sum2(float (&u)[2][3], int S) {
  for (int o = 1; o < S; o <<= 1)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) u[t][q] += __shfl_xor_sync(kFull, u[t][q], o);
}
// Sum of the two halves of each of the 6 packed sums.
__device__ __forceinline__ void fold_halves(const float2 (&u2)[2][3], float (&u)[2][3]) {
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) u[t][q] = u2[t][q].x + u2[t][q].y;
}

// ------------------------------------------------------------------ set-up
// K chunks of the inverse-DFT product: 2 nfreq reals (re, im per frequency).
__host__ __device__ inline int ifft_chunks(int p) {
  return (2 * freq_count(p) + tc::kChunk - 1) / tc::kChunk;
}
__host__ __device__ inline int ifft_tiles(int ns) { return (ns + tc::kCols - 1) / tc::kCols; }

// child8, bflag and the lattice DFT tables (the inverse one as the B table of
// the tensor-core product, zeroed before); e runs over max(nbox, ns nfreq).
__global__ void k_fast_tables(Pass P, int64_t n) {
  const int nf = freq_count(P.p), G = 2 * P.p, nz = P.p + 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    if (e < P.t.nbox) {
      const int32_t b = (int32_t)e;
      int32_t flag = 0;
      if (b > 0) {
        const int32_t pb = P.t.parent[b];
        if (in_range(P, pb, P.t.nbox)) {
          const int oct = ((P.t.anchor[3 * b] & 1) << 2) | ((P.t.anchor[3 * b + 1] & 1) << 1) |
                          (P.t.anchor[3 * b + 2] & 1);
          P.child8[8 * (size_t)pb + oct] = b;
          flag = P.t.child_ptr[pb] == b ? 1 : 0;
        }
      }
      P.bflag[b] = flag;
    }
    if (P.ftab && e < (int64_t)P.ns * nf) {
      // forward: ftab[j][w]; inverse: the B table of the inverse-DFT product
      // (the same angle), B[j][2 w + ri] = the weighted (cos, -sin) / G^3
      const int j = (int)(e / nf), w = (int)(e % nf);
      const int kx = w / (G * nz), ky = (w / nz) % G, kz = w % nz;
      const int t = (P.sidx[3 * j] * kx + P.sidx[3 * j + 1] * ky + P.sidx[3 * j + 2] * kz) % G;
      double sn, c;
      sincospi((double)t / (double)P.p, &sn, &c);  // angle 2 pi t / G, G = 2p
      P.ftab[2 * e] = (float)c;
      P.ftab[2 * e + 1] = (float)(-sn);
      const double wt = (kz == 0 || kz == P.p) ? 1.0 : 2.0;
      const double inv = wt / ((double)G * G * G);
      const int nkc = ifft_chunks(P.p);
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        const float v = (float)(ri == 0 ? inv * c : -inv * sn);
        const int kk = 2 * w + ri;
        float *tl = P.fitab + ((size_t)(j / tc::kCols) * nkc + kk / tc::kChunk) * 2 * tc::kCols *
                                  tc::kChunk;
        const uint32_t o = tc::b_table_offset(j % tc::kCols, kk % tc::kChunk);
        const float h = tf32_rna(v);
        tl[o] = h;
        tl[tc::kCols * tc::kChunk + o] = tf32_rna(v - h);
      }
    }
  }
}

__global__ void k_fast_plist(Pass P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < P.t.nbox; b += stride)
    if (P.bflag[b]) P.plist[P.bpos[b]] = P.t.parent[b];  // checked by k_fast_tables
}

// The operators' (hi, lo) FP32 split, stored column by column (OPSPLIT).
__global__ void k_fast_opsplit(Pass P, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
    OPSPLIT()(P, e);
}

// Kernel spectra at FP32, frequency-major: spec32[w][offset][3 nc][2].
__global__ void k_fast_spec(Pass P, int64_t n) {
  const int nf = freq_count(P.p), m = 3 * P.nc * 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t oi = e / ((int64_t)nf * m), r = e % ((int64_t)nf * m);
    const int64_t w = r / m, k = r % m;
    P.spec32[(w * 343 + oi) * m + k] = (float)P.spec[e];
  }
}

// Points relative to their leaf's centre and pre-scaled FP32 densities; one
// warp per leaf (leaves hold about 64 points), kPackLeaves leaves per CTA.
constexpr int kPackLeaves = 4;
__global__ void __launch_bounds__(kPackLeaves * 32) k_fast_pack(Pass P) {
  const int32_t l = blockIdx.x * kPackLeaves + (int)(threadIdx.x >> 5);
  if (l >= P.t.nleaf) return;
  const int lane = threadIdx.x & 31;
  const int32_t b = P.t.leaf_box[l];
  if (!in_range(P, b, P.t.nbox)) return;
  const int d = P.t.depth[b];
  double c[3];
  centre(P.t, b, d, c);
  const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
  if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1)) return;
  // (the FP32 roundings on the integer pipe: f64_to_f32_rn)
  for (int64_t i = i0 + lane; i < i1; i += 32) {
    const double wi = P.w[i];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      P.ploc[3 * i + q] = f64_to_f32_rn(P.pts[3 * i + q] - c[q]);
      if (P.qf) P.qf[3 * i + q] = f64_to_f32_rn(P.csl * (wi * P.f[3 * i + q]));
      if (P.pf) {
        P.pf[3 * i + q] = f64_to_f32_rn(P.cdl * (wi * P.phi[3 * i + q]));
        P.nf[3 * i + q] = f64_to_f32_rn(P.nrm[3 * i + q]);
      }
    }
  }
}

// ---------------------------------------------------------------- upward
// S2M: one CTA per leaf; threads 2c and 2c + 1 take check points 2c and
// 2c + 1 on the 2.95 r surface, each every other staged source pair.
__global__ void k_fast_s2m(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4 *S = reinterpret_cast<float4 *>(smem);  // kSrcFields planes of blockDim pairs
  const int cap = blockDim.x;
  const int32_t l = blockIdx.x;
  const int32_t b = P.t.leaf_box[l];
  if (!in_range(P, b, P.t.nbox)) return;
  const int d = P.t.depth[b];
  if (d < kFirstDepth) return;
  const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
  if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1) || i1 < i0) return;
  const int k0 = threadIdx.x & ~1, sl = threadIdx.x & 1;
  const bool act = k0 + 1 < P.ns;  // ns is even
  const float rad = (float)(kOuter * (double)half_width(P.t, d));
  float x[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if (act)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) x[t][q] = rad * P.surf32[3 * (k0 + t) + q];
  float2 x2[2][3], u2[2][3];
  dup_targets(x, x2);
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) u2[t][q] = make_float2(0.f, 0.f);
  const int chunk = 2 * (int)blockDim.x;
  for (int64_t c0 = i0; c0 < i1; c0 += chunk) {
    const int n = (int)min((int64_t)chunk, i1 - c0);
    __syncthreads();
    stage_point_pairs(P, S, cap, c0, n);
    __syncthreads();
    if (act) eval_src_pairs_any(P, S, cap, sl, (n + 1) / 2, 2, x2, u2);
  }
  float u[2][3];
  fold_halves(u2, u);
  lane_sum2(u, 2);
  if (act && sl == 0)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) P.chk32[(size_t)b * 3 * P.ns + 3 * (k0 + t) + q] = u[t][q];
}

// M2M: one CTA per box of one depth with children; threads 2c, 2c + 1 take
// check points 2c, 2c + 1 (every other staged pair each); the children's
// upward densities staged in batches, in this box's frame.
__global__ void k_fast_m2m(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[8];
  float4 *E = reinterpret_cast<float4 *>(smem);  // kEqFields planes of cap pairs
  const int32_t b = P.box0 + blockIdx.x;
  const int32_t c0 = P.t.child_ptr[b], c1 = P.t.child_ptr[b + 1];
  if (c0 >= c1) return;
  if (c1 - c0 > 8) {
    bad_index(P);
    return;
  }
  const int nch = c1 - c0, neq = min(8, eq_batch_boxes(P.ns));
  const int cap = (neq * P.ns + 1) / 2;
  const int k0 = threadIdx.x & ~1, sl = threadIdx.x & 1;
  const bool act = k0 + 1 < P.ns;
  const float r = half_width(P.t, P.depth);
  const float rad = (float)(kOuter * (double)r), rc = (float)(kInner * (double)r / 2);
  if ((int)threadIdx.x < nch) {
    const int32_t ch = c0 + threadIdx.x;
    EqSrc e;
    if (in_range(P, ch, P.t.nbox)) {
      e.dens = P.up32 + (size_t)ch * P.nc * P.ns;
      e.nc = P.nc;
      e.rad = rc;
      offset_f(P.t, b, P.depth, ch, P.depth + 1, e.off);
    } else {
      e = eq_none(P);
    }
    src[threadIdx.x] = e;
  }
  float x[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if (act)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) x[t][q] = rad * P.surf32[3 * (k0 + t) + q];
  float2 x2[2][3], uf[2][3], uq[2][3];
  dup_targets(x, x2);
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) uf[t][q] = uq[t][q] = make_float2(0.f, 0.f);
  for (int e0 = 0; e0 < nch; e0 += neq) {
    const int nb = min(neq, nch - e0);
    __syncthreads();
    stage_eq_pairs(P, E, cap, src + e0, nb);
    __syncthreads();
    if (act) {
      if (P.nc == 4) eval_eq_pairs<true>(E, cap, sl, (nb * P.ns + 1) / 2, 2, x2, uf, uq);
      else eval_eq_pairs<false>(E, cap, sl, (nb * P.ns + 1) / 2, 2, x2, uf, uq);
    }
  }
  float a1[2][3], a2[2][3], u[2][3];
  fold_halves(uf, a1);
  fold_halves(uq, a2);
  const float csl = (float)P.csl, csrc = (float)P.csrc;
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) u[t][q] = csl * a1[t][q] + csrc * a2[t][q];
  lane_sum2(u, 2);
  if (act && sl == 0)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) P.chk32[(size_t)b * 3 * P.ns + 3 * (k0 + t) + q] = u[t][q];
}

// Check-to-equivalent products of a tile of NB boxes of one depth:
// out[b][i] = (hi + lo)[i] . chk32[b] in double-FP32 arithmetic (the exact
// FMA product and two-sum accumulation of apply_row_df), operator stored
// column by column, read four columns ahead of their use; the boxes in pairs
// on packed FP32 instructions (per half the same operations and roundings).
template <bool UP, int NB>
__global__ void __launch_bounds__(256) k_fast_c2e(Pass P) {
  static_assert(NB % 2 == 0, "boxes in pairs");
  extern __shared__ __align__(16) unsigned char smem[];
  float *X = reinterpret_cast<float *>(smem);  // [cols][NB]: a column's boxes adjacent
  const int cols = 3 * P.ns;
  const int rows = UP ? P.nc * P.ns : 3 * P.ns;
  const int32_t bt = P.box0 + blockIdx.x * NB;
  const int nbt = min(NB, P.box1 - bt);
  for (int e = threadIdx.x; e < NB * cols; e += blockDim.x) {
    const int bb = e / cols, j = e % cols;
    X[j * NB + bb] = bb < nbt ? P.chk32[(size_t)(bt + bb) * cols + j] : 0.f;
  }
  __syncthreads();
  const size_t off = UP ? (size_t)(P.depth - kFirstDepth) * rows * cols
                        : (size_t)P.n_uc2e + (size_t)(P.depth - kFirstDepth) * rows * cols;
  const float *hi = P.ops_hi + off, *lo = P.ops_lo + off;
  float *out = UP ? P.up32 : P.dn32;
  const float2 m1 = make_float2(-1.f, -1.f);
  // a - b as one packed FMA: b (-1) + a, exact product, one rounding
  auto sub2 = [&](float2 a2, float2 b2) { return p_fma(b2, m1, a2); };
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    // packed over box pairs: per half the operations of the scalar double-FP32 form
    float2 sh[NB / 2], sl[NB / 2];
#pragma unroll
    for (int h = 0; h < NB / 2; ++h) sh[h] = sl[h] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < cols; j0 += 4) {
      float ah[4], al[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool ok = j0 + q < cols;
        ah[q] = ok ? hi[(size_t)(j0 + q) * rows + i] : 0.f;
        al[q] = ok ? lo[(size_t)(j0 + q) * rows + i] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (j0 + q >= cols) break;
        const float2 ah2 = p_dup(ah[q]), al2 = p_dup(al[q]);
        const float2 *x2p = reinterpret_cast<const float2 *>(X + (j0 + q) * NB);
#pragma unroll
        for (int h = 0; h < NB / 2; ++h) {
          const float2 x = x2p[h];
          const float2 p = p_mul(ah2, x);
          const float2 err = p_fma(al2, x, p_fma(ah2, x, p_mul(p, m1)));
          const float2 t = p_add(sh[h], p), bv = sub2(t, sh[h]);
          sl[h] = p_add(sl[h], p_add(p_add(sub2(sh[h], sub2(t, bv)), sub2(p, bv)), err));
          sh[h] = t;
        }
      }
    }
#pragma unroll
    for (int h = 0; h < NB / 2; ++h) {
      if (2 * h < nbt) out[(size_t)(bt + 2 * h) * rows + i] = __fadd_rn(sh[h].x, sl[h].x);
      if (2 * h + 1 < nbt) out[(size_t)(bt + 2 * h + 1) * rows + i] = __fadd_rn(sh[h].y, sl[h].y);
    }
  }
}

// ------------------------------------------------------------- downward
// UFFT: spectra of the upward densities of the children of one parent (the
// CTA's plist position k at this depth), one octant each,
// uhat[w][8 k + o][c] = sum_j up[child o][j][c] (cos - i sin)(2 pi (s_j . k_w mod G) / G),
// zero for a missing child; thread = frequency.
constexpr int kUfftRow = kFastTile * 8 + 4;  // staged output row, padded for float4 stores
static_assert(kFastTile == 8, "one octant per box of the tile");
inline size_t ufft_smem(int ns, int nc) {
  return sizeof(float) * std::max<size_t>((size_t)kFastTile * ns * nc, (size_t)128 * kUfftRow);
}
template <int NC>
__global__ void __launch_bounds__(128) k_fast_ufft(Pass P, int32_t first_child0,
                                                   int32_t first_child1) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *U = reinterpret_cast<float *>(smem);  // [8 octants][ns][NC]
  const int nf = freq_count(P.p);
  const int32_t pos0 = P.bpos[first_child0], pos1 = P.bpos[first_child1];
  const int32_t kp = (int32_t)blockIdx.x;
  if (pos0 + kp >= pos1) return;  // the whole CTA
  if ((int64_t)8 * kp + 8 > P.uslots) {
    if (threadIdx.x == 0) bad_index(P);
    return;
  }
  const int32_t par = P.plist[pos0 + kp];
  const bool okp = in_range(P, par, P.t.nbox);
  const int per = P.ns * NC;
  for (int e = threadIdx.x; e < kFastTile * per; e += blockDim.x) {
    const int o = e / per, r = e % per;
    const int32_t b = okp ? P.child8[8 * (size_t)par + o] : -1;  // a box of this depth or -1
    U[e] = b >= 0 ? P.up32[(size_t)b * per + r] : 0.f;
  }
  __syncthreads();
  const int w = blockIdx.y * blockDim.x + threadIdx.x;
  const bool active = w < nf;  // every thread stays for the staged store
  float re[kFastTile][NC], im[kFastTile][NC];
#pragma unroll
  for (int bb = 0; bb < kFastTile; ++bb)
#pragma unroll
    for (int c = 0; c < NC; ++c) re[bb][c] = im[bb][c] = 0.f;
  const float r = half_width(P.t, P.depth);
  const float sf = 1.0f / r, sq = 1.0f / (r * r);
  const float2 *F = reinterpret_cast<const float2 *>(P.ftab);
  for (int j0 = 0; j0 < P.ns; j0 += 4) {
    float2 fq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      fq[q] = active && j0 + q < P.ns ? F[(size_t)(j0 + q) * nf + w] : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q;
      if (j >= P.ns) break;
#pragma unroll
      for (int bb = 0; bb < kFastTile; ++bb)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float v = U[(bb * P.ns + j) * NC + c];
          re[bb][c] = fmaf(v, fq[q].x, re[bb][c]);
          im[bb][c] = fmaf(v, fq[q].y, im[bb][c]);
        }
    }
  }
  // the tensor-core products read the spectra as TF32 hi + lo parts, four
  // components per child and frequency (the fourth zero without flux); at one
  // frequency a parent's 8 children are 256 contiguous bytes, the unit its
  // neighbours gather.  The [w][8][8] block is staged in shared memory and
  // written out as one contiguous run per frequency
  constexpr int kRow = kUfftRow;
  float *S = U;                            // reused after every thread is done with U
  const int wl = threadIdx.x;
  const int w0 = blockIdx.y * blockDim.x;
  const int nw = min((int)blockDim.x, nf - w0);
  constexpr int per_w = kFastTile * 2;  // float4 per frequency
  for (int half = 0; half < 2; ++half) {
    __syncthreads();
    if (active) {
#pragma unroll
      for (int bb = 0; bb < kFastTile; ++bb)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float v[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            // component c = 2q + k/2, real part for even k; scaled to the depth:
            // the kernel spectra are those of half-width 1, the Stokeslet
            // homogeneous of degree -1, the source of degree -2
            const int c = 2 * q + (k >> 1);
            const float x = c < NC ? (c < 3 ? sf : sq) * ((k & 1) ? im[bb][c < NC ? c : 0]
                                                                  : re[bb][c < NC ? c : 0])
                                   : 0.f;
            const float h = tf32_rna(x);
            v[k] = half ? tf32_rna(x - h) : h;
          }
          *reinterpret_cast<float4 *>(&S[wl * kRow + bb * 8 + 4 * q]) =
              make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    __syncthreads();
    float *dst = half ? P.uhl : P.uhh;
    for (int e = threadIdx.x; e < nw * per_w; e += blockDim.x) {
      const int ww = e / per_w, q = e % per_w;
      const float4 v = *reinterpret_cast<const float4 *>(&S[ww * kRow + 4 * q]);
      *reinterpret_cast<float4 *>(dst + ((size_t)(w0 + ww) * P.uslots + 8 * (size_t)kp) * 8 +
                                  4 * q) = v;
    }
  }
}

// The plist position of the neighbour of every parent (in plist order) in
// each of its 26 directions, -1 where there is no neighbour or it has no
// children: vpar[direction][plist position] (direction-major, so that
// consecutive parents are adjacent).  The children of the neighbour at that
// position are the sources of the direction.
__global__ void k_fast_vpar(Pass P) {
  const int32_t total = P.bpos[P.t.nbox];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)total * 26;
       e += stride) {
    const int32_t i = (int32_t)(e / 26);
    const int dd = (int)(e % 26);
    const int dir = dd < 13 ? dd : dd + 1;  // direction 13 is the parent itself
    const int32_t par = P.plist[i];
    int32_t q = -1;
    if (in_range(P, par, P.t.nbox)) {
      const int32_t Q = P.t.colleague[27 * (size_t)par + dir];
      if (Q >= 0 && in_range(P, Q, P.t.nbox)) {
        const int32_t c0 = P.t.child_ptr[Q], c1 = P.t.child_ptr[Q + 1];
        if (c1 > c0) {
          if (c0 < 0 || c0 >= P.t.nbox)
            bad_index(P);
          else
            q = P.bpos[c0];
        }
      }
    }
    P.vpar[(size_t)dd * P.t.nbox + i] = q;
  }
}

__device__ __forceinline__ void cp_async_zfill(void *dst, const void *src, bool valid, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int sz = valid ? bytes : 0;
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(sz)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sz)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ----------------------------------------------------------------------
// The spectral products on the tensor cores (tcgen05, kind::tf32).  For one
// frequency w the products of a parent P are one dense complex contraction:
// the 24 check-spectrum values of its 8 children (3 components each) are the
// 832 source-spectrum values of the 208 children of its 26 neighbours
// (4 components each) times an 832 x 24 matrix of kernel spectra, the same
// for every parent (zero where a pair touches).  Written with real numbers
// (re, im interleaved along both dimensions: [re im] x [[Kr Ki] [-Ki Kr]]) it
// is D[128 parents][48] = A[128][1664] B[48][1664]^T per tile of parents: A
// gathered from the source spectra, B built from the staged kernel spectra,
// both in FP32 split into TF32 hi + lo parts (hi = tf32(x), lo = tf32(x - hi))
// so that hi.hi + hi.lo + lo.hi carries FP32 accuracy (the lo.lo term is below
// it).  The K dimension runs in 52 chunks of 32 (one neighbour direction,
// four of its children's octants), 128 contiguous bytes per parent row in the
// parent-major spectra; a chunk is staged in shared memory in the MMA's
// K-major layout with the 128-byte swizzle (a row's 128 bytes in one line,
// its 16-byte pieces permuted by the row index within each 8-row group).
constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;
constexpr int kTcCols = 48;        // 8 targets x 3 components x (re, im)
constexpr int kTcK = 32;           // K per chunk (128 bytes of TF32)
constexpr int kTcChunks = 52;      // 26 neighbour directions x 2 octant halves
constexpr long long kTcSpinLimit = 4000000000LL;  // SM cycles, about 2 s
constexpr int kErrTimeout = 4;

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool tc_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
  if (tc_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!tc_try_wait(bar, parity))
    if (clock64() - t0 > kTcSpinLimit) return false;
  return true;
}
// Shared-memory matrix descriptor, K-major with the 128-byte swizzle: 8-row
// groups 1024 bytes apart (stride byte offset), the leading byte offset unused
// within one swizzle row, version 1, layout type 2 (128-byte swizzle).  The
// K-step inside a swizzle row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t tc_sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void tc_mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// Byte offset of element (row, k), k < 32, in a K-major tile with the 128-byte
// swizzle (tile base 1024-byte aligned): row r's 128 bytes at 128 r within its
// 8-row group, the 16-byte piece j stored at position j ^ (r mod 8).
__host__ __device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)(((row >> 3) << 10) + ((row & 7) << 7) + ((((k >> 2) ^ (row & 7)) & 7) << 4) +
                    ((k & 3) << 2));
}

// Per CTA: one frequency and kTcTiles tiles of 128 parents.  Warp roles:
//   warps 0-3 (producers): for each chunk, copy the TF32 hi/lo spectra of the
//     4 octants of their rows' neighbour by cp.async into the swizzled MMA
//     layout (8 lanes per row: one 128-byte line per row; zero-filled where the
//     neighbour has no children) and the chunk's B from the table k_fast_btab
//     built for the call; once a chunk's copies have landed, fence them for the
//     tensor core and arrive on the chunk's "full" barrier;
//   thread 128 (MMA): wait "full", issue 4 K-steps x 2 MMAs per tile, commit
//     to the chunk's "empty" barrier (producers refill a buffer only after it);
//   warps 4-7 (epilogue): after the final commit, read the accumulators from
//     tensor memory (one lane quarter each) and write the check spectra.
// A ring of kTcStages buffers lets the producers run ahead of the MMAs.
// Every wait is bounded; on expiry the role records STK_ETIMEOUT in the error
// word and stops, and the CTA still drains its copies and MMAs before it
// frees tensor memory.
constexpr int kTcTiles = 1;
constexpr int kTcStages = 2;
constexpr int kTcAhead = 1;  // chunks of copies a producer keeps in flight (< kTcStages)
constexpr int kTcMinBlocks = 2;  // 2 x 90 KB: one CTA's set-up and epilogue overlap the other's loop
// per tile 96 accumulator columns: [0, 48) hi.hi + lo.hi, [48, 96) hi.lo (summed at the end)
constexpr uint32_t kTcTmemCols = kTcTiles == 1 ? 128 : 256;  // accumulators 128 columns apart
constexpr int kTcProducers = 128;
struct TcShape {
  static constexpr int ATILE = kTcRows * kTcK * 4;      // bytes of one A tile (hi or lo)
  static constexpr int ASTAGE = kTcTiles * 2 * ATILE;   // hi, lo of every tile
  static constexpr int BTILE = kTcCols * kTcK * 4;      // 6 swizzle groups of 8 rows
  static constexpr int STAGE = ASTAGE + 2 * BTILE;      // a multiple of 1024
  static constexpr int NBAR = 2 * kTcStages + 1;        // full, empty, done
  static constexpr size_t SMEM = 1024 + (size_t)kTcStages * STAGE + 8 * NBAR + 16;
};
static_assert(TcShape::STAGE % 1024 == 0, "swizzle groups stay 1024-byte aligned");
static_assert(kTcChunks % 2 == 0, "two octant halves per direction");

// The B operand of every (frequency, chunk): for direction dd, octant half h
// (source octants 4h..4h+3) and target octant t, the 3 x 4 complex kernel
// spectra of their offsets (zero where they touch) as real 6 x 8 blocks
// [[Kr Ki] [-Ki Kr]], split into TF32 hi + lo, in the swizzled K-major layout
// the MMA reads: btab[w][2 dd + h][hi, lo][sw128_off(n, k)].
__global__ void k_fast_btab(Pass P, int64_t n) {
  const int m = 3 * P.nc * 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // e4 runs over the table four floats at a time in its own order (coalesced
  // float4 stores): float pos of row nn of tile wc holds k = ((pos / 4) ^ (nn
  // mod 8)) 4 + pos mod 4, so the four floats pos = 4 a .. 4 a + 3 hold
  // k = 4 b + j, b = a ^ (nn mod 8): one source octant sl and offset, the
  // components c = 2 b mod 4 (j = 0, 1) and c + 1 (j = 2, 3), re/im rk = j mod 2
  for (int64_t e4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * e4 < n; e4 += stride) {
    const int64_t e = 4 * e4;
    const int64_t wc = e / (kTcCols * kTcK);
    const int r = (int)(e % (kTcCols * kTcK));
    const int w = (int)(wc / kTcChunks), ch = (int)(wc % kTcChunks);
    const int nn = r / kTcK, pos = r % kTcK;
    const int bq = ((pos >> 2) ^ (nn & 7)) & 7;
    const int t = nn / 6, q = (nn >> 1) % 3, rn = nn & 1;
    const int sl = 4 * (ch & 1) + (bq >> 1);
    const int dd = ch >> 1, dir = dd < 13 ? dd : dd + 1;
    const int ox = 2 * (dir / 9 - 1) + (sl >> 2) - (t >> 2);
    const int oy = 2 * ((dir / 3) % 3 - 1) + ((sl >> 1) & 1) - ((t >> 1) & 1);
    const int oz = 2 * (dir % 3 - 1) + (sl & 1) - (t & 1);
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (!(ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1)) {
      const int oi = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
      const float *K = P.spec32 + ((size_t)w * 343 + oi) * m + (size_t)q * P.nc * 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = (2 * bq + h) & 3;
        if (c < P.nc) {
          const float2 kc = *reinterpret_cast<const float2 *>(K + 2 * c);
#pragma unroll
          for (int rk = 0; rk < 2; ++rk)
            v[2 * h + rk] = (rk == rn) ? kc.x : (rk == 0 ? kc.y : -kc.y);
        }
      }
    }
    float4 hi, lo;
    hi.x = tf32_rna(v[0]);
    hi.y = tf32_rna(v[1]);
    hi.z = tf32_rna(v[2]);
    hi.w = tf32_rna(v[3]);
    lo.x = tf32_rna(v[0] - hi.x);
    lo.y = tf32_rna(v[1] - hi.y);
    lo.z = tf32_rna(v[2] - hi.z);
    lo.w = tf32_rna(v[3] - hi.w);
    float *o = P.btab + (size_t)wc * 2 * kTcCols * kTcK + (size_t)nn * kTcK + pos;
    *reinterpret_cast<float4 *>(o) = hi;  // sw128_off(nn, k) / 4 == nn kTcK + pos
    *reinterpret_cast<float4 *>(o + kTcCols * kTcK) = lo;
  }
}

__device__ __forceinline__ void tc_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   saddr(bar))
               : "memory");
}

__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks) k_fast_kmulp_tc(
    Pass P, int32_t first_child0, int32_t first_child1) {
  using T = TcShape;
  extern __shared__ __align__(16) unsigned char smem[];
  // the swizzle is a function of the address: stages start 1024-byte aligned
  unsigned char *stages = smem + ((1024u - (saddr(smem) & 1023u)) & 1023u);  // [kTcStages][STAGE]
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + kTcStages * T::STAGE);
  uint64_t *full = bars, *empty = bars + kTcStages, *done = bars + 2 * kTcStages;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + T::NBAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nf = freq_count(P.p);
  const int w = blockIdx.y;
  const int32_t pos0 = P.bpos[first_child0], pos1 = P.bpos[first_child1];
  const int32_t row0 = pos0 + blockIdx.x * (kTcTiles * kTcRows);
  if (row0 >= pos1) return;  // the whole CTA: nothing allocated yet
  if (tid == 0) {
    for (int b = 0; b < kTcStages; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[b])),
                   "r"(kTcProducers)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[b])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int32_t nbox = P.t.nbox;
  bool ok = true;

  if (warp < 4) {
    // ---------------------------------------------------------- producers
    // warp pw copies rows 32 pw .. 32 pw + 31 of every tile; lane holds the
    // neighbour's local plist position for row 32 pw + lane, and in a copy
    // round 8 lanes take one row (lane / 8) and its 16-byte pieces (lane % 8)
    const unsigned char *UHH = reinterpret_cast<const unsigned char *>(P.uhh);
    const unsigned char *UHL = reinterpret_cast<const unsigned char *>(P.uhl);
    const int32_t npar = min(pos1 - pos0, P.uslots / 8);
    const size_t wrow = (size_t)w * P.uslots;  // first slot of this frequency
    int32_t rowi[kTcTiles];
#pragma unroll
    for (int k = 0; k < kTcTiles; ++k) rowi[k] = row0 + k * kTcRows + 32 * warp + lane;
    // neighbour positions of the next direction are loaded while the current
    // one is copied
    auto load_q = [&](int dd, int32_t *q) {
#pragma unroll
      for (int k = 0; k < kTcTiles; ++k) {
        int32_t v = rowi[k] < pos1 ? P.vpar[(size_t)dd * nbox + rowi[k]] : -1;
        if (v >= 0) {
          v -= pos0;
          if (v < 0 || v >= npar) {
            bad_index(P);
            v = -1;
          }
        }
        q[k] = v;
      }
    };
    int32_t qcur[kTcTiles], qnext[kTcTiles];
    load_q(0, qcur);
    const int rsub = lane >> 3, piece = lane & 7;
    for (int g = 0; g < kTcChunks && ok; ++g) {
      const int s = g % kTcStages, dd = g >> 1, half = g & 1;
      if (half == 0 && dd + 1 < kTcChunks / 2) load_q(dd + 1, qnext);
      if (g >= kTcStages && !tc_wait(&empty[s], (uint32_t)(((g / kTcStages) - 1) & 1))) {
        ok = false;
        if (P.err) atomicCAS(P.err, 0, kErrTimeout);
        break;
      }
      unsigned char *st = stages + (size_t)s * T::STAGE;
#pragma unroll
      for (int k = 0; k < kTcTiles; ++k) {
        unsigned char *ah = st + (size_t)k * 2 * T::ATILE, *al = ah + T::ATILE;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rw = 4 * i + rsub;            // row within the warp's 32
          const int32_t lq = __shfl_sync(kFull, qcur[k], rw);
          const int r = 32 * warp + rw;            // row within the tile
          const bool okc = lq >= 0;
          const size_t go = okc ? ((wrow + 8 * (size_t)lq + 4 * half) * 32 + 16 * piece) : 0;
          const uint32_t o = sw128_off(r, 4 * piece);
          cp_async_zfill(ah + o, UHH + go, okc, 16);
          cp_async_zfill(al + o, UHL + go, okc, 16);
        }
      }
      {  // B: the chunk's kernel spectra, hi then lo, as laid out in the table
        unsigned char *bdst = st + T::ASTAGE;
        const unsigned char *bsrc = reinterpret_cast<const unsigned char *>(
            P.btab + ((size_t)w * kTcChunks + g) * 2 * kTcCols * kTcK);
        for (int e = tid; e < 2 * T::BTILE / 16; e += kTcProducers)
          cp_async_zfill(bdst + 16 * e, bsrc + 16 * e, true, 16);
      }
      cp_async_commit();
      if (g >= kTcAhead) {  // chunk g - kTcAhead: its copies have landed
        cp_async_wait<kTcAhead>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_arrive(&full[(g - kTcAhead) % kTcStages]);
      }
      if (half == 1)
#pragma unroll
        for (int k = 0; k < kTcTiles; ++k) qcur[k] = qnext[k];
    }
    cp_async_wait<0>();
    if (ok) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int c = kTcChunks - kTcAhead; c < kTcChunks; ++c) tc_arrive(&full[c % kTcStages]);
    }
  } else if (tid == kTcProducers) {
    // ---------------------------------------------------------------- MMA
    // D F32, A and B TF32, K-major; N = 96 (B hi then B lo, adjacent in the
    // stage) or 48 (B hi), M = 128
    const uint32_t idesc96 = (1u << 4) | (2u << 7) | (2u << 10) |
                             ((uint32_t)(2 * kTcCols >> 3) << 17) |
                             ((uint32_t)(kTcRows >> 4) << 24);
    const uint32_t idesc48 = (1u << 4) | (2u << 7) | (2u << 10) |
                             ((uint32_t)(kTcCols >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
    int last = -1;
    for (int g = 0; g < kTcChunks; ++g) {
      const int s = g % kTcStages;
      if (!tc_wait(&full[s], (uint32_t)((g / kTcStages) & 1))) {
        ok = false;
        if (P.err) atomicCAS(P.err, 0, kErrTimeout);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned char *st = stages + (size_t)s * T::STAGE;
      const uint32_t bh = saddr(st + T::ASTAGE);
#pragma unroll
      for (int tt = 0; tt < kTcTiles; ++tt) {
        const uint32_t ah = saddr(st + (size_t)tt * 2 * T::ATILE), al = ah + T::ATILE;
        const uint32_t d = tmem + (uint32_t)(tt * 128);
#pragma unroll
        for (int ks = 0; ks < kTcK / 8; ++ks) {
          const uint32_t kb = 32u * ks;  // 8 TF32 per K-step
          // [hi.hi | hi.lo] in one product of N = 96, then lo.hi into the first half
          tc_mma(d, tc_sdesc_sw128(ah + kb), tc_sdesc_sw128(bh + kb), idesc96,
                 (g > 0 || ks > 0) ? 1u : 0u);
          tc_mma(d, tc_sdesc_sw128(al + kb), tc_sdesc_sw128(bh + kb), idesc48, 1u);
        }
      }
      tc_commit(&empty[s]);
      last = g;
    }
    if (ok) {
      tc_commit(done);
    } else if (last >= 0 &&
               !tc_wait(&empty[last % kTcStages], (uint32_t)((last / kTcStages) & 1))) {
      if (P.err) atomicCAS(P.err, 0, kErrTimeout);
    }
  }
  if (warp >= 4) {
    // ----------------------------------------------------------- epilogue
    __syncwarp();
    const bool fin = tc_wait(done, 0);
    if (!fin && lane == 0 && P.err) atomicCAS(P.err, 0, kErrTimeout);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__all_sync(kFull, fin)) {
      const int quarter = warp & 3;
#pragma unroll 1
      for (int tt = 0; tt < kTcTiles; ++tt) {
        const int32_t i = row0 + tt * kTcRows + quarter * 32 + lane;
        float d[kTcCols];
#pragma unroll
        for (int part = 0; part < 2 * kTcCols / 16; ++part) {
          uint32_t v[16];
          const uint32_t taddr =
              tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tt * 128 + part * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
              "%10, %11, %12, %13, %14, %15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int c = part * 16 + e;  // hi.hi + lo.hi, then hi.lo
            if (c < kTcCols)
              d[c] = __uint_as_float(v[e]);
            else
              d[c - kTcCols] += __uint_as_float(v[e]);
          }
        }
        if (i < pos1) {
          const int32_t par = P.plist[i];
          if (in_range(P, par, nbox)) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int32_t ct = P.child8[8 * (size_t)par + t];
              if (ct < 0 || !in_range(P, ct, nbox)) continue;
              // check spectra [box][component][2 nfreq] (re, im per frequency):
              // the rows of the inverse-DFT product
              float2 *o = reinterpret_cast<float2 *>(P.chat32 + (size_t)ct * 6 * nf) + w;
#pragma unroll
              for (int q = 0; q < 3; ++q)
                o[(size_t)q * nf] = make_float2(d[t * 6 + 2 * q], d[t * 6 + 2 * q + 1]);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcTmemCols)
                 : "memory");
  }
}


// Work items of the L2T (leaf points against the leaf's downward density and
// its W-list boxes' upward densities): a block of pb points (a power of two,
// 8 <= pb <= 256) against all of the leaf's sources, S = 256 / pb threads per
// point (adjacent lanes, each taking every S-th staged source pair, summed by
// shuffles in a fixed order).  pb is the largest with pb x sources <=
// kItemWork (and no larger than the points need), so that a leaf with a long
// W-list is spread over many CTAs; every point is evaluated by one item,
// whatever the grid.
constexpr int kItemThreads = 256;
constexpr int64_t kItemWork = (int64_t)1 << 16;  // point-source pairs per item aimed at
__device__ __forceinline__ int item_targets(int ntarget, int64_t nsrc) {
  int pb = kItemThreads;
  while (pb > 8 && (int64_t)pb * nsrc > kItemWork) pb >>= 1;
  int cap = 8;
  while (cap < ntarget && cap < kItemThreads) cap <<= 1;
  return pb < cap ? pb : cap;
}
// Items per leaf: icnt[l], the block size in ipb[l] (log2).
__global__ void k_fast_item_counts(Pass P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < P.t.nleaf; l += stride) {
    int32_t cnt = 0, lg = 3;
    int pb = 8;
    const int32_t b = P.t.leaf_box[l];
    if (in_range(P, b, P.t.nbox)) {
      const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
      if (i1 > i0 && in_range(P, i0, P.n + 1) && in_range(P, i1, P.n + 1)) {
        const int64_t nsrc =
            (int64_t)P.ns * ((P.t.depth[b] >= kFirstDepth ? 1 : 0) + P.t.w_ptr[b + 1] - P.t.w_ptr[b]);
        pb = item_targets((int)min(i1 - i0, (int64_t)kItemThreads), nsrc);
        cnt = (int32_t)((i1 - i0 + pb - 1) / pb);
      }
    }
    while ((1 << lg) < pb) ++lg;
    P.icnt[l] = cnt;
    P.ipb[l] = lg;
  }
}
// The items in leaf order: items[ioff[l] + i] = (l, i | log2(pb) << 24).
__global__ void k_fast_item_expand(Pass P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < P.t.nleaf; l += stride) {
    const int32_t o = P.ioff[l], c = P.icnt[l], lg = P.ipb[l];
    for (int32_t i = 0; i < c; ++i) {
      P.items[2 * (size_t)(o + i)] = (int32_t)l;
      P.items[2 * (size_t)(o + i) + 1] = i | (lg << 24);
    }
  }
}

// DCHK: one CTA per box of one depth; threads 2c, 2c + 1 take downward check
// points 2c, 2c + 1 (every other staged pair each): M2L (spectral result, or
// dense over the V-list in batches of boxes), X-list sources (one leaf at a
// time, in this box's frame), L2L.  Offsets of source boxes are computed once
// per box, by one thread.
__global__ void k_fast_dchk(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[kEqBatchMax];
  __shared__ float xoff[3];
  const int neq = eq_batch_boxes(P.ns);
  const int cap = (neq * P.ns + 1) / 2, scap = blockDim.x;
  float4 *E = reinterpret_cast<float4 *>(smem);  // kEqFields planes of cap pairs
  float4 *S = E + (size_t)kEqFields * cap;       // kSrcFields planes of scap pairs
  const int32_t b = P.box0 + blockIdx.x;
  const int k0 = threadIdx.x & ~1, sl = threadIdx.x & 1;
  const bool act = k0 + 1 < P.ns;  // ns is even
  const float r = half_width(P.t, P.depth);
  const float rad = (float)(kInner * (double)r);
  float xs[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if (act)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) xs[t][q] = rad * P.surf32[3 * (k0 + t) + q];
  float2 x2[2][3], u2[2][3], uf[2][3], uq[2][3];
  dup_targets(xs, x2);
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) u2[t][q] = uf[t][q] = uq[t][q] = make_float2(0.f, 0.f);
  // equivalent sources: the dense V-list (no spectra) and the parent (L2L)
  const int32_t v0 = P.spec ? 0 : P.t.v_ptr[b], v1 = P.spec ? 0 : P.t.v_ptr[b + 1];
  const int nl2l = P.depth > kFirstDepth ? 1 : 0;
  const int neqs = (v1 - v0) + nl2l;
  for (int e0 = 0; e0 < neqs; e0 += neq) {
    const int nb = min(neq, neqs - e0);
    __syncthreads();
    if ((int)threadIdx.x < nb) {
      const int e = e0 + threadIdx.x;
      EqSrc q;
      if (e < v1 - v0) {
        const int32_t a = P.t.v_idx[v0 + e];
        if (in_range(P, a, P.t.nbox)) {
          q.dens = P.up32 + (size_t)a * P.nc * P.ns;
          q.nc = P.nc;
          q.rad = rad;
          offset_f(P.t, b, P.depth, a, P.depth, q.off);
        } else {
          q = eq_none(P);
        }
      } else {
        const int32_t pb = P.t.parent[b];
        if (in_range(P, pb, P.t.nbox)) {
          q.dens = P.dn32 + (size_t)pb * 3 * P.ns;
          q.nc = 3;
          q.rad = (float)(kOuter * 2.0 * (double)r);
          offset_f(P.t, b, P.depth, pb, P.depth - 1, q.off);
        } else {
          q = eq_none(P);
        }
      }
      src[threadIdx.x] = q;
    }
    __syncthreads();
    stage_eq_pairs(P, E, cap, src, nb);
    __syncthreads();
    if (act) {
      if (P.nc == 4) eval_eq_pairs<true>(E, cap, sl, (nb * P.ns + 1) / 2, 2, x2, uf, uq);
      else eval_eq_pairs<false>(E, cap, sl, (nb * P.ns + 1) / 2, 2, x2, uf, uq);
    }
  }
  const int chunk = 2 * (int)blockDim.x;
  for (int32_t v = P.t.x_ptr[b]; v < P.t.x_ptr[b + 1]; ++v) {  // X-list sources
    const int32_t a = P.t.x_idx[v];
    if (!in_range(P, a, P.t.nbox)) continue;
    const int32_t l = P.t.box_leaf[a];
    if (l < 0) continue;  // not a leaf: not an X-list entry
    if (!in_range(P, l, P.t.nleaf)) continue;
    const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
    if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1)) continue;
    __syncthreads();
    if (threadIdx.x == 0) offset_f(P.t, b, P.depth, a, P.t.depth[a], xoff);
    __syncthreads();
    float2 xo[2][3];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) xo[t][q] = p_dup(xoff[q] + xs[t][q]);
    for (int64_t c0 = i0; c0 < i1; c0 += chunk) {
      const int n = (int)min((int64_t)chunk, i1 - c0);
      __syncthreads();
      stage_point_pairs(P, S, scap, c0, n);
      __syncthreads();
      if (act) eval_src_pairs_any(P, S, scap, sl, (n + 1) / 2, 2, xo, u2);
    }
  }
  float a0[2][3], a1[2][3], a2[2][3], u[2][3];
  fold_halves(u2, a0);
  fold_halves(uf, a1);
  fold_halves(uq, a2);
  const float csl = (float)P.csl, csrc = (float)P.csrc;
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) u[t][q] = a0[t][q] + csl * a1[t][q] + csrc * a2[t][q];
  lane_sum2(u, 2);
  if (act && sl == 0)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int k = k0 + t;
        const float m2l = P.spec ? P.m2l32[((size_t)b * 3 + q) * P.ns + k] : 0.f;
        P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = m2l + u[t][q];
      }
}

// L2T + W-list: items of the leaves (k_fast_item_counts); a thread takes one
// point and every S-th staged source pair (S adjacent lanes per point); the
// leaf's downward density and its W-list boxes' upward densities are staged
// in batches in the leaf's frame.
__global__ void __launch_bounds__(kItemThreads) k_fast_l2t(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[kEqBatchMax];
  const int neq = eq_batch_boxes(P.ns);
  const int cap = (neq * P.ns + 1) / 2;
  float4 *E = reinterpret_cast<float4 *>(smem);  // kEqFields planes of cap pairs
  const int32_t it1 = P.ioff[P.t.nleaf];
  const float csl = (float)P.csl, csrc = (float)P.csrc;
  for (int32_t it = blockIdx.x; it < it1; it += gridDim.x) {
    const int2 item = make_int2(P.items[2 * (size_t)it], P.items[2 * (size_t)it + 1]);
    const int32_t l = item.x;
    if (l < 0 || l >= P.t.nleaf) {  // uniform over the CTA
      if (threadIdx.x == 0) bad_index(P);
      continue;
    }
    const int32_t b = P.t.leaf_box[l];
    if (!in_range(P, b, P.t.nbox)) continue;
    const int d = P.t.depth[b];
    const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
    if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1) || i1 <= i0) continue;
    const int pb = 1 << (item.y >> 24), sw = kItemThreads / pb;
    const int64_t e = i0 + (int64_t)(item.y & 0xffffff) * pb + (int)threadIdx.x / sw;
    const int sl = (int)threadIdx.x % sw;
    const bool act = e < i1;
    const float r = half_width(P.t, d);
    const int32_t w0 = P.t.w_ptr[b], w1 = P.t.w_ptr[b + 1];
    const int ndn = d >= kFirstDepth ? 1 : 0;
    const int neqs = ndn + (w1 - w0);
    float2 x2[1][3], uf[1][3], uq[1][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      x2[0][q] = p_dup(act ? P.ploc[3 * e + q] : 0.f);
      uf[0][q] = uq[0][q] = make_float2(0.f, 0.f);
    }
    for (int e0 = 0; e0 < neqs; e0 += neq) {
      const int nb = min(neq, neqs - e0);
      __syncthreads();
      if ((int)threadIdx.x < nb) {
        const int ee = e0 + threadIdx.x;
        EqSrc q;
        if (ee < ndn) {
          q.dens = P.dn32 + (size_t)b * 3 * P.ns;
          q.nc = 3;
          q.rad = (float)(kOuter * (double)r);
          q.off[0] = q.off[1] = q.off[2] = 0.f;
        } else {
          const int32_t a = P.t.w_idx[w0 + ee - ndn];
          if (in_range(P, a, P.t.nbox)) {
            const int da = P.t.depth[a];
            q.dens = P.up32 + (size_t)a * P.nc * P.ns;
            q.nc = P.nc;
            q.rad = (float)(kInner * (double)half_width(P.t, da));
            offset_f(P.t, b, d, a, da, q.off);
          } else {
            q = eq_none(P);
          }
        }
        src[threadIdx.x] = q;
      }
      __syncthreads();
      stage_eq_pairs(P, E, cap, src, nb);
      __syncthreads();
      if (act) {
        if (P.nc == 4) eval_eq_pairs<true, 1>(E, cap, sl, (nb * P.ns + 1) / 2, sw, x2, uf, uq);
        else eval_eq_pairs<false, 1>(E, cap, sl, (nb * P.ns + 1) / 2, sw, x2, uf, uq);
      }
    }
    float u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      u[q] = csl * (uf[0][q].x + uf[0][q].y) + csrc * (uq[0][q].x + uq[0][q].y);
      for (int o = 1; o < sw; o <<= 1) u[q] += __shfl_xor_sync(kFull, u[q], o);
    }
    if (act && sl == 0) {
      double *out = P.out + 3 * e;
#pragma unroll
      for (int a = 0; a < 3; ++a) out[a] = (P.accumulate ? out[a] : 0.0) + f32_to_f64(u[a]);
    }
  }
}

// Threads per CTA of the per-box kernels: the check points, rounded up to
// whole warps.
int box_threads(int ns) { return ((ns + 31) / 32) * 32; }

// Check-to-equivalent products of the nb boxes of one depth: kFastTile boxes
// per CTA, one operator row per thread (16 boxes per CTA measured slower).
template <bool UP>
void launch_c2e(const Pass &P, int32_t nb, int ns, cudaStream_t st) {
  const int rows = UP ? P.nc * ns : 3 * ns;
  int threads = ((rows + 31) / 32) * 32;
  if (threads > 256) threads = 256;
  const size_t cols = 3 * (size_t)ns;
  k_fast_c2e<UP, kFastTile><<<(unsigned)((nb + kFastTile - 1) / kFastTile), threads,
                              sizeof(float) * kFastTile * cols, st>>>(P);
}

}  // namespace

// Host launch sequence of the CTA-blocked mixed form (p <= kFastMaxP).
cudaError_t far_field_fast(const Pass &P0, const int32_t *depth_ptr, int32_t max_depth,
                           int sms, cudaStream_t st, const FastHooks &hk) {
  Pass P = P0;
  const int ns = P.ns, nf = freq_count(P.p);
  const bool fft = P.spec != nullptr;
  const int bt = box_threads(ns);
  cudaError_t err = cudaSuccess;
  int seq = 0;
  auto pre = [&](const char *name) { hk.before(seq, name, st); };
  auto post = [&]() {
    if (err == cudaSuccess) err = cudaGetLastError();
    hk.after(seq, st);
    ++seq;
    count_launches(1);
  };
  const int64_t grid_cap = (int64_t)sms * 8;
  auto gs = [&](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, grid_cap)); };

  // the spectral products take more than 48 KB of dynamic shared memory (the
  // attribute is set on every call: it is per device and cheap)
  if (fft) {
    if ((err = cudaFuncSetAttribute(k_fast_kmulp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TcShape::SMEM)) != cudaSuccess)
      return err;
  }
  // set-up: octant table, first-child flags, parent list, DFT tables
  if ((err = cudaMemsetAsync(P.child8, 0xff, sizeof(int32_t) * 8 * (size_t)P.t.nbox, st)) !=
      cudaSuccess)
    return err;
  const int64_t ntab = std::max<int64_t>(P.t.nbox, fft ? (int64_t)ns * nf : 0);
  CUtensorMap chat_map;
  if (fft) {
    const size_t nb_tab = tc::b_table_floats(ifft_tiles(ns), ifft_chunks(P.p));
    if ((err = cudaMemsetAsync(P.fitab, 0, sizeof(float) * nb_tab, st)) != cudaSuccess) return err;
    // check spectra [box][component][2 nfreq] as the rows of the inverse DFT
    if ((err = tc::encode_a(&chat_map, P.chat32, 3 * (uint64_t)P.t.nbox, 2 * (uint64_t)nf,
                            2 * (uint64_t)nf)) != cudaSuccess)
      return err;
  }
  pre("tables");
  k_fast_tables<<<gs(ntab), 256, 0, st>>>(P, ntab);
  post();
  pre("scan");
  launch_scan(P.bflag, P.t.nbox, P.bpos, P.bpos + P.t.nbox, st);
  if (err == cudaSuccess) err = cudaGetLastError();
  hk.after(seq, st);
  ++seq;
  pre("plist");
  k_fast_plist<<<gs(P.t.nbox), 256, 0, st>>>(P);
  post();
  {
    // work items of the L2T (counts, their scan, the item list)
    const int64_t ne = P.t.nleaf;
    pre("items");
    k_fast_item_counts<<<gs(ne), 256, 0, st>>>(P);
    count_launches(1);
    if (err == cudaSuccess) err = cudaGetLastError();
    launch_scan(P.icnt, ne, P.ioff, P.ioff + ne, st);
    if (err == cudaSuccess) err = cudaGetLastError();
    k_fast_item_expand<<<gs(ne), 256, 0, st>>>(P);
    post();
  }
  if (fft) {
    pre("vpar");
    k_fast_vpar<<<gs((int64_t)P.t.nbox * 26), 256, 0, st>>>(P);
    post();
  }
  pre("pack");
  k_fast_pack<<<(P.t.nleaf + kPackLeaves - 1) / kPackLeaves, kPackLeaves * 32, 0, st>>>(P);
  post();
  {
    const int64_t n = P.n_uc2e + P.n_dc2e;
    pre("opsplit");
    if (n > 0) k_fast_opsplit<<<gs(n), 256, 0, st>>>(P, n);
    post();
  }
  if (fft) {
    const int64_t n = (int64_t)343 * nf * 3 * P.nc * 2;
    pre("spec");
    k_fast_spec<<<gs(n), 256, 0, st>>>(P, n);
    post();
    const int64_t nb = (int64_t)nf * kTcChunks * kTcCols * kTcK;
    pre("btab");
    k_fast_btab<<<gs(nb / 4), 256, 0, st>>>(P, nb);
    post();
  }
  pre("s2m");
  k_fast_s2m<<<P.t.nleaf, bt, sizeof(float4) * kSrcFields * bt, st>>>(P);
  post();
  for (int32_t d = max_depth; d >= kFirstDepth; --d) {
    P.depth = d;
    P.box0 = depth_ptr[d];
    P.box1 = depth_ptr[d + 1];
    const int32_t nb = P.box1 - P.box0;
    if (nb <= 0) continue;
    if (d < max_depth) {
      pre("m2m");
      k_fast_m2m<<<nb, bt,
                   sizeof(float4) * kEqFields * ((std::min(8, eq_batch_boxes(ns)) * ns + 1) / 2),
                   st>>>(P);
      post();
    }
    pre("uc2e");
    launch_c2e<true>(P, nb, ns, st);
    post();
  }
  for (int32_t d = kFirstDepth; d <= max_depth; ++d) {
    P.depth = d;
    P.box0 = depth_ptr[d];
    P.box1 = depth_ptr[d + 1];
    const int32_t nb = P.box1 - P.box0;
    if (nb <= 0) continue;
    if (fft) {
      // parents of this depth's boxes: at most the boxes of the depth above,
      // and at most the boxes of this depth
      const int32_t npar_max = std::min(depth_ptr[d] - depth_ptr[d - 1], nb);
      pre("ufft");
      const dim3 gu((unsigned)npar_max, (unsigned)((nf + 127) / 128));
      if (P.nc == 4)
        k_fast_ufft<4><<<gu, 128, ufft_smem(ns, 4), st>>>(P, depth_ptr[d], depth_ptr[d + 1]);
      else
        k_fast_ufft<3><<<gu, 128, ufft_smem(ns, 3), st>>>(P, depth_ptr[d], depth_ptr[d + 1]);
      post();
      pre("kmulp");
      {
        const int rows = kTcTiles * kTcRows;
        const dim3 gt((unsigned)((npar_max + rows - 1) / rows), (unsigned)nf);
        k_fast_kmulp_tc<<<gt, kTcThreads, TcShape::SMEM, st>>>(P, depth_ptr[d], depth_ptr[d + 1]);
      }
      post();
      pre("ifft");
      {
        // the M2L part of the downward check velocities: rows (box, component)
        // of the check spectra times the inverse-DFT table, on the tensor cores
        tc::Args a{};
        a.a_row0 = 3 * (int64_t)P.box0;
        a.m = 3 * nb;
        a.k_chunks = ifft_chunks(P.p);
        a.n_tiles = ifft_tiles(ns);
        a.n = ns;
        a.btab = P.fitab;
        a.out = P.m2l32 + 3 * (size_t)P.box0 * ns;
        a.ldo = ns;
        a.err = P.err;
        a.spin_limit = kTcSpinLimit;
        const cudaError_t e = tc::gemm3(chat_map, a, st);
        if (err == cudaSuccess) err = e;
      }
      post();
    }
    pre("dchk");
    k_fast_dchk<<<nb, bt,
                  sizeof(float4) * (kEqFields * ((eq_batch_boxes(ns) * ns + 1) / 2) +
                                    kSrcFields * bt),
                  st>>>(P);
    post();
    pre("dc2e");
    launch_c2e<false>(P, nb, ns, st);
    post();
  }
  pre("l2t");
  {
    const int64_t bound = (int64_t)P.t.nleaf + (P.n + 7) / 8;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(bound, (int64_t)sms * 8));
    k_fast_l2t<<<g, kItemThreads,
                 sizeof(float4) * kEqFields * ((eq_batch_boxes(ns) * ns + 1) / 2), st>>>(P);
  }
  post();
  return err;
}

}  // namespace fmm
}  // namespace stk
