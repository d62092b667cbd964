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

namespace stk {
namespace fmm {

namespace {

constexpr int kFastTile = 8;       // boxes per CTA of the products
constexpr int kKmulThreads = 128;  // parents per CTA of the spectral products
constexpr int kStageThreads = 128; // CTA of the leaf kernels
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

// Source points staged in shared memory: local position, q = w f csl,
// psi = w phi cdl, normal (unused parts zero).
struct SrcStage {
  float4 y, q, p, n;
};

// Adds the single and double layer of n staged points at x.
template <bool SL, bool DL>
__device__ __forceinline__ void eval_sources(const SrcStage *S, int n, float x0, float x1, float x2,
                                             float u[3]) {
  for (int i = 0; i < n; ++i) {
    const float4 y = S[i].y;
    const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(r2 > 0.0f)) continue;
    const float ri = rsqrtf(r2), ri2 = ri * ri;
    if (SL) {
      const float4 q = S[i].q;
      const float dq = (d0 * q.x + d1 * q.y + d2 * q.z) * ri2 * ri;
      u[0] += q.x * ri + d0 * dq;
      u[1] += q.y * ri + d1 * dq;
      u[2] += q.z * ri + d2 * dq;
    }
    if (DL) {
      const float4 s = S[i].p, nn = S[i].n;
      const float c = (d0 * s.x + d1 * s.y + d2 * s.z) * (d0 * nn.x + d1 * nn.y + d2 * nn.z) *
                      ri2 * ri2 * ri;
      u[0] += d0 * c;
      u[1] += d1 * c;
      u[2] += d2 * c;
    }
  }
}

__device__ __forceinline__ void eval_sources_any(const Pass &P, const SrcStage *S, int n, float x0,
                                                 float x1, float x2, float u[3]) {
  if (P.qf && P.pf) eval_sources<true, true>(S, n, x0, x1, x2, u);
  else if (P.qf) eval_sources<true, false>(S, n, x0, x1, x2, u);
  else eval_sources<false, true>(S, n, x0, x1, x2, u);
}

// Stages points [i0, i0 + n) (n <= blockDim.x) of the packed arrays.
__device__ __forceinline__ void stage_points(const Pass &P, SrcStage *S, int64_t i0, int n) {
  const int t = threadIdx.x;
  if (t < n) {
    const int64_t i = i0 + t;
    SrcStage s;
    s.y = make_float4(P.ploc[3 * i], P.ploc[3 * i + 1], P.ploc[3 * i + 2], 0.f);
    s.q = P.qf ? make_float4(P.qf[3 * i], P.qf[3 * i + 1], P.qf[3 * i + 2], 0.f)
               : make_float4(0.f, 0.f, 0.f, 0.f);
    s.p = P.pf ? make_float4(P.pf[3 * i], P.pf[3 * i + 1], P.pf[3 * i + 2], 0.f)
               : make_float4(0.f, 0.f, 0.f, 0.f);
    s.n = P.nf ? make_float4(P.nf[3 * i], P.nf[3 * i + 1], P.nf[3 * i + 2], 0.f)
               : make_float4(0.f, 0.f, 0.f, 0.f);
    S[t] = s;
  }
}

// Equivalent density staged in shared memory: surface point (already scaled
// by the radius) and density (force x, y, z and source strength).
struct EqStage {
  float4 y, e;
};

// Adds the field of ns staged equivalent points at x (csl, csrc applied).
template <bool FLUX>
__device__ __forceinline__ void eval_equiv(const EqStage *E, int ns, float x0, float x1, float x2,
                                           float csl, float csrc, float u[3]) {
  float uf[3] = {0.f, 0.f, 0.f}, uq[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < ns; ++j) {
    const float4 y = E[j].y, e = E[j].e;
    const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(r2 > 0.0f)) continue;
    const float ri = rsqrtf(r2), ri3 = ri * ri * ri;
    const float df = (d0 * e.x + d1 * e.y + d2 * e.z) * ri3;
    uf[0] += e.x * ri + d0 * df;
    uf[1] += e.y * ri + d1 * df;
    uf[2] += e.z * ri + d2 * df;
    if (FLUX) {
      const float s = e.w * ri3;
      uq[0] += d0 * s;
      uq[1] += d1 * s;
      uq[2] += d2 * s;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] += csl * uf[a] + csrc * uq[a];
}

// A source box of a batch of equivalent densities: its density [ns][nc], the
// radius of its surface and its centre's offset from the target box's centre.
struct EqSrc {
  const float *dens;
  int32_t nc;
  float rad;
  float off[3];  // centre(target box) - centre(source box), FP32
};

// Stages the boxes src[0, nb) into E (nb ns points), each surface point in
// the target box's frame: rad s_j - off.
__device__ __forceinline__ void stage_eq_batch(const Pass &P, EqStage *E, const EqSrc *src,
                                               int nb) {
  const int total = nb * P.ns;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int k = e / P.ns, j = e % P.ns;
    const EqSrc &S = src[k];
    const float *sp = P.surf32 + 3 * j;
    const float *d = S.dens + (size_t)S.nc * j;
    E[e].y = make_float4(S.rad * sp[0] - S.off[0], S.rad * sp[1] - S.off[1],
                         S.rad * sp[2] - S.off[2], 0.f);
    E[e].e = S.nc == 0 ? make_float4(0.f, 0.f, 0.f, 0.f)
                       : make_float4(d[0], d[1], d[2], S.nc == 4 ? d[3] : 0.f);
  }
}

// Adds the field of the staged points j0, j0 + js, ... < n at x (csl, csrc
// applied by the caller through uf, uq).
template <bool FLUX>
__device__ __forceinline__ void eval_equiv_acc(const EqStage *E, int j0, int n, int js, float x0,
                                               float x1, float x2, float uf[3], float uq[3]) {
  for (int j = j0; j < n; j += js) {
    const float4 y = E[j].y, e = E[j].e;
    const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(r2 > 0.0f)) continue;
    const float ri = rsqrtf(r2), ri3 = ri * ri * ri;
    const float df = (d0 * e.x + d1 * e.y + d2 * e.z) * ri3;
    uf[0] += e.x * ri + d0 * df;
    uf[1] += e.y * ri + d1 * df;
    uf[2] += e.z * ri + d2 * df;
    if (FLUX) {
      const float sv = e.w * ri3;
      uq[0] += d0 * sv;
      uq[1] += d1 * sv;
      uq[2] += d2 * sv;
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

// ------------------------------------------------------------------ set-up
// child8, bflag and the lattice DFT tables; e runs over max(nbox, ns nfreq).
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
      // forward: ftab[j][w]; inverse: fitab[w][k] (k = j), the same angle
      const int j = (int)(e / nf), w = (int)(e % nf);
      const int kx = w / (G * nz), ky = (w / nz) % G, kz = w % nz;
      const int t = (P.sidx[3 * j] * kx + P.sidx[3 * j + 1] * ky + P.sidx[3 * j + 2] * kz) % G;
      double sn, c;
      sincospi((double)t / (double)P.p, &sn, &c);  // angle 2 pi t / G, G = 2p
      P.ftab[2 * e] = (float)c;
      P.ftab[2 * e + 1] = (float)(-sn);
      const double wt = (kz == 0 || kz == P.p) ? 1.0 : 2.0;
      const double inv = wt / ((double)G * G * G);
      const size_t o = 2 * ((size_t)w * P.ns + j);
      P.fitab[o] = (float)(inv * c);
      P.fitab[o + 1] = (float)(-inv * sn);
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
// CTA per leaf.
__global__ void k_fast_pack(Pass P) {
  const int32_t l = blockIdx.x;
  const int32_t b = P.t.leaf_box[l];
  if (!in_range(P, b, P.t.nbox)) return;
  const int d = P.t.depth[b];
  double c[3];
  centre(P.t, b, d, c);
  const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
  if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1)) return;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      P.ploc[3 * i + q] = (float)(P.pts[3 * i + q] - c[q]);
      if (P.qf) P.qf[3 * i + q] = (float)(P.csl * (P.w[i] * P.f[3 * i + q]));
      if (P.pf) {
        P.pf[3 * i + q] = (float)(P.cdl * (P.w[i] * P.phi[3 * i + q]));
        P.nf[3 * i + q] = (float)P.nrm[3 * i + q];
      }
    }
}

// ---------------------------------------------------------------- upward
// S2M: one CTA per leaf, thread k = check point on the 2.95 r surface.
__global__ void k_fast_s2m(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  SrcStage *S = reinterpret_cast<SrcStage *>(smem);
  const int32_t l = blockIdx.x;
  const int32_t b = P.t.leaf_box[l];
  if (!in_range(P, b, P.t.nbox)) return;
  const int d = P.t.depth[b];
  if (d < kFirstDepth) return;
  const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
  if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1) || i1 < i0) return;
  const int k = threadIdx.x;
  const float rad = (float)(kOuter * (double)half_width(P.t, d));
  float x[3] = {0.f, 0.f, 0.f}, u[3] = {0.f, 0.f, 0.f};
  if (k < P.ns)
#pragma unroll
    for (int q = 0; q < 3; ++q) x[q] = rad * P.surf32[3 * k + q];
  for (int64_t c0 = i0; c0 < i1; c0 += blockDim.x) {
    const int n = (int)min((int64_t)blockDim.x, i1 - c0);
    __syncthreads();
    stage_points(P, S, c0, n);
    __syncthreads();
    if (k < P.ns) eval_sources_any(P, S, n, x[0], x[1], x[2], u);
  }
  if (k < P.ns)
#pragma unroll
    for (int q = 0; q < 3; ++q) P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = u[q];
}

// M2M: one CTA per box of one depth with children; thread k = check point;
// the children's upward densities staged in batches, in this box's frame.
__global__ void k_fast_m2m(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[8];
  EqStage *E = reinterpret_cast<EqStage *>(smem);  // [min(8, neq) ns]
  const int32_t b = P.box0 + blockIdx.x;
  const int32_t c0 = P.t.child_ptr[b], c1 = P.t.child_ptr[b + 1];
  if (c0 >= c1) return;
  if (c1 - c0 > 8) {
    bad_index(P);
    return;
  }
  const int nch = c1 - c0, neq = min(8, eq_batch_boxes(P.ns));
  const int k = threadIdx.x;
  const float r = half_width(P.t, P.depth);
  const float rad = (float)(kOuter * (double)r), rc = (float)(kInner * (double)r / 2);
  if (k < nch) {
    const int32_t ch = c0 + k;
    EqSrc e;
    if (in_range(P, ch, P.t.nbox)) {
      e.dens = P.up32 + (size_t)ch * P.nc * P.ns;
      e.nc = P.nc;
      e.rad = rc;
      offset_f(P.t, b, P.depth, ch, P.depth + 1, e.off);
    } else {
      e = eq_none(P);
    }
    src[k] = e;
  }
  float x[3] = {0.f, 0.f, 0.f}, uf[3] = {0.f, 0.f, 0.f}, uq[3] = {0.f, 0.f, 0.f};
  if (k < P.ns)
#pragma unroll
    for (int q = 0; q < 3; ++q) x[q] = rad * P.surf32[3 * k + q];
  for (int e0 = 0; e0 < nch; e0 += neq) {
    const int nb = min(neq, nch - e0);
    __syncthreads();
    stage_eq_batch(P, E, src + e0, nb);
    __syncthreads();
    if (k < P.ns) {
      if (P.nc == 4) eval_equiv_acc<true>(E, 0, nb * P.ns, 1, x[0], x[1], x[2], uf, uq);
      else eval_equiv_acc<false>(E, 0, nb * P.ns, 1, x[0], x[1], x[2], uf, uq);
    }
  }
  if (k < P.ns) {
    const float csl = (float)P.csl, csrc = (float)P.csrc;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = csl * uf[q] + csrc * uq[q];
  }
}

// Check-to-equivalent products of a tile of NB boxes of one depth:
// out[b][i] = (hi + lo)[i] . chk32[b] in double-FP32 arithmetic (the exact
// FMA product and two-sum accumulation of apply_row_df), operator stored
// column by column, read four columns ahead of their use.
template <bool UP, int NB>
__global__ void __launch_bounds__(256) k_fast_c2e(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *X = reinterpret_cast<float *>(smem);  // [NB][cols]
  const int cols = 3 * P.ns;
  const int rows = UP ? P.nc * P.ns : 3 * P.ns;
  const int32_t bt = P.box0 + blockIdx.x * NB;
  const int nbt = min(NB, P.box1 - bt);
  for (int e = threadIdx.x; e < NB * cols; e += blockDim.x) {
    const int bb = e / cols, j = e % cols;
    X[e] = bb < nbt ? P.chk32[(size_t)(bt + bb) * cols + j] : 0.f;
  }
  __syncthreads();
  const size_t off = UP ? (size_t)(P.depth - kFirstDepth) * rows * cols
                        : (size_t)P.n_uc2e + (size_t)(P.depth - kFirstDepth) * rows * cols;
  const float *hi = P.ops_hi + off, *lo = P.ops_lo + off;
  float *out = UP ? P.up32 : P.dn32;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    float sh[NB], sl[NB];
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) sh[bb] = sl[bb] = 0.f;
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
#pragma unroll
        for (int bb = 0; bb < NB; ++bb) {
          const float x = X[bb * cols + j0 + q];
          const float p = __fmul_rn(ah[q], x);
          const float err = __fmaf_rn(al[q], x, __fmaf_rn(ah[q], x, -p));
          const float t = __fadd_rn(sh[bb], p), bv = __fsub_rn(t, sh[bb]);
          sl[bb] = __fadd_rn(sl[bb], __fadd_rn(__fadd_rn(__fsub_rn(sh[bb], __fsub_rn(t, bv)),
                                                         __fsub_rn(p, bv)),
                                               err));
          sh[bb] = t;
        }
      }
    }
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
      if (bb < nbt) out[(size_t)(bt + bb) * rows + i] = __fadd_rn(sh[bb], sl[bb]);
  }
}

// ------------------------------------------------------------- downward
// UFFT: spectra of the upward densities of a tile of boxes,
// uhat[b][w][c] = sum_j up[b][j][c] (cos - i sin)(2 pi (s_j . k_w mod G) / G);
// thread = frequency.
template <int NC>
__global__ void __launch_bounds__(128) k_fast_ufft(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *U = reinterpret_cast<float *>(smem);  // [kFastTile][ns][NC]
  const int nf = freq_count(P.p);
  const int32_t bt = P.box0 + blockIdx.y * kFastTile;
  const int nbt = min(kFastTile, P.box1 - bt);
  const int per = P.ns * NC;
  for (int e = threadIdx.x; e < kFastTile * per; e += blockDim.x) {
    const int bb = e / per, r = e % per;
    U[e] = bb < nbt ? P.up32[(size_t)(bt + bb) * per + r] : 0.f;
  }
  __syncthreads();
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nf) return;
  float re[kFastTile][NC], im[kFastTile][NC];
#pragma unroll
  for (int bb = 0; bb < kFastTile; ++bb)
#pragma unroll
    for (int c = 0; c < NC; ++c) re[bb][c] = im[bb][c] = 0.f;
  const float2 *F = reinterpret_cast<const float2 *>(P.ftab);
  for (int j = 0; j < P.ns; ++j) {
    const float2 f = F[(size_t)j * nf + w];
#pragma unroll
    for (int bb = 0; bb < kFastTile; ++bb)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float v = U[(bb * P.ns + j) * NC + c];
        re[bb][c] = fmaf(v, f.x, re[bb][c]);
        im[bb][c] = fmaf(v, f.y, im[bb][c]);
      }
  }
#pragma unroll
  for (int bb = 0; bb < kFastTile; ++bb) {
    if (bb >= nbt) break;
    float *o = P.uhat32 + ((size_t)(bt + bb) * nf + w) * NC * 2;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      o[2 * c] = re[bb][c];
      o[2 * c + 1] = im[bb][c];
    }
  }
}

// KMULP: the spectral M2L products of one depth (the boxes' parents one depth
// up), blocked by parent and walked by child octant.  Grid: (parent tiles of
// 128, frequencies).  V(b) for a child b of parent P is every child of P's
// 26 neighbours that does not touch b; in child-box units the offset of a
// source child in octant s of the neighbour in direction dv from the target
// in octant t is o = 2 dv + s - t, and the pair is in V exactly when some
// |o_q| >= 2.  The kernel spectra of the CTA's frequency are staged with a
// row stride of MP floats (a multiple of 4, so that a row is read as float4).
template <int NC>
__global__ void __launch_bounds__(kKmulThreads, 4) k_fast_kmulp(Pass P, int32_t first_child0,
                                                               int32_t first_child1) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int M = 3 * NC * 2;             // floats per offset and frequency
  constexpr int MP = (M + 3) / 4 * 4;       // staged row stride
  float *S = reinterpret_cast<float *>(smem);  // [343][MP]
  const int nf = freq_count(P.p);
  const int w = blockIdx.y;
  {
    const float *src = P.spec32 + (size_t)w * 343 * M;
    for (int e = threadIdx.x; e < 343 * M; e += blockDim.x) S[(e / M) * MP + e % M] = src[e];
  }
  __syncthreads();
  const int32_t pos0 = P.bpos[first_child0], pos1 = P.bpos[first_child1];
  const int32_t i = pos0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pos1) return;
  const int32_t par = P.plist[i];
  if (!in_range(P, par, P.t.nbox)) return;
  const float r = half_width(P.t, P.depth);
  const float sf = 1.0f / r, sq = 1.0f / (r * r);
  float acc[8][6];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[t][q] = 0.f;
  const float2 *UH = reinterpret_cast<const float2 *>(P.uhat32);
  const int4 *C8 = reinterpret_cast<const int4 *>(P.child8);
  for (int dir = 0; dir < 27; ++dir) {
    if (dir == 13) continue;  // the parent itself: its children touch each other
    int32_t Q = P.t.colleague[27 * (size_t)par + dir];
    if (Q >= P.t.nbox) {
      bad_index(P);
      Q = -1;
    }
    int4 ca = make_int4(-1, -1, -1, -1), cb = ca;
    if (Q >= 0) {
      ca = C8[2 * (size_t)Q];
      cb = C8[2 * (size_t)Q + 1];
    }
    const int32_t an[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    const int dx = dir / 9 - 1, dy = (dir / 3) % 3 - 1, dz = dir % 3 - 1;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int32_t a = an[s];
      if (a >= P.t.nbox) {
        bad_index(P);
        a = -1;
      }
      float2 u[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float sc = c < 3 ? sf : sq;
        const float2 v = a >= 0 ? UH[((size_t)a * nf + w) * NC + c] : make_float2(0.f, 0.f);
        u[c] = make_float2(v.x * sc, v.y * sc);
      }
      const int sx = s >> 2, sy = (s >> 1) & 1, sz = s & 1;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int ox = 2 * dx + sx - (t >> 2), oy = 2 * dy + sy - ((t >> 1) & 1),
                  oz = 2 * dz + sz - (t & 1);
        if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
        const float4 *K4 =
            reinterpret_cast<const float4 *>(S + ((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)) * MP);
        float K[MP];
#pragma unroll
        for (int v = 0; v < MP / 4; ++v) {
          const float4 kv = K4[v];
          K[4 * v] = kv.x;
          K[4 * v + 1] = kv.y;
          K[4 * v + 2] = kv.z;
          K[4 * v + 3] = kv.w;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float kr = K[2 * (q * NC + c)], ki = K[2 * (q * NC + c) + 1];
            acc[t][2 * q] = fmaf(kr, u[c].x, fmaf(-ki, u[c].y, acc[t][2 * q]));
            acc[t][2 * q + 1] = fmaf(kr, u[c].y, fmaf(ki, u[c].x, acc[t][2 * q + 1]));
          }
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int32_t ct = P.child8[8 * (size_t)par + t];
    if (ct < 0) continue;
    if (!in_range(P, ct, P.t.nbox)) continue;
    float *o = P.chat32 + ((size_t)ct * nf + w) * 6;
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = acc[t][q];
  }
}

// IFFT: the M2L part of the downward check velocity of a tile of 16 boxes at
// their check points, from the half spectrum.  Two groups of box_threads(ns)
// threads (8 boxes each) share the staged inverse-DFT rows of wc frequencies.
constexpr int kIfftBoxes = 16;
__global__ void k_fast_ifft(Pass P, int wc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nf = freq_count(P.p);
  const int bt_threads = blockDim.x / 2;
  float2 *F = reinterpret_cast<float2 *>(smem);                        // [wc][ns]
  float *C = reinterpret_cast<float *>(F + (size_t)wc * P.ns);         // [16][wc][6]
  const int32_t bt = P.box0 + blockIdx.x * kIfftBoxes;
  const int nbt = min(kIfftBoxes, P.box1 - bt);
  const int k = threadIdx.x % bt_threads, half = threadIdx.x / bt_threads;
  float acc[8][3];
#pragma unroll
  for (int bb = 0; bb < 8; ++bb) acc[bb][0] = acc[bb][1] = acc[bb][2] = 0.f;
  const float2 *FI = reinterpret_cast<const float2 *>(P.fitab);
  for (int w0 = 0; w0 < nf; w0 += wc) {
    const int nw = min(wc, nf - w0);
    __syncthreads();
    for (int e = threadIdx.x; e < nw * P.ns; e += blockDim.x) F[e] = FI[(size_t)w0 * P.ns + e];
    for (int e = threadIdx.x; e < kIfftBoxes * wc * 6; e += blockDim.x) {
      const int bb = e / (wc * 6), r = e % (wc * 6);
      const int ww = r / 6, q = r % 6;
      C[e] = (bb < nbt && ww < nw) ? P.chat32[((size_t)(bt + bb) * nf + w0 + ww) * 6 + q] : 0.f;
    }
    __syncthreads();
    if (k < P.ns)
      for (int ww = 0; ww < nw; ++ww) {
        const float2 f = F[ww * P.ns + k];
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) {
          const float *c = C + ((half * 8 + bb) * wc + ww) * 6;
#pragma unroll
          for (int q = 0; q < 3; ++q) acc[bb][q] = fmaf(c[2 * q], f.x, fmaf(c[2 * q + 1], f.y, acc[bb][q]));
        }
      }
  }
  if (k < P.ns)
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      const int b2 = half * 8 + bb;
      if (b2 < nbt)
#pragma unroll
        for (int q = 0; q < 3; ++q) P.m2l32[(size_t)(bt + b2) * 3 * P.ns + 3 * k + q] = acc[bb][q];
    }
}

// DCHK: one CTA per box of one depth, thread k = downward check point:
// M2L (spectral result, or dense over the V-list in batches of boxes), X-list
// sources (one leaf at a time, in this box's frame), L2L.  Offsets of source
// boxes are computed once per box, by one thread.
__global__ void k_fast_dchk(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[kEqBatchMax];
  __shared__ float xoff[3];
  const int neq = eq_batch_boxes(P.ns);
  EqStage *E = reinterpret_cast<EqStage *>(smem);                                  // [neq ns]
  SrcStage *S = reinterpret_cast<SrcStage *>(smem + sizeof(EqStage) * neq * P.ns);  // [blockDim]
  const int32_t b = P.box0 + blockIdx.x;
  const int k = threadIdx.x;
  const bool act = k < P.ns;
  const float r = half_width(P.t, P.depth);
  const float rad = (float)(kInner * (double)r);
  float xs[3] = {0.f, 0.f, 0.f}, u[3] = {0.f, 0.f, 0.f};
  float uf[3] = {0.f, 0.f, 0.f}, uq[3] = {0.f, 0.f, 0.f};
  if (act) {
#pragma unroll
    for (int q = 0; q < 3; ++q) xs[q] = rad * P.surf32[3 * k + q];
    if (P.spec)
#pragma unroll
      for (int q = 0; q < 3; ++q) u[q] = P.m2l32[(size_t)b * 3 * P.ns + 3 * k + q];
  }
  // equivalent sources: the dense V-list (no spectra) and the parent (L2L)
  const int32_t v0 = P.spec ? 0 : P.t.v_ptr[b], v1 = P.spec ? 0 : P.t.v_ptr[b + 1];
  const int nl2l = P.depth > kFirstDepth ? 1 : 0;
  const int neqs = (v1 - v0) + nl2l;
  for (int e0 = 0; e0 < neqs; e0 += neq) {
    const int nb = min(neq, neqs - e0);
    __syncthreads();
    if (k < nb) {
      const int e = e0 + k;
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
      src[k] = q;
    }
    __syncthreads();
    stage_eq_batch(P, E, src, nb);
    __syncthreads();
    if (act) {
      if (P.nc == 4) eval_equiv_acc<true>(E, 0, nb * P.ns, 1, xs[0], xs[1], xs[2], uf, uq);
      else eval_equiv_acc<false>(E, 0, nb * P.ns, 1, xs[0], xs[1], xs[2], uf, uq);
    }
  }
  for (int32_t v = P.t.x_ptr[b]; v < P.t.x_ptr[b + 1]; ++v) {  // X-list sources
    const int32_t a = P.t.x_idx[v];
    if (!in_range(P, a, P.t.nbox)) continue;
    const int32_t l = P.t.box_leaf[a];
    if (l < 0) continue;  // not a leaf: not an X-list entry
    if (!in_range(P, l, P.t.nleaf)) continue;
    const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
    if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1)) continue;
    __syncthreads();
    if (k == 0) offset_f(P.t, b, P.depth, a, P.t.depth[a], xoff);
    __syncthreads();
    const float o0 = xoff[0], o1 = xoff[1], o2 = xoff[2];
    for (int64_t c0 = i0; c0 < i1; c0 += blockDim.x) {
      const int n = (int)min((int64_t)blockDim.x, i1 - c0);
      __syncthreads();
      stage_points(P, S, c0, n);
      __syncthreads();
      if (act) eval_sources_any(P, S, n, o0 + xs[0], o1 + xs[1], o2 + xs[2], u);
    }
  }
  if (act) {
    const float csl = (float)P.csl, csrc = (float)P.csrc;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = u[q] + csl * uf[q] + csrc * uq[q];
  }
}

// L2T + W-list: one CTA of kL2tThreads per leaf, leaves in descending order
// of work (the few leaves with long W-lists start first); the leaf's
// downward density and its W-list boxes' upward densities are staged in
// batches in the leaf's frame.  A leaf of n points takes S = 1, 2, 4 or 8
// threads per point (the most with S n <= kL2tThreads); the S threads of a
// point (adjacent lanes) take every S-th staged source and are summed by
// shuffles in a fixed order.
constexpr int kL2tThreads = 256;
__global__ void __launch_bounds__(kL2tThreads) k_fast_l2t(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[kEqBatchMax];
  const int neq = eq_batch_boxes(P.ns);
  EqStage *E = reinterpret_cast<EqStage *>(smem);  // [neq ns]
  const int32_t l = P.lorder[blockIdx.x];
  if (!in_range(P, l, P.t.nleaf)) return;
  const int32_t b = P.t.leaf_box[l];
  if (!in_range(P, b, P.t.nbox)) return;
  const int d = P.t.depth[b];
  const int64_t i0 = P.t.leaf_ptr[l], i1 = P.t.leaf_ptr[l + 1];
  if (!in_range(P, i0, P.n + 1) || !in_range(P, i1, P.n + 1) || i1 <= i0) return;
  const int npts = (int)(i1 - i0);
  int S = 1;
  while (S < 8 && 2 * S * npts <= kL2tThreads) S *= 2;
  const int per_round = kL2tThreads / S;
  const int pi = threadIdx.x / S, sl = threadIdx.x % S;
  const float r = half_width(P.t, d);
  const int32_t w0 = P.t.w_ptr[b], w1 = P.t.w_ptr[b + 1];
  const int ndn = d >= kFirstDepth ? 1 : 0;
  const int neqs = ndn + (w1 - w0);
  const float csl = (float)P.csl, csrc = (float)P.csrc;
  for (int64_t p0 = i0; p0 < i1; p0 += per_round) {
    const int64_t e = p0 + pi;
    const bool act = e < i1;
    float x[3] = {0.f, 0.f, 0.f}, uf[3] = {0.f, 0.f, 0.f}, uq[3] = {0.f, 0.f, 0.f};
    if (act)
#pragma unroll
      for (int q = 0; q < 3; ++q) x[q] = P.ploc[3 * e + q];
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
      stage_eq_batch(P, E, src, nb);
      __syncthreads();
      if (act) {
        if (P.nc == 4) eval_equiv_acc<true>(E, sl, nb * P.ns, S, x[0], x[1], x[2], uf, uq);
        else eval_equiv_acc<false>(E, sl, nb * P.ns, S, x[0], x[1], x[2], uf, uq);
      }
    }
    float u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = csl * uf[q] + csrc * uq[q];
    for (int o = 1; o < S; o <<= 1)
#pragma unroll
      for (int q = 0; q < 3; ++q) u[q] += __shfl_xor_sync(kFull, u[q], o);
    if (act && sl == 0) {
      double *out = P.out + 3 * e;
#pragma unroll
      for (int a = 0; a < 3; ++a) out[a] = (P.accumulate ? out[a] : 0.0) + (double)u[a];
    }
  }
}

// Cost keys of the leaves for the L2T order (the bucket order of the
// near-field items: targets in the high word, sources in the low word).
__global__ void k_fast_l2t_keys(Pass P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < P.t.nleaf; l += stride) {
    const int32_t b = P.t.leaf_box[l];
    int64_t npts = 0, nw = 0;
    if (b >= 0 && b < P.t.nbox) {
      npts = (int64_t)P.t.leaf_ptr[l + 1] - P.t.leaf_ptr[l];
      nw = (int64_t)P.t.w_ptr[b + 1] - P.t.w_ptr[b];
    }
    const int64_t work = npts * (1 + nw);
    const uint64_t tn = work >= 4096 ? 129 : 1;  // long W-lists first
    const uint64_t ns = (uint64_t)min(work, (int64_t)0xffffffff);
    P.lkeys[l] = (tn << 32) | ns;
    P.lvals[l] = (int32_t)l;
  }
}

// Threads per CTA of the per-box kernels: the check points, rounded up to
// whole warps.
int box_threads(int ns) { return ((ns + 31) / 32) * 32; }

// Check-to-equivalent products of the nb boxes of one depth: kFastTile boxes
// per CTA, one operator row per thread.
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

  // the spectral products keep as many CTAs resident as shared memory allows
  static bool carveout_set = false;
  if (!carveout_set && fft) {
    cudaFuncSetAttribute(k_fast_kmulp<4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fast_kmulp<3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    carveout_set = true;
  }
  // set-up: octant table, first-child flags, parent list, DFT tables
  if ((err = cudaMemsetAsync(P.child8, 0xff, sizeof(int32_t) * 8 * (size_t)P.t.nbox, st)) !=
      cudaSuccess)
    return err;
  const int64_t ntab = std::max<int64_t>(P.t.nbox, fft ? (int64_t)ns * nf : 0);
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
  pre("pack");
  k_fast_pack<<<P.t.nleaf, kStageThreads, 0, st>>>(P);
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
  }
  pre("s2m");
  k_fast_s2m<<<P.t.nleaf, bt, sizeof(SrcStage) * bt, st>>>(P);
  post();
  for (int32_t d = max_depth; d >= kFirstDepth; --d) {
    P.depth = d;
    P.box0 = depth_ptr[d];
    P.box1 = depth_ptr[d + 1];
    const int32_t nb = P.box1 - P.box0;
    if (nb <= 0) continue;
    if (d < max_depth) {
      pre("m2m");
      k_fast_m2m<<<nb, bt, sizeof(EqStage) * std::min(8, eq_batch_boxes(ns)) * ns, st>>>(P);
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
    const unsigned tiles = (unsigned)((nb + kFastTile - 1) / kFastTile);
    if (fft) {
      pre("ufft");
      dim3 gu((unsigned)((nf + 127) / 128), tiles);
      if (P.nc == 4)
        k_fast_ufft<4><<<gu, 128, sizeof(float) * kFastTile * ns * 4, st>>>(P);
      else
        k_fast_ufft<3><<<gu, 128, sizeof(float) * kFastTile * ns * 3, st>>>(P);
      post();
      // parents of this depth's boxes: at most the boxes of the depth above
      const int32_t npar_max = depth_ptr[d] - depth_ptr[d - 1];
      dim3 gk((unsigned)((npar_max + kKmulThreads - 1) / kKmulThreads), (unsigned)nf);
      pre("kmulp");
      if (P.nc == 4)
        k_fast_kmulp<4><<<gk, kKmulThreads, sizeof(float) * 343 * 24, st>>>(P, depth_ptr[d],
                                                                             depth_ptr[d + 1]);
      else
        k_fast_kmulp<3><<<gk, kKmulThreads, sizeof(float) * 343 * 20, st>>>(P, depth_ptr[d],
                                                                             depth_ptr[d + 1]);
      post();
      pre("ifft");
      {
        int wc = 20480 / (ns * 8);
        wc = wc < 4 ? 4 : (wc > 32 ? 32 : wc);
        const size_t sm = sizeof(float2) * (size_t)wc * ns + sizeof(float) * kIfftBoxes * wc * 6;
        k_fast_ifft<<<(unsigned)((nb + kIfftBoxes - 1) / kIfftBoxes), 2 * bt, sm, st>>>(P, wc);
      }
      post();
    }
    pre("dchk");
    k_fast_dchk<<<nb, bt, sizeof(EqStage) * eq_batch_boxes(ns) * ns + sizeof(SrcStage) * bt, st>>>(P);
    post();
    pre("dc2e");
    launch_c2e<false>(P, nb, ns, st);
    post();
  }
  pre("l2t_order");
  k_fast_l2t_keys<<<gs(P.t.nleaf), 256, 0, st>>>(P);
  if (err == cudaSuccess) err = cudaGetLastError();
  count_launches(1);
  launch_bucket_order(P.t.nleaf, P.lkeys, P.lvals, P.lcnt, P.loff, P.lrank, P.lorder, st);
  if (err == cudaSuccess) err = cudaGetLastError();
  hk.after(seq, st);
  ++seq;
  pre("l2t");
  k_fast_l2t<<<P.t.nleaf, kL2tThreads, sizeof(EqStage) * eq_batch_boxes(ns) * ns, st>>>(P);
  post();
  return err;
}

}  // namespace fmm
}  // namespace stk
