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

// Adds the single and double layer of the staged points j0, j0 + js, ... < n
// at x.
template <bool SL, bool DL>
__device__ __forceinline__ void eval_sources(const SrcStage *S, int j0, int n, int js, float x0,
                                             float x1, float x2, float u[3]) {
  for (int i = j0; i < n; i += js) {
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

__device__ __forceinline__ void eval_sources_any(const Pass &P, const SrcStage *S, int j0, int n,
                                                 int js, float x0, float x1, float x2,
                                                 float u[3]) {
  if (P.qf && P.pf) eval_sources<true, true>(S, j0, n, js, x0, x1, x2, u);
  else if (P.qf) eval_sources<true, false>(S, j0, n, js, x0, x1, x2, u);
  else eval_sources<false, true>(S, j0, n, js, x0, x1, x2, u);
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
    if (k < P.ns) eval_sources_any(P, S, 0, n, 1, x[0], x[1], x[2], u);
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
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t wc = e / (kTcCols * kTcK);
    const int r = (int)(e % (kTcCols * kTcK));
    const int w = (int)(wc / kTcChunks), ch = (int)(wc % kTcChunks);
    const int nn = r / kTcK, k = r % kTcK;
    const int t = nn / 6, q = (nn >> 1) % 3, rn = nn & 1;
    const int sl = 4 * (ch & 1) + (k >> 3), c = (k >> 1) & 3, rk = k & 1;
    const int dd = ch >> 1, dir = dd < 13 ? dd : dd + 1;
    const int ox = 2 * (dir / 9 - 1) + (sl >> 2) - (t >> 2);
    const int oy = 2 * ((dir / 3) % 3 - 1) + ((sl >> 1) & 1) - ((t >> 1) & 1);
    const int oz = 2 * (dir % 3 - 1) + (sl & 1) - (t & 1);
    float val = 0.f;
    if (c < P.nc && !(ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1)) {
      const int oi = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
      const float *K = P.spec32 + ((size_t)w * 343 + oi) * m + (q * P.nc + c) * 2;
      val = (rk == rn) ? K[0] : (rk == 0 ? K[1] : -K[1]);
    }
    const float hi = tf32_rna(val), lo = tf32_rna(val - hi);
    float *o = P.btab + (size_t)wc * 2 * kTcCols * kTcK;
    const uint32_t off = sw128_off(nn, k) >> 2;
    o[off] = hi;
    o[kTcCols * kTcK + off] = lo;
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
// point (adjacent lanes, each taking every S-th staged source, summed by
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

// Sums u over the S adjacent lanes of a target (S a power of two <= 32).
__device__ __forceinline__ void lane_sum(float u[3], int S) {
  for (int o = 1; o < S; o <<= 1)
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] += __shfl_xor_sync(kFull, u[q], o);
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
      for (int q = 0; q < 3; ++q) u[q] = P.m2l32[((size_t)b * 3 + q) * P.ns + k];
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
      if (act) eval_sources_any(P, S, 0, n, 1, o0 + xs[0], o1 + xs[1], o2 + xs[2], u);
    }
  }
  if (act) {
    const float csl = (float)P.csl, csrc = (float)P.csrc;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      P.chk32[(size_t)b * 3 * P.ns + 3 * k + q] = u[q] + csl * uf[q] + csrc * uq[q];
  }
}

// L2T + W-list: items of the leaves (k_fast_item_counts), thread = (point,
// lane of S); the leaf's downward density and its W-list boxes' upward
// densities are staged in batches in the leaf's frame.
__global__ void __launch_bounds__(kItemThreads) k_fast_l2t(Pass P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ EqSrc src[kEqBatchMax];
  const int neq = eq_batch_boxes(P.ns);
  EqStage *E = reinterpret_cast<EqStage *>(smem);  // [neq ns]
  const int32_t it0 = 0, it1 = P.ioff[P.t.nleaf];
  const float csl = (float)P.csl, csrc = (float)P.csrc;
  for (int32_t it = it0 + blockIdx.x; it < it1; it += gridDim.x) {
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
        if (P.nc == 4) eval_equiv_acc<true>(E, sl, nb * P.ns, sw, x[0], x[1], x[2], uf, uq);
        else eval_equiv_acc<false>(E, sl, nb * P.ns, sw, x[0], x[1], x[2], uf, uq);
      }
    }
    float u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = csl * uf[q] + csrc * uq[q];
    lane_sum(u, sw);
    if (act && sl == 0) {
      double *out = P.out + 3 * e;
#pragma unroll
      for (int a = 0; a < 3; ++a) out[a] = (P.accumulate ? out[a] : 0.0) + (double)u[a];
    }
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
    const int64_t nb = (int64_t)nf * kTcChunks * kTcCols * kTcK;
    pre("btab");
    k_fast_btab<<<gs(nb), 256, 0, st>>>(P, nb);
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
    k_fast_dchk<<<nb, bt, sizeof(EqStage) * eq_batch_boxes(ns) * ns + sizeof(SrcStage) * bt, st>>>(P);
    post();
    pre("dc2e");
    launch_c2e<false>(P, nb, ns, st);
    post();
  }
  pre("l2t");
  {
    const int64_t bound = (int64_t)P.t.nleaf + (P.n + 7) / 8;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(bound, (int64_t)sms * 8));
    k_fast_l2t<<<g, kItemThreads, sizeof(EqStage) * eq_batch_boxes(ns) * ns, st>>>(P);
  }
  post();
  return err;
}

}  // namespace fmm
}  // namespace stk
