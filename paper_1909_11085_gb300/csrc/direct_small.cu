// direct_small.cu -- small direct sums (Eq. "sl_stokes" and the double-layer
// kernel of Sec. 2.1) in one launch, for the mixed form with
// default options when targets x sources is small (kSmallPairs): no pack, no
// Morton sort, no items, no separate near-pair pass.
//
// Grid: blocks of 256 targets (two per thread, sharing every staged source) x
// source splits (split y holds sources y, y + nsplit, ...: near pairs, which
// cluster where sources and targets share a region, spread evenly over the
// CTAs).  A CTA stages its split's sources 128 at a time in shared
// memory, two by two (eight float4 per pair, read as broadcasts): positions
// hi/lo relative to the CTA's origin (its first target), so that
// d = (x_h - y_h) + (x_l - y_l) is accurate relative to |x - y| wherever the
// targets lie; q = w f / (8 pi mu) and psi = 6 w phi / (8 pi) in FP32;
// (alpha h_j)^2.  A pair with |r|^2 <= (alpha h_j)^2 (exactly coincident
// pairs included) takes the FP64 difference and 1/|r| (near_contrib): each
// warp queues them in shared memory and evaluates them 32 at a time, one per
// lane, since GB300's FP64 pipe is only fed efficiently by full warps; the
// values of one target are added in queue order (deterministic).  The FP32
// pairs run packed (two staged sources per instruction).  Each thread sums a
// tile of 128 sources in FP32 and two-sums the tile into (hi, lo); the
// split's (hi, lo) goes to part[split][target], and the last split of a
// target block to finish (a counter per block) adds the splits in order
// (FP32 two-sum, one conversion to FP64 at the end) and writes out
// (deterministic, no second launch and no waiting).
#include "common.cuh"
#include "prep.cuh"

namespace stk {

namespace {

constexpr int kSmallThreads = 128;

struct SmallArgs {
  const double *src, *f, *nrm, *phi, *w, *h, *trg;
  int64_t ns, nt;
  double alpha, csl, cdl;
  int32_t nsplit;
  int32_t accumulate;
  float2 *part;     // [nsplit][nt][3]: a split's compensated sum (hi, lo)
  int32_t *blocks;  // per target block: splits done (zero before the launch)
  double *out;      // [nt][3]
};

constexpr int kSmallT = 2;  // targets per thread
constexpr int kSmallBlock = kSmallThreads * kSmallT;
constexpr int kSmallPairsPerTile = kSmallThreads / 2;
static_assert(kSmallT == 2, "the near-pair queue encodes the target slot in 6 bits");

// Staged sources, two by two (halves interleaved) in 8 float4 fields per pair:
//   0: -yh.x, -yh.y   1: -yh.z, (alpha h)^2   2: -yl.x, -yl.y   3: -yl.z, q.x
//   4: q.y, q.z       5: n.x, n.y             6: n.z, psi.x     7: psi.y, psi.z
// each entry a (first, second) pair.
constexpr int kSmallFields = 8;

__device__ __forceinline__ float2 s_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 s_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 s_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 s_lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 s_hi(float4 v) { return make_float2(v.z, v.w); }

// One staged source pair against one target (coordinates hi/lo, each
// duplicated into both halves): the FP32 sum into u (per half), and in near
// the halves whose pair is near or coincident (left out of u, queued for FP64).
template <int KIND>
__device__ __forceinline__ void small_pair(const float4 (&s)[kSmallFields], const float2 (&xh)[3],
                                           const float2 (&xl)[3], float2 (&u)[3],
                                           unsigned &near) {
  const float2 d0 = s_add(s_add(xh[0], s_lo(s[0])), s_add(xl[0], s_lo(s[2])));
  const float2 d1 = s_add(s_add(xh[1], s_hi(s[0])), s_add(xl[1], s_hi(s[2])));
  const float2 d2 = s_add(s_add(xh[2], s_lo(s[1])), s_add(xl[2], s_lo(s[3])));
  float2 r2 = s_fma(d0, d0, s_fma(d1, d1, s_mul(d2, d2)));
  const float2 hh = s_hi(s[1]);
  near = (r2.x > hh.x ? 0u : 1u) | (r2.y > hh.y ? 0u : 2u);
  // a near half: rsqrt(+inf) = 0 takes it out of the FP32 sum
  if (near & 1u) r2.x = __int_as_float(0x7f800000);
  if (near & 2u) r2.y = __int_as_float(0x7f800000);
  const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y)), ri2 = s_mul(ri, ri);
  const float2 qx = s_hi(s[3]), qy = s_lo(s[4]), qz = s_hi(s[4]);
  const float2 nx = s_lo(s[5]), ny = s_hi(s[5]), nz = s_lo(s[6]);
  const float2 px = s_hi(s[6]), py = s_lo(s[7]), pz = s_hi(s[7]);
  if (KIND == K_SL) {
    const float2 c = s_mul(s_fma(d0, qx, s_fma(d1, qy, s_mul(d2, qz))), ri2);
    u[0] = s_fma(s_fma(d0, c, qx), ri, u[0]);
    u[1] = s_fma(s_fma(d1, c, qy), ri, u[1]);
    u[2] = s_fma(s_fma(d2, c, qz), ri, u[2]);
  } else if (KIND == K_DL) {
    const float2 dp = s_fma(d0, px, s_fma(d1, py, s_mul(d2, pz)));
    const float2 dn = s_fma(d0, nx, s_fma(d1, ny, s_mul(d2, nz)));
    const float2 c = s_mul(s_mul(dp, dn), s_mul(s_mul(ri2, ri2), ri));
    u[0] = s_fma(d0, c, u[0]);
    u[1] = s_fma(d1, c, u[1]);
    u[2] = s_fma(d2, c, u[2]);
  } else {
    const float2 dq = s_fma(d0, qx, s_fma(d1, qy, s_mul(d2, qz)));
    const float2 dp = s_fma(d0, px, s_fma(d1, py, s_mul(d2, pz)));
    const float2 dn = s_fma(d0, nx, s_fma(d1, ny, s_mul(d2, nz)));
    const float2 c = s_mul(s_fma(s_mul(dp, dn), ri2, dq), ri2);
    u[0] = s_fma(s_fma(d0, c, qx), ri, u[0]);
    u[1] = s_fma(s_fma(d1, c, qy), ri, u[1]);
    u[2] = s_fma(s_fma(d2, c, qz), ri, u[2]);
  }
}

constexpr int kSmallQueue = 256;  // near pairs queued per warp (>= 128 free before a pair)

// A warp's shared scratch for evaluating its queued near pairs.
struct SmallNear {
  int32_t queue[kSmallQueue];  // source within the staged tile | target slot << 8
  float val[32][3];            // one round's values, by lane
  float tot[32 * kSmallT][3];  // one round's sums, by target slot (zero between rounds)
};

// Evaluates a warp's queued near pairs, one per lane, with the FP64
// difference and 1/|r| (near_contrib), and adds them to the near sums un of
// the lanes owning their targets.  In each round the lanes of one target
// (found with match_any) are summed in queue order by the group's first lane;
// the owner then adds the round's sum: the order is fixed, so the result is
// deterministic.  t0: the warp's first target (slot s is target t0 + s);
// staged source j is source c0 + cs j.
template <int KIND>
__device__ __forceinline__ void small_flush(SmallNear &sn, int qn,
                                            const float4 (*S)[kSmallFields], const double *src,
                                            const double *trg, int64_t c0, int64_t cs, int64_t t0,
                                            int lane,
                                            float (&un)[kSmallT][3]) {
  for (int e0 = 0; e0 < qn; e0 += 32) {
    const int e = e0 + lane;
    int slot = -1 - lane;  // idle lanes: keys of their own
    float c[3] = {0.f, 0.f, 0.f};
    if (e < qn) {
      const int32_t ent = sn.queue[e];
      const int j = ent & 0xff;
      slot = ent >> 8;
      const float *F = reinterpret_cast<const float *>(S[j >> 1]);
      const int h = j & 1;
      const float4 qq = make_float4(F[14 + h], F[16 + h], F[18 + h], 0.f);
      const float4 nn = make_float4(F[20 + h], F[22 + h], F[24 + h], 0.f);
      const float4 pp = make_float4(F[26 + h], F[28 + h], F[30 + h], 0.f);
      if (!near_contrib(trg + 3 * (t0 + slot), src + 3 * (c0 + cs * j), qq, nn, pp, KIND, c))
        c[0] = c[1] = c[2] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) sn.val[lane][q] = c[q];
    const unsigned grp = __match_any_sync(kFull, slot);
    __syncwarp();
    if (slot >= 0 && lane == __ffs(grp) - 1) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float v = 0.f;
        for (unsigned m = grp; m; m &= m - 1) v += sn.val[__ffs(m) - 1][q];
        sn.tot[slot][q] = v;
      }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kSmallT; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        un[k][q] += sn.tot[lane + 32 * k][q];
        sn.tot[lane + 32 * k][q] = 0.f;
      }
    __syncwarp();
  }
}

template <int KIND>
__global__ void __launch_bounds__(kSmallThreads) k_direct_small(SmallArgs a) {
  __shared__ float4 S[kSmallPairsPerTile][kSmallFields];
  __shared__ SmallNear near_all[kSmallThreads / 32];
  __shared__ int last;
  const int tid = threadIdx.x, lane = tid & 31;
  SmallNear &sn = near_all[tid >> 5];
  int32_t *queue = sn.queue;
#pragma unroll
  for (int k = 0; k < kSmallT; ++k)
#pragma unroll
    for (int q = 0; q < 3; ++q) sn.tot[lane + 32 * k][q] = 0.f;
  const unsigned lt = (1u << lane) - 1u;
  // a thread's targets: lane + 32 k of its warp's 64 (k < kSmallT)
  const int64_t tb = (int64_t)blockIdx.x * kSmallBlock;
  const int64_t t0 = tb + (int64_t)(tid >> 5) * 32 * kSmallT;
  const int y = blockIdx.y;
  // the split's sources: y, y + nsplit, y + 2 nsplit, ... (strided, so that
  // the near pairs, which cluster where sources and targets share a region,
  // spread over all splits instead of loading a few CTAs of the one wave)
  const int64_t cnt = (a.ns - y + a.nsplit - 1) / a.nsplit;
  // the CTA's origin: its first target
  const double oo[3] = {a.trg[3 * tb], a.trg[3 * tb + 1], a.trg[3 * tb + 2]};
  float2 xh[kSmallT][3], xl[kSmallT][3];
  float hi[kSmallT][3], lo[kSmallT][3];
  bool act[kSmallT];
#pragma unroll
  for (int k = 0; k < kSmallT; ++k) {
    const int64_t t = t0 + 32 * k + lane;
    act[k] = t < a.nt;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double xq = act[k] ? a.trg[3 * t + q] : oo[q];
      float vh, vl;
      split_hl(xq - oo[q], vh, vl);
      xh[k][q] = make_float2(vh, vh);
      xl[k][q] = make_float2(vl, vl);
      hi[k][q] = lo[k][q] = 0.f;
    }
  }
  for (int64_t i0 = 0; i0 < cnt; i0 += kSmallThreads) {
    const int n = (int)min((int64_t)kSmallThreads, cnt - i0), np = (n + 1) / 2;
    const int64_t c0 = y + (int64_t)a.nsplit * i0;  // staged source k is c0 + nsplit k
    __syncthreads();
    {  // source c0 + nsplit tid into half tid & 1 of pair tid / 2 (a missing one: far,
       // zero strength)
      float v[16];
      if (tid < n) {
        const int64_t j = c0 + (int64_t)a.nsplit * tid;
        float vh[3], vl[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) split_hl(a.src[3 * j + q] - oo[q], vh[q], vl[q]);
        double hh = 0.0;
        if (a.h) {
          const double al = a.alpha * a.h[j];
          hh = al * al;
        }
        const double wj = a.w ? a.w[j] : 1.0, ws = wj * a.csl, wd = wj * a.cdl;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          v[q] = -vh[q];
          v[4 + q] = -vl[q];
          v[7 + q] = (KIND & K_SL) ? f64_to_f32_rn(ws * a.f[3 * j + q]) : 0.f;
          v[10 + q] = (KIND & K_DL) ? f64_to_f32_rn(a.nrm[3 * j + q]) : 0.f;
          v[13 + q] = (KIND & K_DL) ? f64_to_f32_rn(wd * a.phi[3 * j + q]) : 0.f;
        }
        v[3] = fminf(f64_to_f32_rn(hh), 3.0e38f);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
        v[0] = v[1] = v[2] = -1e18f;  // far away
      }
      if (tid < 2 * np) {
        // quantity i of the field layout (yh.x yh.y yh.z hh yl.x yl.y yl.z q.x q.y q.z
        // n.x n.y n.z psi.x psi.y psi.z) at float 2 i + half
        float *F = reinterpret_cast<float *>(S[tid >> 1]);
        const int h = tid & 1;
#pragma unroll
        for (int i = 0; i < 16; ++i) F[2 * i + h] = v[i];
      }
    }
    __syncthreads();
    float2 u[kSmallT][3];
    float un[kSmallT][3];
#pragma unroll
    for (int k = 0; k < kSmallT; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        u[k][q] = make_float2(0.f, 0.f);
        un[k][q] = 0.f;
      }
    int qn = 0;
    for (int p = 0; p < np; ++p) {
      float4 s[kSmallFields];
#pragma unroll
      for (int f = 0; f < kSmallFields; ++f) s[f] = S[p][f];
      unsigned nr[kSmallT];
#pragma unroll
      for (int k = 0; k < kSmallT; ++k) {
        small_pair<KIND>(s, xh[k], xl[k], u[k], nr[k]);
        if (!act[k]) nr[k] = 0u;
      }
      if (__any_sync(kFull, (nr[0] | nr[1]) != 0u)) {
        // queue order: by target slot and half, then by lane
#pragma unroll
        for (int k = 0; k < kSmallT; ++k)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const bool b = (nr[k] >> h) & 1u;
            const unsigned m = __ballot_sync(kFull, b);
            if (b) queue[qn + __popc(m & lt)] = (2 * p + h) | ((lane + 32 * k) << 8);
            qn += __popc(m);
          }
        if (qn > kSmallQueue - 32 * 2 * kSmallT) {
          __syncwarp();
          small_flush<KIND>(sn, qn, S, a.src, a.trg, c0, a.nsplit, t0, lane, un);
          qn = 0;
          __syncwarp();
        }
      }
    }
    __syncwarp();
    if (qn) small_flush<KIND>(sn, qn, S, a.src, a.trg, c0, a.nsplit, t0, lane, un);
#pragma unroll
    for (int k = 0; k < kSmallT; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        two_sum_acc(hi[k][q], lo[k][q], u[k][q].x + u[k][q].y);
        two_sum_acc(hi[k][q], lo[k][q], un[k][q]);
      }
  }
#pragma unroll
  for (int k = 0; k < kSmallT; ++k) {
    const int64_t t = t0 + 32 * k + lane;
    if (!act[k]) continue;
    float2 *o = a.part + ((size_t)y * (size_t)a.nt + (size_t)t) * 3;
#pragma unroll
    for (int q = 0; q < 3; ++q) o[q] = make_float2(hi[k][q], lo[k][q]);
  }
  // the last split of this target block to finish adds the splits in order
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&a.blocks[blockIdx.x], 1) == a.nsplit - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the block's partials of one split are 3 x 256 contiguous (hi, lo) pairs:
  // each thread sums 6 of those values over the splits (from L2, written by
  // the other CTAs before their fence; loads of 5 splits in flight), in split
  // order, two-summing the hi parts and adding the lo parts
  constexpr int kPer = 3 * kSmallBlock / kSmallThreads;
  const int64_t v0 = 3 * tb, vend = 3 * min(tb + (int64_t)kSmallBlock, a.nt);
  float sh[kPer], sl[kPer];
#pragma unroll
  for (int m = 0; m < kPer; ++m) sh[m] = sl[m] = 0.f;
  for (int y0 = 0; y0 < a.nsplit; y0 += 5) {
    float2 v[5][kPer];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int m = 0; m < kPer; ++m) {
        const int64_t e = v0 + tid + kSmallThreads * m;
        v[i][m] = (y0 + i < a.nsplit && e < vend)
                      ? __ldcg(a.part + (size_t)(y0 + i) * (size_t)a.nt * 3 + (size_t)e)
                      : make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int m = 0; m < kPer; ++m) {
        two_sum_acc(sh[m], sl[m], v[i][m].x);
        sl[m] += v[i][m].y;
      }
  }
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int64_t e = v0 + tid + kSmallThreads * m;
    if (e < vend) a.out[e] = (a.accumulate ? a.out[e] : 0.0) + ((double)sh[m] + (double)sl[m]);
  }
  if (tid == 0) a.blocks[blockIdx.x] = 0;  // ready for the next call
}
}  // namespace

int64_t direct_small_blocks(int64_t nt) { return (nt + kSmallBlock - 1) / kSmallBlock; }

int direct_small_splits(int64_t ns, int64_t nt, int sms) {
  const int64_t blocks = direct_small_blocks(nt);
  if (blocks <= 0) return 1;
  // one wave: as many splits as the resident CTAs allow (a second, partial
  // wave would double the time)
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_direct_small<K_SLDL>, kSmallThreads,
                                                    0) != cudaSuccess ||
      occ < 1)
    occ = 1;
  int64_t s = (int64_t)occ * sms / blocks;
  const int64_t cap = ns / 64 > 1 ? ns / 64 : 1;  // at least 64 sources per split
  if (s > cap) s = cap;
  if (s > 64) s = 64;
  if (s < 1) s = 1;
  return (int)s;
}

cudaError_t launch_direct_small(int kinds, const double *src, const double *f, const double *nrm,
                                const double *phi, const double *w, const double *h, int64_t ns,
                                const double *trg, int64_t nt, double alpha, double csl,
                                double cdl, int32_t nsplit, int32_t accumulate, double *part,
                                int32_t *blocks, double *out, cudaStream_t st) {
  SmallArgs a{src, f, nrm, phi, w, h, trg, ns, nt, alpha, csl, cdl, nsplit, accumulate,
              reinterpret_cast<float2 *>(part), blocks, out};
  const dim3 grid((unsigned)direct_small_blocks(nt), (unsigned)nsplit);
  if (kinds == K_SL)
    k_direct_small<K_SL><<<grid, kSmallThreads, 0, st>>>(a);
  else if (kinds == K_DL)
    k_direct_small<K_DL><<<grid, kSmallThreads, 0, st>>>(a);
  else
    k_direct_small<K_SLDL><<<grid, kSmallThreads, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stk
