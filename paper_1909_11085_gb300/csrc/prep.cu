// prep.cu -- staging kernels around the two engines: source packing, target
// bounding box and Morton keys, a stable LSD radix sort, exclusive scans,
// work-item builders for the direct, near-field (U-list) and batched forms,
// and the final reduction/scatter into the caller's output.
#include <cfloat>

#include "common.cuh"
#include "prep.cuh"

namespace stk {

// ---------------------------------------------------------------- packing
// Mixed records: positions split hi/lo about the frame centre c = src[0]
// (in FP64: the difference is where FP32 would cancel); quadrature weight and
// kernel constant folded into the densities (q = w f / (8 pi mu), psi = w phi
// * 6 / (8 pi)) and hh = (alpha h)^2, products of the FP32-rounded factors in
// FP32 (a few FP32 ulps, against the FP64 pipe's 1/64 rate for the products).
__global__ void k_pack_mixed(int64_t ns, const double *__restrict__ src,
                             const double *__restrict__ f, const double *__restrict__ nrm,
                             const double *__restrict__ phi, const double *__restrict__ w,
                             const double *__restrict__ h, double alpha, double csl, double cdl,
                             const double *__restrict__ cen, SrcRec *__restrict__ rec) {
  const double cx = cen[0], cy = cen[1], cz = cen[2];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns;
       j += (int64_t)gridDim.x * blockDim.x) {
    SrcRec R;
    float hx, lx, hy, ly, hz, lz;
    split_hl(src[3 * j] - cx, hx, lx);
    split_hl(src[3 * j + 1] - cy, hy, ly);
    split_hl(src[3 * j + 2] - cz, hz, lz);
    float hhf = 0.f;
    if (h) {
      const float a = f64_to_f32_rn(alpha) * f64_to_f32_rn(h[j]);
      hhf = a * a;
    }
    hhf = fmaxf(fminf(hhf, FLT_MAX), FLT_MIN);
    R.yh = make_float4(hx, hy, hz, hhf);
    const float wj = w ? f64_to_f32_rn(w[j]) : 1.f;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f), nn = q, pp = q;
    if (f) {
      const float s = wj * f64_to_f32_rn(csl);
      q = make_float4(s * f64_to_f32_rn(f[3 * j]), s * f64_to_f32_rn(f[3 * j + 1]),
                      s * f64_to_f32_rn(f[3 * j + 2]), 0.f);
    }
    if (phi) {
      const float s = wj * f64_to_f32_rn(cdl);
      nn = make_float4(f64_to_f32_rn(nrm[3 * j]), f64_to_f32_rn(nrm[3 * j + 1]),
                       f64_to_f32_rn(nrm[3 * j + 2]), 0.f);
      pp = make_float4(s * f64_to_f32_rn(phi[3 * j]), s * f64_to_f32_rn(phi[3 * j + 1]),
                       s * f64_to_f32_rn(phi[3 * j + 2]), 0.f);
    }
    q.w = lx;
    nn.w = ly;
    pp.w = lz;
    R.q = q;
    R.n = nn;
    R.p = pp;
    rec[j] = R;
  }
}

__global__ void k_pack_fp64(int64_t ns, const double *__restrict__ src,
                            const double *__restrict__ f, const double *__restrict__ nrm,
                            const double *__restrict__ phi, const double *__restrict__ w,
                            double csl, double cdl, SrcRec64 *__restrict__ rec) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns;
       j += (int64_t)gridDim.x * blockDim.x) {
    SrcRec64 R;
    const double wj = w ? w[j] : 1.0;
    for (int k = 0; k < 3; ++k) {
      R.y[k] = src[3 * j + k];
      R.q[k] = f ? wj * csl * f[3 * j + k] : 0.0;
      R.n[k] = phi ? nrm[3 * j + k] : 0.0;
      R.p[k] = phi ? wj * cdl * phi[3 * j + k] : 0.0;
    }
    rec[j] = R;
  }
}

// ---------------------------------------------------------------- bbox
constexpr int kRedThreads = 256;

__global__ void k_bbox_partial(int64_t n, const double *__restrict__ pts, double *__restrict__ part) {
  __shared__ double sm[6][kRedThreads];
  double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      const double v = pts[3 * i + k];
      mn[k] = fmin(mn[k], v);
      mx[k] = fmax(mx[k], v);
    }
  for (int k = 0; k < 3; ++k) {
    sm[k][threadIdx.x] = mn[k];
    sm[3 + k][threadIdx.x] = mx[k];
  }
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 3; ++k) {
        sm[k][threadIdx.x] = fmin(sm[k][threadIdx.x], sm[k][threadIdx.x + s]);
        sm[3 + k][threadIdx.x] = fmax(sm[3 + k][threadIdx.x], sm[3 + k][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) part[6 * blockIdx.x + k] = sm[k][0];
}

__global__ void k_bbox_final(int nblk, const double *__restrict__ part, double *__restrict__ box) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double b[6] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int i = 0; i < nblk; ++i)
    for (int k = 0; k < 3; ++k) {
      b[k] = fmin(b[k], part[6 * i + k]);
      b[3 + k] = fmax(b[3 + k], part[6 * i + 3 + k]);
    }
  for (int k = 0; k < 6; ++k) box[k] = b[k];
}

// ---------------------------------------------------------------- Morton keys
__device__ __forceinline__ uint64_t spread10(uint32_t v) {
  uint64_t x = v & 0x3ffu;
  x = (x | (x << 16)) & 0x030000FFull;
  x = (x | (x << 8)) & 0x0300F00Full;
  x = (x | (x << 4)) & 0x030C30C3ull;
  x = (x | (x << 2)) & 0x09249249ull;
  return x;
}

// 30-bit Morton key of each point in the bounding box; with group_ptr the key
// is prefixed by the point's group (suspension) so that groups stay contiguous.
__global__ void k_morton(int64_t n, const double *__restrict__ pts, const double *__restrict__ box,
                         const int64_t *__restrict__ group_ptr, int32_t ngroup,
                         uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
  const double lo[3] = {box[0], box[1], box[2]};
  double ext = fmax(fmax(box[3] - box[0], box[4] - box[1]), box[5] - box[2]);
  const double inv = ext > 0.0 ? 1024.0 / (ext * (1.0 + 1e-12)) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      double v = (pts[3 * i + k] - lo[k]) * inv;
      v = fmin(fmax(v, 0.0), 1023.0);
      q[k] = (uint32_t)v;
    }
    uint64_t key = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    if (group_ptr) {
      int32_t a = 0, b = ngroup - 1;
      while (a < b) {
        const int32_t m = a + (b - a + 1) / 2;
        if (group_ptr[m] <= i) a = m;
        else b = m - 1;
      }
      key |= (uint64_t)a << 30;
    }
    keys[i] = key;
    vals[i] = (int32_t)i;
  }
}

// ---------------------------------------------------------------- scan
// Single-block exclusive scan of n int32 values; out has n + 1 entries.
// A tile is kScanThreads * kScanPer values; warp w takes kScanPer rows of 32
// consecutive values (loads and stores coalesced, all loads in flight at
// once), scans each row with shuffles and chains the rows, and the block
// scans the warps' totals.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 16;

__global__ void __launch_bounds__(kScanThreads) k_scan_excl(const int32_t *__restrict__ in,
                                                            int64_t n, int32_t *__restrict__ out,
                                                            int32_t *__restrict__ total) {
  __shared__ int32_t warp_sums[kScanThreads / kWarp];
  __shared__ int32_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += (int64_t)kScanThreads * kScanPer) {
    const int64_t w0 = base + (int64_t)wid * kWarp * kScanPer + lane;  // row k: w0 + 32 k
    int32_t v[kScanPer], x[kScanPer];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) v[k] = w0 + kWarp * k < n ? in[w0 + kWarp * k] : 0;
    int32_t run = 0;  // the warp's values before row k
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      int32_t t = v[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, t, o);
        if (lane >= o) t += y;
      }
      x[k] = run + t - v[k];  // exclusive within the warp's rows
      run += __shfl_sync(kFull, t, 31);
    }
    if (lane == 0) warp_sums[wid] = run;
    __syncthreads();
    if (wid == 0) {
      int32_t s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const int32_t carry = carry_s, before = carry + (wid > 0 ? warp_sums[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
      if (w0 + kWarp * k < n) out[w0 + kWarp * k] = before + x[k];
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + warp_sums[kScanThreads / kWarp - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[n] = carry_s;
    if (total) *total = carry_s;
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t *__restrict__ keys,
                                                             int64_t n, int shift, int nblk,
                                                             int32_t *__restrict__ hist) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: keys of equal digit keep their order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, int64_t n, int shift,
    int nblk, const int32_t *__restrict__ offs, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout) {
  __shared__ int32_t running[256];
  __shared__ int32_t cnt[kSortThreads / kWarp][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  running[threadIdx.x] = offs[(int64_t)threadIdx.x * nblk + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    for (int d = lane; d < 256; d += 32) cnt[wid][d] = 0;
    __syncthreads();
    const int64_t i = base + r * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    uint64_t key = 0;
    int32_t val = 0;
    unsigned digit = 256u + lane;  // invalid slots get unique dummy digits
    if (valid) {
      key = kin[i];
      val = vin[i];
      digit = (unsigned)((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(kFull, digit);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) cnt[wid][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      int32_t pos = running[digit] + rank;
      for (int w2 = 0; w2 < wid; ++w2) pos += cnt[w2][digit];
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    {
      int32_t s = 0;
      for (int w2 = 0; w2 < kSortThreads / kWarp; ++w2) s += cnt[w2][threadIdx.x];
      running[threadIdx.x] += s;
    }
    __syncthreads();
  }
}

size_t radix_hist_entries(int64_t n) {
  const int64_t nblk = (n + kSortTile - 1) / kSortTile;
  return (size_t)(256 * (nblk > 0 ? nblk : 1));
}

// Sorts (keys, vals) by the low `bits` bits of the keys.  Returns 0 if the
// result is in (ka, va), 1 if in (kb, vb).
int radix_sort(uint64_t *ka, int32_t *va, uint64_t *kb, int32_t *vb, int64_t n, int bits,
               int32_t *hist, int32_t *hist_scan, cudaStream_t st) {
  if (n <= 1) return 0;
  const int nblk = (int)((n + kSortTile - 1) / kSortTile);
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    uint64_t *ki = cur ? kb : ka, *ko = cur ? ka : kb;
    int32_t *vi = cur ? vb : va, *vo = cur ? va : vb;
    k_radix_hist<<<nblk, kSortThreads, 0, st>>>(ki, n, shift, nblk, hist);
    count_launches(1);
    k_scan_excl<<<1, kScanThreads, 0, st>>>(hist, (int64_t)256 * nblk, hist_scan, nullptr);
    count_launches(1);
    k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(ki, vi, n, shift, nblk, hist_scan, ko, vo);
    count_launches(1);
    cur ^= 1;
  }
  return cur;
}

// ---------------------------------------------------------------- items
// Item key for the ordering below: targets (high word) and sources (low word).
__device__ __forceinline__ uint64_t cost_key(int64_t tn, int64_t nsrc) {
  const uint64_t s = nsrc > 0xffffffffll ? 0xffffffffull : (uint64_t)(nsrc > 0 ? nsrc : 0);
  return ((uint64_t)tn << 32) | s;
}

__global__ void k_items_direct(int32_t nt, int64_t ns, int32_t nsplit, int32_t item_max,
                               Item *__restrict__ items, int64_t *__restrict__ range_ptr,
                               int32_t *__restrict__ n_items) {
  const int32_t nchunk = (nt + item_max - 1) / item_max;
  const int64_t tot = (int64_t)nchunk * nsplit;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)(i / nsplit), s = (int32_t)(i % nsplit);
    Item it;
    it.t0 = c * item_max;
    const int32_t tn = min(item_max, nt - it.t0);
    it.tn_part = tn | (s << 8);
    it.seg0 = s;
    it.seg1 = s + 1;
    items[i] = it;
  }
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g <= nsplit) range_ptr[g] = (ns * g) / nsplit;
  if (g == 0) *n_items = (int32_t)tot;
}

__global__ void k_p2p_count(int32_t nleaf, const int32_t *__restrict__ leaf_ptr, int32_t item_max,
                            int32_t *__restrict__ cnt) {
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nleaf; b += gridDim.x * blockDim.x) {
    const int32_t nb = leaf_ptr[b + 1] - leaf_ptr[b];
    cnt[b] = (nb + item_max - 1) / item_max;
  }
}

__global__ void k_p2p_emit(int32_t nleaf, const int32_t *__restrict__ leaf_ptr,
                           const int32_t *__restrict__ ulist_ptr,
                           const int32_t *__restrict__ ulist_idx, int32_t item_max,
                           const int32_t *__restrict__ offs, Item *__restrict__ items,
                           uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nleaf; b += gridDim.x * blockDim.x) {
    const int32_t nb = leaf_ptr[b + 1] - leaf_ptr[b];
    if (nb <= 0) continue;
    int64_t nsrc = 0;
    for (int32_t e = ulist_ptr[b]; e < ulist_ptr[b + 1]; ++e) {
      const int32_t a = ulist_idx[e];
      nsrc += leaf_ptr[a + 1] - leaf_ptr[a];
    }
    const int32_t nc = (nb + item_max - 1) / item_max;
    const int32_t base = nb / nc, extra = nb % nc;
    int32_t t0 = leaf_ptr[b];
    for (int32_t c = 0; c < nc; ++c) {
      const int32_t tn = base + (c < extra ? 1 : 0);
      const int32_t id = offs[b] + c;
      Item it;
      it.t0 = t0;
      it.tn_part = tn;
      it.seg0 = ulist_ptr[b];
      it.seg1 = ulist_ptr[b + 1];
      items[id] = it;
      keys[id] = cost_key(tn, nsrc);
      vals[id] = id;
      t0 += tn;
    }
  }
}

__global__ void k_batched_count(int32_t nsusp, const int64_t *__restrict__ susp_ptr,
                                int32_t item_max, int32_t *__restrict__ cnt) {
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsusp; s += gridDim.x * blockDim.x) {
    const int64_t ns = susp_ptr[s + 1] - susp_ptr[s];
    cnt[s] = (int32_t)((ns + item_max - 1) / item_max);
  }
}

__global__ void k_batched_emit(int32_t nsusp, const int64_t *__restrict__ susp_ptr,
                               const int64_t *__restrict__ n_cell, int32_t item_max,
                               const int32_t *__restrict__ offs,
                               Item *__restrict__ items, int64_t *__restrict__ range_ptr,
                               uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nsusp; s += gridDim.x * blockDim.x) {
    const int64_t p0 = susp_ptr[s], p1 = susp_ptr[s + 1];
    range_ptr[2 * s] = p0;
    range_ptr[2 * s + 1] = p0 + n_cell[s];
    if (s == nsusp - 1) range_ptr[2 * nsusp] = p1;
    const int64_t nb = p1 - p0;
    if (nb <= 0) continue;
    const int32_t nc = (int32_t)((nb + item_max - 1) / item_max);
    const int64_t base = nb / nc, extra = nb % nc;
    int64_t t0 = p0;
    for (int32_t c = 0; c < nc; ++c) {
      const int32_t tn = (int32_t)(base + (c < extra ? 1 : 0));
      const int32_t id = offs[s] + c;
      Item it;
      it.t0 = (int32_t)t0;
      it.tn_part = tn;
      it.seg0 = 2 * s;
      it.seg1 = 2 * s + 2;
      items[id] = it;
      keys[id] = cost_key(tn, nb);
      vals[id] = id;
      t0 += tn;
    }
  }
}

// ---------------------------------------------------------------- item order
// Items are ordered by a counting sort on 256 buckets: 16 classes of target
// count (8 targets wide, most targets first), each split into 16 half-octave
// classes of source count (most sources first).  So the longest items start
// first (for the persistent queues) and items with the same lane layout --
// the same engine code -- run together, which keeps the engine's hot loops
// few at a time in the instruction cache.  Items of one bucket keep their
// order of arrival, which differs between runs; that only changes which warp
// runs which item, never a result (every item computes its targets' sums on
// its own, in a fixed order).
__device__ __forceinline__ int cost_bucket(uint64_t key) {
  const uint32_t tn = (uint32_t)(key >> 32), ns = (uint32_t)key;
  const int cls = tn > 128u ? 15 : (int)((tn > 0 ? tn - 1 : 0) / 8u);
  int lv = 0;
  if (ns > 0) {
    const int msb = 31 - __clz(ns);
    lv = 2 * msb + (msb > 0 ? (int)((ns >> (msb - 1)) & 1u) : 0) - 12;  // 2 log2(ns) - 12
    lv = lv < 0 ? 0 : (lv > 15 ? 15 : lv);
  }
  return (15 - cls) * 16 + (15 - lv);
}

__global__ void k_bucket_rank(int64_t n, const uint64_t *__restrict__ keys,
                              const int32_t *__restrict__ vals, int32_t *__restrict__ cnt,
                              int32_t *__restrict__ rank) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (vals[i] >= 0) rank[i] = atomicAdd(&cnt[cost_bucket(keys[i])], 1);
}

__global__ void k_bucket_offsets(const int32_t *__restrict__ cnt, int32_t *__restrict__ off) {
  __shared__ int32_t s[256];
  const int t = threadIdx.x;
  s[t] = cnt[t];
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int32_t v = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  off[t] = s[t] - cnt[t];
}

__global__ void k_bucket_scatter(int64_t n, const uint64_t *__restrict__ keys,
                                 const int32_t *__restrict__ vals, const int32_t *__restrict__ off,
                                 const int32_t *__restrict__ rank, int32_t *__restrict__ order) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (vals[i] >= 0) order[off[cost_bucket(keys[i])] + rank[i]] = vals[i];
}

// ---------------------------------------------------------------- finish
// out[perm[i]] (+)= sum over parts of part_out[p][i], parts added in order.
__global__ void k_finish(int64_t nt, int32_t nparts, const double *__restrict__ part_out,
                         const int32_t *__restrict__ tperm, int32_t accumulate,
                         double *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int32_t p = 0; p < nparts; ++p)
      for (int k = 0; k < 3; ++k) v[k] += part_out[((size_t)p * nt + i) * 3 + k];
    const int64_t ci = tperm ? tperm[i] : i;
    for (int k = 0; k < 3; ++k) {
      double *o = out + 3 * ci + k;
      *o = accumulate ? *o + v[k] : v[k];
    }
  }
}

__global__ void k_zero_ints(int32_t *p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0;
}

// ---------------------------------------------------------------- launchers
static thread_local int64_t t_launches = 0;
int64_t launch_count() { return t_launches; }
void count_launches(int n) { t_launches += n; }

static int grid_for(int64_t n, int threads, int cap = 4096) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

void launch_pack_mixed(int64_t ns, const double *src, const double *f, const double *nrm,
                       const double *phi, const double *w, const double *h, double alpha,
                       double csl, double cdl, const double *cen, SrcRec *rec, cudaStream_t st) {
  k_pack_mixed<<<grid_for(ns, 256), 256, 0, st>>>(ns, src, f, nrm, phi, w, h, alpha, csl, cdl,
                                                  cen ? cen : src, rec);
  count_launches(1);
}

void launch_pack_fp64(int64_t ns, const double *src, const double *f, const double *nrm,
                      const double *phi, const double *w, double csl, double cdl, SrcRec64 *rec,
                      cudaStream_t st) {
  k_pack_fp64<<<grid_for(ns, 256), 256, 0, st>>>(ns, src, f, nrm, phi, w, csl, cdl, rec);
  count_launches(1);
}

int bbox_partial_blocks(int64_t n) { return grid_for(n, kRedThreads, 1024); }

void launch_bbox(int64_t n, const double *pts, double *partial, double *box, cudaStream_t st) {
  const int nb = bbox_partial_blocks(n);
  k_bbox_partial<<<nb, kRedThreads, 0, st>>>(n, pts, partial);
  count_launches(1);
  k_bbox_final<<<1, 32, 0, st>>>(nb, partial, box);
  count_launches(1);
}

void launch_morton(int64_t n, const double *pts, const double *box, const int64_t *group_ptr,
                   int32_t ngroup, uint64_t *keys, int32_t *vals, cudaStream_t st) {
  k_morton<<<grid_for(n, 256), 256, 0, st>>>(n, pts, box, group_ptr, ngroup, keys, vals);
  count_launches(1);
}

void launch_scan(const int32_t *in, int64_t n, int32_t *out, int32_t *total, cudaStream_t st) {
  k_scan_excl<<<1, kScanThreads, 0, st>>>(in, n, out, total);
  count_launches(1);
}

void launch_items_direct(int32_t nt, int64_t ns, int32_t nsplit, int32_t item_max, Item *items,
                         int64_t *range_ptr, int32_t *n_items, cudaStream_t st) {
  const int64_t tot = (int64_t)((nt + item_max - 1) / item_max) * nsplit;
  const int64_t need = tot > nsplit + 1 ? tot : nsplit + 1;
  k_items_direct<<<grid_for(need, 256), 256, 0, st>>>(nt, ns, nsplit, item_max, items, range_ptr,
                                                      n_items);
  count_launches(1);
}

void launch_p2p_items(int32_t nleaf, const int32_t *leaf_ptr, const int32_t *ulist_ptr,
                      const int32_t *ulist_idx, int32_t item_max, int32_t *cnt, int32_t *offs,
                      int32_t *n_items, Item *items, uint64_t *keys, int32_t *vals,
                      cudaStream_t st) {
  k_p2p_count<<<grid_for(nleaf, 256), 256, 0, st>>>(nleaf, leaf_ptr, item_max, cnt);
  count_launches(1);
  k_scan_excl<<<1, kScanThreads, 0, st>>>(cnt, nleaf, offs, n_items);
  count_launches(1);
  k_p2p_emit<<<grid_for(nleaf, 128), 128, 0, st>>>(nleaf, leaf_ptr, ulist_ptr, ulist_idx, item_max,
                                                   offs, items, keys, vals);
  count_launches(1);
}

void launch_batched_items(int32_t nsusp, const int64_t *susp_ptr, const int64_t *n_cell,
                          int32_t item_max, int32_t *cnt, int32_t *offs, int32_t *n_items,
                          Item *items, int64_t *range_ptr, uint64_t *keys, int32_t *vals,
                          cudaStream_t st) {
  k_batched_count<<<grid_for(nsusp, 256), 256, 0, st>>>(nsusp, susp_ptr, item_max, cnt);
  count_launches(1);
  k_scan_excl<<<1, kScanThreads, 0, st>>>(cnt, nsusp, offs, n_items);
  count_launches(1);
  k_batched_emit<<<grid_for(nsusp, 128), 128, 0, st>>>(nsusp, susp_ptr, n_cell, item_max, offs,
                                                       items, range_ptr, keys, vals);
  count_launches(1);
}

void launch_bucket_order(int64_t n, const uint64_t *keys, const int32_t *vals, int32_t *cnt,
                         int32_t *off, int32_t *rank, int32_t *order, cudaStream_t st) {
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 256, st);
  k_bucket_rank<<<grid_for(n, 256), 256, 0, st>>>(n, keys, vals, cnt, rank);
  k_bucket_offsets<<<1, 256, 0, st>>>(cnt, off);
  k_bucket_scatter<<<grid_for(n, 256), 256, 0, st>>>(n, keys, vals, off, rank, order);
  count_launches(3);
}

void launch_finish(int64_t nt, int32_t nparts, const double *part_out, const int32_t *tperm,
                   int32_t accumulate, double *out, cudaStream_t st) {
  k_finish<<<grid_for(nt, 256), 256, 0, st>>>(nt, nparts, part_out, tperm, accumulate, out);
  count_launches(1);
}

void launch_zero_ints(int32_t *p, int n, cudaStream_t st) {
  k_zero_ints<<<(n + 127) / 128, 128, 0, st>>>(p, n);
  count_launches(1);
}

}  // namespace stk

namespace stk {
__global__ void k_widen(int64_t n, const int32_t *__restrict__ in, int64_t *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}
void launch_widen(int64_t n, const int32_t *in, int64_t *out, cudaStream_t st) {
  k_widen<<<grid_for(n, 256), 256, 0, st>>>(n, in, out);
  count_launches(1);
}
}  // namespace stk
