// near.cu -- the near pairs of the mixed-precision sums (Eq. "sl_stokes" and
// the double-layer kernel of Sec. 2.1, summed as in Sec. 3.1).
//
// The mixed engine leaves out of its FP32 sums every candidate pair with
// |r| < alpha h_j, where FP32 cancellation in x - y would dominate the error.
// This kernel adds exactly those pairs back, with the difference x - y and
// 1/|r| in FP64 (near_contrib).  It walks the same work items as the engine
// and takes the same decisions with the same arithmetic (frame_origin,
// local_coord, box_dist2, pair_r2 in common.cuh), so every pair is summed by
// exactly one of the two kernels.
//
// One warp per item, persistent, items in the engine's cost order:
//  1. the item's targets (lane + 32 t) in the item's local frame;
//  2. its sources, 32 at a time: local coordinates and the box test; each
//     candidate is broadcast and every lane tests its targets;
//  3. near pairs go to a queue in shared memory in a fixed order; a full
//     queue is evaluated one pair per lane (the FP64 pipe of GB300 runs at
//     1/64 of the FP32 rate, so it is only ever fed full warps), and the
//     values are added per target in queue order (compensated FP32), which
//     makes the result independent of scheduling;
//  4. the item's sums are added to its targets' partial results.
// The self pair (target and source are the same caller point) contributes
// nothing and is not queued.
#include "common.cuh"
#include "prep.cuh"

namespace stk {

namespace {

constexpr int kNearWarps = 4;
constexpr int kNearT = kItemMax / kWarp;  // targets per lane
constexpr int kNearQueue = 256;           // >= 128 free slots before each candidate

struct __align__(16) NearSmem {
  float sv[kWarp][3];           // values of one round of evaluations
  float acc[2][3][kItemMax];    // per-target compensated sums (hi, lo)
  int32_t qj[kNearQueue];       // queued pair: source index | kind << 30
  uint8_t qt[kNearQueue];       //   target within the item
};

__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Evaluates the queued pairs, one per lane per round, and adds each value to
// its target's sum; pairs of one target are added in queue order.
__device__ void eval_queue(NearSmem &sm, const EngineParams &P, int32_t t0, int qn, int lane) {
  for (int e0 = 0; e0 < qn; e0 += kWarp) {
    const int e = e0 + lane;
    const bool act = e < qn;
    float v[3] = {0.f, 0.f, 0.f};
    int li = -1 - lane;  // idle lanes get keys of their own
    if (act) {
      li = sm.qt[e];
      const uint32_t jj = (uint32_t)sm.qj[e];
      const int64_t j = jj & 0x3fffffffu;
      const int32_t gi = t0 + li;
      const int64_t ci = P.tperm ? P.tperm[gi] : gi;
      const SrcRec r = P.rec[j];
      if (!near_contrib(P.trg64 + 3 * ci, P.src64 + 3 * j, r.q, r.n, r.p, (int)(jj >> 30), v))
        v[0] = v[1] = v[2] = 0.f;
    }
    sm.sv[lane][0] = v[0];
    sm.sv[lane][1] = v[1];
    sm.sv[lane][2] = v[2];
    const unsigned grp = __match_any_sync(kFull, li);
    __syncwarp();
    if (act && lane == __ffs(grp) - 1) {  // the group's first lane adds its members in order
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float h = sm.acc[0][k][li], l = sm.acc[1][k][li];
        for (unsigned m = grp; m; m &= m - 1) two_sum_acc(h, l, sm.sv[__ffs(m) - 1][k]);
        sm.acc[0][k][li] = h;
        sm.acc[1][k][li] = l;
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kNearWarps *kWarp) k_near(EngineParams P) {
  __shared__ NearSmem smem[kNearWarps];
  NearSmem &sm = smem[threadIdx.x / kWarp];
  const int lane = threadIdx.x & (kWarp - 1);
  const unsigned lt = (1u << lane) - 1u;
  const int n_items = *P.n_items;
  const double cc[3] = {P.src64[0], P.src64[1], P.src64[2]};
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(P.near_counter, 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= n_items) break;
    const Item it = P.items[P.item_order ? P.item_order[idx] : idx];
    const int tn = it.tn_part & 0xFF, part = it.tn_part >> 8;

    // 1. targets and the item frame, as the engine builds them
    const int64_t c0 = P.tperm ? P.tperm[it.t0] : it.t0;
    const double x0[3] = {P.trg64[3 * c0], P.trg64[3 * c0 + 1], P.trg64[3 * c0 + 2]};
    bool valid[kNearT];
    int64_t ci[kNearT];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int t = 0; t < kNearT; ++t) {
      const int li = lane + kWarp * t;
      valid[t] = li < tn;
      ci[t] = -1;
      if (valid[t]) {
        const int32_t gi = it.t0 + li;
        ci[t] = P.tperm ? P.tperm[gi] : gi;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float rk = __double2float_rn(P.trg64[3 * ci[t] + k] - x0[k]);
          mn[k] = fminf(mn[k], rk);
          mx[k] = fmaxf(mx[k], rk);
        }
      }
    }
    float oh[3], ol[3], blo[3], bhi[3], x[kNearT][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) frame_origin(x0[k], warp_min_f(mn[k]), warp_max_f(mx[k]), cc[k], oh[k], ol[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      blo[k] = INFINITY;
      bhi[k] = -INFINITY;
    }
#pragma unroll
    for (int t = 0; t < kNearT; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        x[t][k] = 1e30f;
        if (valid[t]) {
          x[t][k] = local_coord(P.trg64[3 * ci[t] + k], cc[k], oh[k], ol[k]);
          blo[k] = fminf(blo[k], x[t][k]);
          bhi[k] = fmaxf(bhi[k], x[t][k]);
        }
      }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      blo[k] = warp_min_f(blo[k]);
      bhi[k] = warp_max_f(bhi[k]);
    }
    for (int li = lane; li < tn; li += kWarp)
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.acc[0][k][li] = sm.acc[1][k][li] = 0.f;
    __syncwarp();

    // 2./3. sources: box test, per-pair test of the candidates, queue
    int qn = 0;
    for (int32_t e = it.seg0; e < it.seg1; ++e) {
      const int32_t sid = P.seg_list ? P.seg_list[e] : e;
      const int64_t s0 = P.range_ptr[sid], s1 = P.range_ptr[sid + 1];
      const uint32_t kind_bits = (uint32_t)seg_kind(P, sid) << 30;
      for (int64_t j0 = s0; j0 < s1; j0 += kWarp) {
        const int64_t j = j0 + lane;
        float y[3] = {0.f, 0.f, 0.f}, hh = 0.f;
        bool cand = false;
        if (j < s1) {
          const SrcRec r = P.rec[j];
          y[0] = to_local(r.yh.x, r.q.w, oh[0], ol[0]);
          y[1] = to_local(r.yh.y, r.n.w, oh[1], ol[1]);
          y[2] = to_local(r.yh.z, r.p.w, oh[2], ol[2]);
          hh = r.yh.w;
          cand = is_candidate(box_dist2(y[0], y[1], y[2], blo, bhi), hh);
        }
        for (unsigned cm = __ballot_sync(kFull, cand); cm; cm &= cm - 1) {
          const int l = __ffs(cm) - 1;
          const float y0 = __shfl_sync(kFull, y[0], l), y1 = __shfl_sync(kFull, y[1], l),
                      y2 = __shfl_sync(kFull, y[2], l), h2 = __shfl_sync(kFull, hh, l);
          const int32_t jl = (int32_t)(j0 + l);
#pragma unroll
          for (int t = 0; t < kNearT; ++t) {
            const float r2 =
                pair_r2(__fsub_rn(x[t][0], y0), __fsub_rn(x[t][1], y1), __fsub_rn(x[t][2], y2));
            const bool nr = valid[t] && is_near(r2, h2) && !(P.self_index && ci[t] == jl);
            const unsigned m = __ballot_sync(kFull, nr);
            if (nr) {
              const int pos = qn + __popc(m & lt);
              sm.qt[pos] = (uint8_t)(lane + kWarp * t);
              sm.qj[pos] = (int32_t)((uint32_t)jl | kind_bits);
            }
            qn += __popc(m);
          }
          if (qn > kNearQueue - kNearT * kWarp) {
            __syncwarp();
            eval_queue(sm, P, it.t0, qn, lane);
            qn = 0;
          }
        }
      }
    }
    __syncwarp();
    if (qn) eval_queue(sm, P, it.t0, qn, lane);

    // 4. add the item's near sums to its targets' partial results
    for (int li = lane; li < tn; li += kWarp) {
      double v[3];
      bool any = false;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        v[k] = (double)sm.acc[0][k][li] + (double)sm.acc[1][k][li];
        any |= sm.acc[0][k][li] != 0.f || sm.acc[1][k][li] != 0.f;
      }
      if (any) {
        double *o = P.part_out + ((size_t)part * (size_t)P.nt + (size_t)(it.t0 + li)) * 3;
        o[0] += v[0];
        o[1] += v[1];
        o[2] += v[2];
      }
    }
    __syncwarp();
  }
}

}  // namespace

// Runs after the engine on the same stream; P is the engine's parameter block
// (items, segments, records, partial results) and P.near_counter is zeroed.
void launch_near(const EngineParams &P, int sms, int64_t max_items, cudaStream_t st) {
  int64_t grid = (int64_t)sms * 8;
  const int64_t need = (max_items + kNearWarps - 1) / kNearWarps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_near<<<(int)grid, kNearWarps * kWarp, 0, st>>>(P);
  count_launches(1);
}

}  // namespace stk
