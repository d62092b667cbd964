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
//  1. the item's frame and its targets' local coordinates, as the engine
//     stored them (so the decisions below match the engine's bit for bit);
//  2. the candidate sources the engine listed for the item: each lane takes
//     one, computes its local coordinates and tests it against every target
//     (two per packed FP32 instruction) into a bit mask.  An item whose list
//     overflowed has all its sources scanned again, 32 per round across
//     segment boundaries: a conservative box test on the 16-byte position
//     record, then for the few sources it keeps the exact local coordinates
//     and the engine's box test; each candidate is broadcast and every lane
//     tests its targets;
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
constexpr int kNearMinBlocks = 8;
constexpr int kNearT = kItemMax / kWarp;  // targets per lane
constexpr int kNearQueue = 192;           // >= 128 free slots before each candidate
constexpr int kNearSegWin = 32;           // segments per window

struct __align__(16) NearSmem {
  float xs[3][kItemMax];             // targets: local coordinates (slots to a multiple of 8;
                                     //   padding far away),
  int32_t sid[kItemMax];             //   caller index (self pairs; -1: none)
  float sv[kWarp][3];                // values of one round of evaluations
  float acc[2][3][kItemMax];         // per-target compensated sums (hi, lo)
  int32_t qj[kNearQueue];            // queued pair: source index | kind << 30
  uint8_t qt[kNearQueue];            //   target within the item
  int32_t seg_start[kNearSegWin];    // window of segments: first source (< 2^30),
  int32_t seg_pre[kNearSegWin + 1];  //   sources before it in the window,
  int32_t seg_kind[kNearSegWin];     //   kind bits
};

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

__global__ void __launch_bounds__(kNearWarps *kWarp, kNearMinBlocks) k_near(EngineParams P) {
  __shared__ NearSmem smem[kNearWarps];
  NearSmem &sm = smem[threadIdx.x / kWarp];
  const int lane = threadIdx.x & (kWarp - 1);
  const unsigned lt = (1u << lane) - 1u;
  const int n_items = *P.n_items;
  if (*P.err_flag) return;  // the engine stopped early: its lists are incomplete
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(P.near_counter, 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= n_items) break;
    const int32_t id = P.item_order ? P.item_order[idx] : idx;
    const Item it = P.items[id];
    const int tn = it.tn_part & 0xFF, part = it.tn_part >> 8;

    // 1. the engine's frame and target coordinates
    const float *fr = P.frames + 12 * (size_t)id;
    float oh[3], ol[3], blo[3], bhi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      oh[k] = fr[k];
      ol[k] = fr[3 + k];
      blo[k] = fr[6 + k];
      bhi[k] = fr[9 + k];
    }
    const float tol0 = 4.8e-7f * (fabsf(oh[0]) + fabsf(oh[1]) + fabsf(oh[2]));
    int32_t self_id[kNearT];  // caller index of each target when targets are the sources
    float x[kNearT][3];
#pragma unroll
    for (int t = 0; t < kNearT; ++t) {
      const int li = lane + kWarp * t;
      self_id[t] = -1;
      x[t][0] = x[t][1] = x[t][2] = 1e30f;  // padding: never near (|r|^2 = inf)
      if (li < tn) {
        const int32_t gi = it.t0 + li;
        if (P.self_index) self_id[t] = P.tperm ? P.tperm[gi] : gi;
        const float *xl = P.xloc + 3 * (size_t)gi;
        x[t][0] = xl[0];
        x[t][1] = xl[1];
        x[t][2] = xl[2];
      }
    }
    for (int li = lane; li < tn; li += kWarp)
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.acc[0][k][li] = sm.acc[1][k][li] = 0.f;
    const int tn8 = (tn + 7) & ~7;
#pragma unroll
    for (int t = 0; t < kNearT; ++t) {
      const int li = lane + kWarp * t;
      if (li < tn8) {  // x holds 1e30 and self_id -1 beyond tn
        sm.xs[0][li] = x[t][0];
        sm.xs[1][li] = x[t][1];
        sm.xs[2][li] = x[t][2];
        sm.sid[li] = self_id[t];
      }
    }
    __syncwarp();

    // 2./3. candidate sources: each is broadcast and every lane tests its
    // targets; near pairs are queued (by lane, then target slot)
    int qn = 0;
    auto test_round = [&](bool cand, const float (&y)[3], float hh, int32_t j, uint32_t kb) {
      for (unsigned cm = __ballot_sync(kFull, cand); cm; cm &= cm - 1) {
        const int l = __ffs(cm) - 1;
        const float y0 = __shfl_sync(kFull, y[0], l), y1 = __shfl_sync(kFull, y[1], l),
                    y2 = __shfl_sync(kFull, y[2], l), h2 = __shfl_sync(kFull, hh, l);
        const int32_t jl = (int32_t)__shfl_sync(kFull, (int32_t)j, l);
        const uint32_t kind_bits = __shfl_sync(kFull, kb, l);
        // this lane's near targets (slots beyond the item hold padding)
        unsigned nm = 0;
#pragma unroll
        for (int t = 0; t < kNearT; ++t) {
          if (t * kWarp < tn) {
            const float r2 =
                pair_r2(__fsub_rn(x[t][0], y0), __fsub_rn(x[t][1], y1), __fsub_rn(x[t][2], y2));
            if (is_near(r2, h2) && self_id[t] != jl) nm |= 1u << t;
          }
        }
        const unsigned any = __ballot_sync(kFull, nm != 0);
        if (any == 0) continue;
        // queue order: by lane, then by target slot within the lane
        const int cnt = __popc(nm);
        const unsigned b0 = __ballot_sync(kFull, cnt & 1), b1 = __ballot_sync(kFull, cnt & 2),
                       b2 = __ballot_sync(kFull, cnt & 4);
        int pos = qn + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
        for (unsigned mm = nm; mm; mm &= mm - 1, ++pos) {
          sm.qt[pos] = (uint8_t)(lane + kWarp * (__ffs(mm) - 1));
          sm.qj[pos] = (int32_t)((uint32_t)jl | kind_bits);
        }
        qn += __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
        if (qn > kNearQueue - kNearT * kWarp) {
          __syncwarp();
          eval_queue(sm, P, it.t0, qn, lane);
          qn = 0;
        }
      }
    };
    const int32_t ncl = P.cand_cnt[id];
    if (ncl >= 0) {
      // The engine listed this item's candidates.  Each lane takes one
      // candidate and tests it against every target of the item, two targets
      // per packed FP32 instruction (per half the same IEEE operations as the
      // engine's test), into a bit mask without a vote per target; the near
      // pairs are then queued by candidate (lane), then by target.
      const int32_t *cl = P.cand_list + (size_t)id * (size_t)P.cand_cap;
      const int n_list = min(ncl, P.cand_cap);
      for (int p0 = 0; p0 < n_list; p0 += kWarp) {
        const int pp = p0 + lane;
        float2 ny0 = make_float2(0.f, 0.f), ny1 = ny0, ny2 = ny0;
        float hh = -1.f;  // hh < 0: idle lane, never near
        int32_t j = -1;
        uint32_t kb = 0;
        if (pp < n_list) {
          const uint32_t e = (uint32_t)cl[pp];
          j = (int32_t)(e & 0x3fffffffu);
          kb = e & 0xc0000000u;
          const float4 yh = __ldg(&P.rec[j].yh);
          const float ylx = __ldg(&P.rec[j].q.w), yly = __ldg(&P.rec[j].n.w),
                      ylz = __ldg(&P.rec[j].p.w);
          const float y0 = to_local(yh.x, ylx, oh[0], ol[0]);
          const float y1 = to_local(yh.y, yly, oh[1], ol[1]);
          const float y2 = to_local(yh.z, ylz, oh[2], ol[2]);
          ny0 = make_float2(-y0, -y0);  // x + (-y) is the IEEE x - y
          ny1 = make_float2(-y1, -y1);
          ny2 = make_float2(-y2, -y2);
          hh = yh.w;
        }
        unsigned mask[kNearT];
#pragma unroll
        for (int w = 0; w < kNearT; ++w) {
          mask[w] = 0u;
          if (w * kWarp < tn) {
#pragma unroll
            for (int i = 0; i < kWarp; i += 2) {
              const int ti = w * kWarp + i;
              if (ti >= tn8) break;
              const float2 X0 = *reinterpret_cast<const float2 *>(&sm.xs[0][ti]);
              const float2 X1 = *reinterpret_cast<const float2 *>(&sm.xs[1][ti]);
              const float2 X2 = *reinterpret_cast<const float2 *>(&sm.xs[2][ti]);
              const int2 S2 = *reinterpret_cast<const int2 *>(&sm.sid[ti]);
              const float2 d0 = __fadd2_rn(X0, ny0), d1 = __fadd2_rn(X1, ny1),
                           d2 = __fadd2_rn(X2, ny2);
              const float2 r2 = __ffma2_rn(d0, d0, __ffma2_rn(d1, d1, __fmul2_rn(d2, d2)));
              if (is_near(r2.x, hh) && S2.x != j) mask[w] |= 1u << i;
              if (is_near(r2.y, hh) && S2.y != j) mask[w] |= 2u << i;
            }
          }
        }
        int cnt = 0;
#pragma unroll
        for (int w = 0; w < kNearT; ++w) cnt += __popc(mask[w]);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, kWarp - 1);
        if (total == 0) continue;
        const int base = incl - cnt;  // this lane's first entry within the round
        const int32_t jq = (int32_t)((uint32_t)j | kb);
        // the round's entries [done, done + room) go to the queue; a full queue
        // is evaluated before the rest
        for (int done = 0;;) {
          const int room = kNearQueue - qn;
          int idx = base;
#pragma unroll
          for (int w = 0; w < kNearT; ++w)
            for (unsigned m = mask[w]; m; m &= m - 1, ++idx)
              if (idx >= done && idx < done + room) {
                const int pos = qn + idx - done;
                sm.qt[pos] = (uint8_t)(w * kWarp + __ffs(m) - 1);
                sm.qj[pos] = jq;
              }
          const int n_emit = min(room, total - done);
          qn += n_emit;
          done += n_emit;
          if (done == total) break;
          __syncwarp();
          eval_queue(sm, P, it.t0, qn, lane);
          qn = 0;
        }
      }
    } else {
      // more candidates than the list holds: scan the item's sources
      for (int32_t w0 = it.seg0; w0 < it.seg1; w0 += kNearSegWin) {
        const int nw = min(kNearSegWin, it.seg1 - w0);
        __syncwarp();
        int run = 0;  // sources in the window before this lane's pair of segments
        int32_t sz[2] = {0, 0};
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = 2 * lane + h;
          if (e < nw) {
            const int32_t sid = P.seg_list ? P.seg_list[w0 + e] : w0 + e;
            const int64_t a = P.range_ptr[sid];
            sz[h] = (int32_t)(P.range_ptr[sid + 1] - a);
            sm.seg_start[e] = (int32_t)a;
            sm.seg_kind[e] = seg_kind(P, sid) << 30;
          }
        }
        int incl = sz[0] + sz[1];
  #pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += v;
        }
        run = incl - sz[0] - sz[1];
        if (2 * lane < nw) sm.seg_pre[2 * lane] = run;
        if (2 * lane + 1 < nw) sm.seg_pre[2 * lane + 1] = run + sz[0];
        const int total = __shfl_sync(kFull, incl, kWarp - 1);
        if (lane == 0) sm.seg_pre[nw] = total;
        __syncwarp();

        for (int p0 = 0; p0 < total; p0 += kWarp) {
          const int pp = p0 + lane;
          int64_t j = 0;
          uint32_t kb = 0;
          float y[3] = {0.f, 0.f, 0.f}, hh = 0.f;
          bool cand = false;
          if (pp < total) {
            int e = 0;  // last segment starting at or before pp
  #pragma unroll
            for (int step = kNearSegWin / 2; step > 0; step >>= 1)
              if (e + step < nw && sm.seg_pre[e + step] <= pp) e += step;
            j = sm.seg_start[e] + (pp - sm.seg_pre[e]);
            kb = (uint32_t)sm.seg_kind[e];
            const float4 yh = __ldg(&P.rec[j].yh);
            hh = yh.w;
            // conservative test: yh - oh differs from the local coordinate by
            // less than tol (the dropped low parts and one rounding each)
            const float tol =
                fmaf(4.8e-7f, fabsf(yh.x) + fabsf(yh.y) + fabsf(yh.z), tol0) + 1e-30f;
            const float lo2[3] = {blo[0] - tol, blo[1] - tol, blo[2] - tol};
            const float hi2[3] = {bhi[0] + tol, bhi[1] + tol, bhi[2] + tol};
            const float bd2a = box_dist2(yh.x - oh[0], yh.y - oh[1], yh.z - oh[2], lo2, hi2);
            if (bd2a < hh * 1.0001f + 1e-30f) {
              const float ylx = __ldg(&P.rec[j].q.w), yly = __ldg(&P.rec[j].n.w),
                          ylz = __ldg(&P.rec[j].p.w);
              y[0] = to_local(yh.x, ylx, oh[0], ol[0]);
              y[1] = to_local(yh.y, yly, oh[1], ol[1]);
              y[2] = to_local(yh.z, ylz, oh[2], ol[2]);
              cand = is_candidate(box_dist2(y[0], y[1], y[2], blo, bhi), hh);
            }
          }
          test_round(cand, y, hh, (int32_t)j, kb);
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
