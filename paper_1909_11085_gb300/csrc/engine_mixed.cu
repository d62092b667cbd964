// engine_mixed.cu -- mixed FP32/FP64 evaluation of the Stokes single- and
// double-layer sums (Eq. "sl_stokes" and the double-layer kernel of Sec. 2.1,
// summed as in Sec. 3.1, Eq. "smooth_double_layer_int_eq_patches_disc").
//
// Design (GB300, sm_103a):
//  * Work unit = one warp-item: up to 128 spatially sorted targets held in
//    registers (T = 3..5 per lane, b = 1, 2 or 4 source slices per warp)
//    against a list of source segments.  Four independent warps per CTA; a
//    persistent grid pulls items from an atomic queue in cost order, so
//    uneven items balance without output atomics.
//  * Sources arrive as 64-byte records in chunks of up to 64, staged into
//    each warp's shared memory by a 1-D bulk async copy (cp.async.bulk)
//    completing on an mbarrier; the copy of chunk c+1 overlaps the arithmetic
//    of chunk c.  Contiguous segments of the same kind are merged so that
//    chunks stay full.
//  * Local frames: positions are stored hi/lo relative to a frame centre;
//    each item re-centres targets and sources on the item's own origin with
//    FP32 adds, so FP32 differences are accurate relative to |x - y| plus the
//    item extent, not the absolute coordinates.
//  * Each staged source is classified against the item's bounding box: far
//    sources (box distance >= alpha h_j) run a branch-free FP32 loop;
//    candidates run a masked loop in which a pair with |r| < alpha h_j is
//    left out of the FP32 sum (its |r|^2 is replaced by +inf, so rsqrt gives
//    0).  Nothing is recorded: k_near (near.cu) takes the same decisions with
//    the same arithmetic afterwards and adds those pairs with the FP64
//    difference and 1/|r|, whose FP64 work would otherwise stall this FP32
//    engine.
//  * Packed FP32 pairs: a lane evaluates two sources at once against each of
//    its targets with the sm_100 two-wide FP32 instructions (add/mul/fma on
//    float2), so one issued instruction does the work of two pairs.  Staged
//    sources are laid out as pairs, field-interleaved (x of both, then y of
//    both, ...), with the position negated so that d = x + (-y) is one packed
//    add; that is the same IEEE operation as x - y, bit for bit.
//  * Accumulation: plain FP32 over eight chunks (<= 256 terms per lane and
//    half), then the two halves are added and two-summed into per-target
//    (hi, lo) kept in shared memory.
//  * The kernel is instantiated per kernel kind (SL, DL, SL+DL, or SL/DL by
//    segment parity for batched suspensions) so that a launch only runs the
//    code of its own kind, which keeps the hot loops inside the instruction
//    cache.
#include "common.cuh"
#include "prep.cuh"

namespace stk {

// Resident CTAs per SM the engine is compiled for (registers per thread =
// 65536 / (128 * this)).
#ifndef STK_ENGINE_MIN_BLOCKS
#define STK_ENGINE_MIN_BLOCKS 3
#endif

constexpr int kSegWin = 64;  // segments read into shared memory at a time
constexpr int kTMax = 5;     // most targets per lane

constexpr int kPairs = kChunk / 2;  // staged source pairs per chunk
constexpr int kFields = 7;          // float4 fields per source pair

// Field f of source pair j holds two quantities of both sources (a0, a1, b0, b1):
//   0: -y_x, -y_y   1: -y_z, hh   2: q_x, q_y   3: q_z, n_x   4: n_y, n_z
//   5: psi_x, psi_y 6: psi_z, -
// hh is (alpha h)^2 for candidates and 0 for far sources (never masked).
struct __align__(16) WarpSmem {
  SrcRec raw[kChunk];               // bulk-copy destination
  float4 S[kFields][kPairs];        // staged source pairs in local coordinates
  float acc[2 * kTMax * 3][kWarp];  // per-lane compensated sums (hi, lo), lane-minor
  float frame[12];                  // item origin (hi x3, lo x3) and bounding box (lo x3, hi x3)
  int32_t run_s[kSegWin];           // source runs of the current segment window: start
  int32_t run_e[kSegWin];           //   end
  int32_t run_k[kSegWin];           //   kernel kind
  unsigned long long mbar;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait on the warp's mbarrier; every lane polls.  `limit` is in SM
// clock cycles (about 2 s by default); on expiry the caller records an error.
__device__ __forceinline__ bool wait_chunk(unsigned long long *bar, uint32_t parity, int64_t limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void issue_chunk(WarpSmem &sm, const SrcRec *rec, int64_t s, int n,
                                            int lane) {
  if (lane == 0) {
    fence_proxy_async();  // order earlier generic reads of raw[] before the async write
    const uint32_t bytes = (uint32_t)n * (uint32_t)sizeof(SrcRec);
    mbar_expect_tx(&sm.mbar, bytes);
    bulk_g2s(sm.raw, rec + s, bytes, &sm.mbar);
  }
}

// ---------------------------------------------------------------- pair math
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Adds the far-field contribution of one staged source pair to T targets
// (x2: each coordinate duplicated into both halves; ps: per-half sums).
// SL:   q/r + d (d.q)/r^3             (q pre-scaled by w / (8 pi mu))
// DL:   d (d.psi)(d.n)/r^5            (psi pre-scaled by 6 w / (8 pi))
// SLDL: q/r + d [(d.q)/r^3 + (d.psi)(d.n)/r^5]
// Per half the operations, operands and rounding are those of a scalar
// evaluation: d = x - y, |r|^2 = dx dx + (dy dy + dz dz) (pair_r2).
template <int T, int KIND, bool MASKED>
__device__ __forceinline__ void pair_block(const float2 (&x2)[T][3], float2 (&ps)[T][3],
                                           const float4 (&s)[kFields]) {
  const float2 ny_x = lo2(s[0]), ny_y = hi2(s[0]), ny_z = lo2(s[1]), hh = hi2(s[1]);
  const float2 qx = lo2(s[2]), qy = hi2(s[2]), qz = lo2(s[3]);
  const float2 nx = hi2(s[3]), ny = lo2(s[4]), nz = hi2(s[4]);
  const float2 px = lo2(s[5]), py = hi2(s[5]), pz = lo2(s[6]);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const float2 dx = add2(x2[t][0], ny_x), dy = add2(x2[t][1], ny_y), dz = add2(x2[t][2], ny_z);
    float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    // near pair: rsqrt(+inf) = 0 removes it from this sum (k_near adds it)
    if (MASKED) {
      if (is_near(r2.x, hh.x)) r2.x = __int_as_float(0x7f800000);
      if (is_near(r2.y, hh.y)) r2.y = __int_as_float(0x7f800000);
    }
    const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    const float2 ri2 = mul2(ri, ri);
    if (KIND == K_SL) {
      const float2 dq = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
      const float2 c = mul2(dq, ri2);
      ps[t][0] = fma2(fma2(dx, c, qx), ri, ps[t][0]);
      ps[t][1] = fma2(fma2(dy, c, qy), ri, ps[t][1]);
      ps[t][2] = fma2(fma2(dz, c, qz), ri, ps[t][2]);
    } else if (KIND == K_DL) {
      const float2 dp = fma2(dx, px, fma2(dy, py, mul2(dz, pz)));
      const float2 dn = fma2(dx, nx, fma2(dy, ny, mul2(dz, nz)));
      const float2 c = mul2(mul2(dp, dn), mul2(mul2(ri2, ri2), ri));
      ps[t][0] = fma2(dx, c, ps[t][0]);
      ps[t][1] = fma2(dy, c, ps[t][1]);
      ps[t][2] = fma2(dz, c, ps[t][2]);
    } else {
      const float2 dq = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
      const float2 dp = fma2(dx, px, fma2(dy, py, mul2(dz, pz)));
      const float2 dn = fma2(dx, nx, fma2(dy, ny, mul2(dz, nz)));
      const float2 c = mul2(fma2(mul2(dp, dn), ri2, dq), ri2);
      ps[t][0] = fma2(fma2(dx, c, qx), ri, ps[t][0]);
      ps[t][1] = fma2(fma2(dy, c, qy), ri, ps[t][1]);
      ps[t][2] = fma2(fma2(dz, c, qz), ri, ps[t][2]);
    }
  }
}

struct ItemCtx {
  int lane, b, G, tgl, sg, tn, part;
  int32_t t0;
};

template <int KIND>
__device__ __forceinline__ void load_pair(const WarpSmem &sm, int j, float4 (&s)[kFields]) {
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  s[0] = sm.S[0][j];
  s[1] = sm.S[1][j];
  s[2] = (KIND & K_SL) ? sm.S[2][j] : z4;
  s[3] = sm.S[3][j];
  s[4] = (KIND & K_DL) ? sm.S[4][j] : z4;
  s[5] = (KIND & K_DL) ? sm.S[5][j] : z4;
  s[6] = (KIND & K_DL) ? sm.S[6][j] : z4;
}

// Pairs [0, nfar / 2) hold far sources only; pairs from nfar / 2 to the end
// hold candidates (and possibly one far source with hh = 0, and a zero pad).
template <int T, int KIND>
__device__ __forceinline__ void chunk_compute(WarpSmem &sm, const EngineParams &P,
                                              const ItemCtx &ic, int n, int nfar,
                                              const float2 (&x2)[T][3], float2 (&ps)[T][3]) {
  const int jfar = nfar >> 1, jend = (n + 1) >> 1;
  for (int j = ic.sg; j < jfar; j += ic.b) {
    float4 s[kFields];
    load_pair<KIND>(sm, j, s);
    pair_block<T, KIND, false>(x2, ps, s);
  }
  for (int j = jfar + ic.sg; j < jend; j += ic.b) {
    float4 s[kFields];
    load_pair<KIND>(sm, j, s);
    pair_block<T, KIND, true>(x2, ps, s);
  }
}

// Converts the staged raw chunk to local coordinates, far sources first.
// Candidates are also listed for k_near (source index | kind << 30, at most
// cap per item; ccount keeps counting past cap to flag an overflow).
template <int KMODE>
__device__ __forceinline__ int convert_chunk(WarpSmem &sm, int n, int lane, int32_t *clist,
                                             int cap, int &ccount, int32_t s0, int kind) {
  const int kd = KMODE ? KMODE : kind;
  const uint32_t kind_bits = (uint32_t)kind << 30;
  float *S = reinterpret_cast<float *>(&sm.S[0][0]);
  const float oh[3] = {sm.frame[0], sm.frame[1], sm.frame[2]};
  const float ol[3] = {sm.frame[3], sm.frame[4], sm.frame[5]};
  const float blo[3] = {sm.frame[6], sm.frame[7], sm.frame[8]};
  const float bhi[3] = {sm.frame[9], sm.frame[10], sm.frame[11]};
  int nfar = 0, ncand = 0;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kChunk / kWarp; ++r) {
    const int k = r * kWarp + lane;
    const bool valid = k < n;
    bool cand = false;
    float4 Y = make_float4(0.f, 0.f, 0.f, 0.f), q = Y, nn = Y, pp = Y, yl4 = Y;
    if (valid) {
      const float4 yh = sm.raw[k].yh;
      q = sm.raw[k].q;
      nn = sm.raw[k].n;
      pp = sm.raw[k].p;
      yl4 = make_float4(q.w, nn.w, pp.w, 0.f);
      Y.x = to_local(yh.x, yl4.x, oh[0], ol[0]);
      Y.y = to_local(yh.y, yl4.y, oh[1], ol[1]);
      Y.z = to_local(yh.z, yl4.z, oh[2], ol[2]);
      Y.w = yh.w;
      cand = is_candidate(box_dist2(Y.x, Y.y, Y.z, blo, bhi), Y.w);
    }
    const unsigned bc = __ballot_sync(kFull, valid && cand);
    const unsigned bf = __ballot_sync(kFull, valid && !cand);
    if (valid && cand) {
      const int rank = ccount + __popc(bc & lt);
      if (rank < cap) clist[rank] = (int32_t)((uint32_t)(s0 + k) | kind_bits);
    }
    ccount += __popc(bc);
    if (valid) {
      const int dst = cand ? (n - 1 - (ncand + __popc(bc & lt))) : (nfar + __popc(bf & lt));
      float *d = S + 4 * (dst >> 1) + (dst & 1);  // component a_h of field 0
      constexpr int F = 4 * kPairs;               // floats per field
      d[0] = -Y.x;
      d[2] = -Y.y;
      d[F] = -Y.z;
      d[F + 2] = cand ? Y.w : 0.f;
      if (kd & K_SL) {
        d[2 * F] = q.x;
        d[2 * F + 2] = q.y;
        d[3 * F] = q.z;
      }
      if (kd & K_DL) {
        d[3 * F + 2] = nn.x;
        d[4 * F] = nn.y;
        d[4 * F + 2] = nn.z;
        d[5 * F] = pp.x;
        d[5 * F + 2] = pp.y;
        d[6 * F] = pp.z;
      }
    }
    nfar += __popc(bf);
    ncand += __popc(bc);
  }
  // an odd count leaves the second half of the last pair: a zero-density
  // source far away (no NaN arises: |r|^2 ~ 3e36 stays finite)
  if ((n & 1) && lane < kFields) {
    float *d = S + lane * 4 * kPairs + 4 * (n >> 1) + 1;
    d[0] = lane < 2 ? -1e18f : 0.f;
    d[2] = lane == 0 ? -1e18f : 0.f;
  }
  return nfar;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Walks the item's segments in chunks of at most kChunk sources.  Segments
// are read kSegWin at a time into shared memory, where runs of contiguous
// segments of the same kind are merged, so that the chunk loop touches no
// global index arrays and chunks stay full across adjacent leaves.
struct Cursor {
  int e0;      // first segment of the loaded window
  int nrun;    // runs in the window
  int r;       // current run
  int kind;
  int64_t s, end;
};

template <int KMODE>
__device__ __forceinline__ void load_window(const EngineParams &P, const Item &it, WarpSmem &sm,
                                            Cursor &c, int lane) {
  const int nwin = min(kSegWin, it.seg1 - c.e0);
  int nrun = 0;
  int32_t prev_end = -1, prev_kind = -1;
  for (int base = 0; base < nwin; base += kWarp) {
    const int e = base + lane;
    const bool valid = e < nwin;
    int32_t ss = 0, ee = 0, kd = 0;
    if (valid) {
      const int sid = P.seg_list ? P.seg_list[c.e0 + e] : c.e0 + e;
      ss = (int32_t)P.range_ptr[sid];
      ee = (int32_t)P.range_ptr[sid + 1];
      kd = KMODE ? KMODE : ((sid & 1) ? K_DL : K_SL);
    }
    int32_t pe = __shfl_up_sync(kFull, ee, 1), pk = __shfl_up_sync(kFull, kd, 1);
    if (lane == 0) {
      pe = prev_end;
      pk = prev_kind;
    }
    const bool start = valid && (ss != pe || kd != pk);
    const unsigned sb = __ballot_sync(kFull, start);
    const unsigned vb = __ballot_sync(kFull, valid);
    // the run an entry belongs to: starts at or before it
    const int ri = nrun + __popc(sb & ((2u << lane) - 1u)) - 1;
    if (start) {
      sm.run_s[ri] = ss;
      sm.run_k[ri] = kd;
    }
    const bool next_valid = (lane < kWarp - 1) && ((vb >> (lane + 1)) & 1u);
    const bool next_starts = (lane < kWarp - 1) && ((sb >> (lane + 1)) & 1u);
    if (valid && (next_starts || !next_valid)) sm.run_e[ri] = ee;
    nrun += __popc(sb);
    const int lastv = 31 - __clz(vb);
    prev_end = __shfl_sync(kFull, ee, lastv);
    prev_kind = __shfl_sync(kFull, kd, lastv);
    __syncwarp();
  }
  __syncwarp();
  c.nrun = nrun;
  c.r = -1;
}

template <int KMODE>
__device__ __forceinline__ bool cursor_next(const EngineParams &P, const Item &it, WarpSmem &sm,
                                            Cursor &c, int lane) {
  while (c.s >= c.end) {
    if (++c.r >= c.nrun) {
      c.e0 += kSegWin;
      if (c.e0 >= it.seg1) return false;
      load_window<KMODE>(P, it, sm, c, lane);
      continue;
    }
    c.s = sm.run_s[c.r];
    c.end = sm.run_e[c.r];
    c.kind = sm.run_k[c.r];
  }
  return true;
}

template <int T, int KMODE>
__device__ __forceinline__ void dispatch_compute(int kind, WarpSmem &sm, const EngineParams &P,
                                                 const ItemCtx &ic, int n, int nfar,
                                                 const float2 (&x2)[T][3], float2 (&ps)[T][3]) {
  if (KMODE != 0) {
    chunk_compute<T, KMODE>(sm, P, ic, n, nfar, x2, ps);
  } else if (kind == K_SL) {
    chunk_compute<T, K_SL>(sm, P, ic, n, nfar, x2, ps);
  } else {
    chunk_compute<T, K_DL>(sm, P, ic, n, nfar, x2, ps);
  }
}

// One work item with T targets per lane and b source slices per warp.
template <int T, int KMODE>
__device__ bool run_item(const EngineParams &P, const Item &it, int id, WarpSmem &sm, int b,
                         uint32_t &phase, int lane) {
  ItemCtx ic;
  ic.lane = lane;
  ic.b = b;
  ic.G = kWarp / b;
  ic.tgl = lane % ic.G;
  ic.sg = lane / ic.G;
  ic.tn = it.tn_part & 0xFF;
  ic.t0 = it.t0;
  const int part = it.tn_part >> 8;
  ic.part = part;

  // Item frame: origin at the centre of the targets' bounding box, targets
  // in local coordinates.  When the targets are the sources, their FP32
  // hi/lo records already hold the split positions; otherwise the FP64
  // target positions are split here.
  bool valid[T];
  float oh[3], ol[3], x[T][3];
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  const int c0 = P.tperm ? P.tperm[it.t0] : it.t0;
  if (P.self_index) {
    const SrcRec r0 = P.rec[c0];
    const float x0h[3] = {r0.yh.x, r0.yh.y, r0.yh.z}, x0l[3] = {r0.q.w, r0.n.w, r0.p.w};
    float xh[T][3], xl[T][3];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int li = ic.tgl + ic.G * t;
      valid[t] = li < ic.tn;
      const int gi = it.t0 + (valid[t] ? li : 0);
      const SrcRec r = P.rec[P.tperm ? P.tperm[gi] : gi];
      xh[t][0] = r.yh.x; xh[t][1] = r.yh.y; xh[t][2] = r.yh.z;
      xl[t][0] = r.q.w;  xl[t][1] = r.n.w;  xl[t][2] = r.p.w;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (valid[t]) {
          const float rk = to_local(xh[t][k], xl[t][k], x0h[k], x0l[k]);
          mn[k] = fminf(mn[k], rk);
          mx[k] = fmaxf(mx[k], rk);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      oh[k] = __fadd_rn(x0h[k], __fmul_rn(0.5f, __fadd_rn(warp_min(mn[k]), warp_max(mx[k]))));
      ol[k] = x0l[k];
    }
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) x[t][k] = valid[t] ? to_local(xh[t][k], xl[t][k], oh[k], ol[k]) : 1e30f;
  } else {
    const double x0[3] = {P.trg64[3 * (size_t)c0], P.trg64[3 * (size_t)c0 + 1],
                          P.trg64[3 * (size_t)c0 + 2]};
    const double cc[3] = {P.src64[0], P.src64[1], P.src64[2]};
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int li = ic.tgl + ic.G * t;
      valid[t] = li < ic.tn;
      if (valid[t]) {
        const int gi = it.t0 + li;
        const double *xp = P.trg64 + 3 * (size_t)(P.tperm ? P.tperm[gi] : gi);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float rk = f64_to_f32_rn(xp[k] - x0[k]);
          mn[k] = fminf(mn[k], rk);
          mx[k] = fmaxf(mx[k], rk);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) frame_origin(x0[k], warp_min(mn[k]), warp_max(mx[k]), cc[k], oh[k], ol[k]);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int li = ic.tgl + ic.G * t;
      const int gi = it.t0 + (valid[t] ? li : 0);
      const double *xp = P.trg64 + 3 * (size_t)(P.tperm ? P.tperm[gi] : gi);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        x[t][k] = valid[t] ? local_coord(xp[k], cc[k], oh[k], ol[k]) : 1e30f;  // 1e30: padding
    }
  }
  float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (valid[t]) {
        blo[k] = fminf(blo[k], x[t][k]);
        bhi[k] = fmaxf(bhi[k], x[t][k]);
      }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    blo[k] = warp_min(blo[k]);
    bhi[k] = warp_max(bhi[k]);
  }
  if (lane == 0) {
    float *fr = P.frames + 12 * (size_t)id;  // k_near decides in this same frame
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sm.frame[k] = fr[k] = oh[k];
      sm.frame[3 + k] = fr[3 + k] = ol[k];
      sm.frame[6 + k] = fr[6 + k] = blo[k];
      sm.frame[9 + k] = fr[9 + k] = bhi[k];
    }
  }
  if (part == 0) {
#pragma unroll
    for (int t = 0; t < T; ++t)
      if (valid[t] && ic.sg == 0) {
        float *xl = P.xloc + 3 * (size_t)(it.t0 + ic.tgl + ic.G * t);
        xl[0] = x[t][0];
        xl[1] = x[t][1];
        xl[2] = x[t][2];
      }
  }

  float2 x2[T][3], ps[T][3];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      x2[t][k] = make_float2(x[t][k], x[t][k]);
      ps[t][k] = make_float2(0.f, 0.f);
      sm.acc[t * 3 + k][lane] = 0.f;
      sm.acc[(T + t) * 3 + k][lane] = 0.f;
    }

  Cursor cur;
  cur.e0 = it.seg0;
  cur.kind = KMODE;
  cur.s = cur.end = 0;
  bool have = false;
  if (it.seg1 > it.seg0) {
    load_window<KMODE>(P, it, sm, cur, lane);
    have = cursor_next<KMODE>(P, it, sm, cur, lane);
  }
  int n_cur = 0, kind_cur = 0;
  int32_t s_cur = 0;
  int ccount = 0;
  int32_t *clist = P.cand_list + (size_t)id * (size_t)P.cand_cap;
  if (have) {
    n_cur = (int)min((int64_t)kChunk, cur.end - cur.s);
    kind_cur = cur.kind;
    s_cur = (int32_t)cur.s;
    issue_chunk(sm, P.rec, cur.s, n_cur, lane);
    cur.s += n_cur;
  }
  bool ok = true;
  int npend = 0;
  while (have) {
    if (P.force_expire || !wait_chunk(&sm.mbar, phase, P.spin_limit)) {
      set_error(P.err_flag, 4);
      ok = false;
      // The copy this warp issued last still writes into its shared memory:
      // the warp waits for it before it leaves (bounded by the drain limit,
      // which is at least the default wait limit, so a copy from valid memory
      // always completes first; only one copy per warp is ever in flight).
      if (!wait_chunk(&sm.mbar, phase, P.drain_limit)) set_error(P.err_flag, 5);
      break;
    }
    phase ^= 1u;
    const int nfar = convert_chunk<KMODE>(sm, n_cur, lane, clist, P.cand_cap, ccount, s_cur,
                                          kind_cur);
    __syncwarp();
    const bool have_next = cursor_next<KMODE>(P, it, sm, cur, lane);
    int n_next = 0, kind_next = 0;
    int32_t s_next = 0;
    if (have_next) {
      n_next = (int)min((int64_t)kChunk, cur.end - cur.s);
      kind_next = cur.kind;
      s_next = (int32_t)cur.s;
      issue_chunk(sm, P.rec, cur.s, n_next, lane);
      cur.s += n_next;
    }
    dispatch_compute<T, KMODE>(kind_cur, sm, P, ic, n_cur, nfar, x2, ps);
    // plain FP32 over eight chunks (<= 256 sources per half), then into the
    // (hi, lo) sums
    if (++npend == 8 || !have_next) {
      npend = 0;
#pragma unroll
      for (int t = 0; t < T; ++t)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float h = sm.acc[t * 3 + k][lane], l = sm.acc[(T + t) * 3 + k][lane];
          two_sum_acc(h, l, ps[t][k].x + ps[t][k].y);
          sm.acc[t * 3 + k][lane] = h;
          sm.acc[(T + t) * 3 + k][lane] = l;
          ps[t][k] = make_float2(0.f, 0.f);
        }
    }
    __syncwarp();
    have = have_next;
    n_cur = n_next;
    kind_cur = kind_next;
    s_cur = s_next;
  }
  if (!ok) return false;
  if (lane == 0) P.cand_cnt[id] = ccount <= P.cand_cap ? ccount : -1;
  float hi[T][3], lo[T][3];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      hi[t][k] = sm.acc[t * 3 + k][lane];
      lo[t][k] = sm.acc[(T + t) * 3 + k][lane];
    }

  // combine the b source slices (lanes tgl, tgl + G, ...)
  for (int o = ic.G; o < kWarp; o <<= 1) {
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float h2 = __shfl_xor_sync(kFull, hi[t][k], o);
        const float l2 = __shfl_xor_sync(kFull, lo[t][k], o);
        two_sum_acc(hi[t][k], lo[t][k], h2);
        lo[t][k] += l2;
      }
  }
  if (ic.sg == 0) {
    double *out = P.part_out + ((size_t)part * (size_t)P.nt + (size_t)it.t0) * 3;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      if (valid[t]) {
        const int li = ic.tgl + ic.G * t;
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * li + k] = (double)hi[t][k] + (double)lo[t][k];
      }
    }
  }
  return true;
}

template <int KMODE>
__global__ void __launch_bounds__(kWarpsPerCta *kWarp, STK_ENGINE_MIN_BLOCKS) k_engine_mixed(EngineParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[threadIdx.x / kWarp];
  const int lane = threadIdx.x & (kWarp - 1);
  if (lane == 0) {
    mbar_init(&sm.mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  __syncwarp();
  uint32_t phase = 0;
  const int n_items = *P.n_items;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(P.item_counter, 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= n_items) break;
    const int id = P.item_order ? P.item_order[idx] : idx;
    const Item it = P.items[id];
    const int tn = it.tn_part & 0xFF;
    bool ok;
    // Lane layout: T = 3, 4 or 5 targets per lane and b source slices, the
    // fewest target slots (32 T / b) that hold the item.  Policy 1 uses no
    // more than two slices.
    const int b = (P.policy != 1 && tn <= 40) ? 4 : (tn <= 80 ? 2 : 1);
    const int slots_per_t = kWarp / b;
    if (tn <= 3 * slots_per_t)
      ok = run_item<3, KMODE>(P, it, id, sm, b, phase, lane);
    else if (tn <= 4 * slots_per_t)
      ok = run_item<4, KMODE>(P, it, id, sm, b, phase, lane);
    else
      ok = run_item<5, KMODE>(P, it, id, sm, b, phase, lane);
    if (!ok) break;
  }
}

size_t engine_mixed_smem_bytes() { return sizeof(WarpSmem) * kWarpsPerCta; }

template <int KMODE>
static cudaError_t launch_kmode(const EngineParams &P, int grid, cudaStream_t stream) {
  k_engine_mixed<KMODE><<<grid, kWarpsPerCta * kWarp, engine_mixed_smem_bytes(), stream>>>(P);
  count_launches(1);
  return cudaGetLastError();
}

// The dynamic shared memory (> 48 KB) needs the opt-in attribute on every
// device; engine_mixed_occupancy() sets it and runs once per device before
// the first launch there.
cudaError_t launch_engine_mixed(const EngineParams &P, int grid, cudaStream_t stream) {
  if (P.kind_alternating) return launch_kmode<0>(P, grid, stream);
  switch (P.kind) {
    case K_SL: return launch_kmode<K_SL>(P, grid, stream);
    case K_DL: return launch_kmode<K_DL>(P, grid, stream);
    default: return launch_kmode<K_SLDL>(P, grid, stream);
  }
}

template <int KMODE>
static cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(k_engine_mixed<KMODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)engine_mixed_smem_bytes());
}

cudaError_t engine_mixed_occupancy(int *blocks_per_sm) {
  cudaError_t e;
  if ((e = set_smem_attr<0>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<K_SL>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<K_DL>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<K_SLDL>()) != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_engine_mixed<K_SLDL>,
                                                       kWarpsPerCta * kWarp,
                                                       engine_mixed_smem_bytes());
}

}  // namespace stk
