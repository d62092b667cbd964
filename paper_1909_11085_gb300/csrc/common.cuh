// common.cuh -- types and device helpers shared by the library's kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace stk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarp = 32;
constexpr int kChunk = 64;      // sources staged per chunk (one bulk copy)
constexpr int kItemMax = 128;   // most targets per work item (32 lanes x 4)

// Work-item shapes the autotuner chooses from: the most targets per item and
// the lane layout (0: T = 3..5 targets per lane with b = 1, 2 or 4 source
// slices, the fewest target slots that hold the item; 1: the same with at
// most two slices).
struct TileConfig {
  int32_t item_max;
  int32_t policy;
};
constexpr int kNumTileConfigs = 4;
constexpr int kMinItemMax = 64;
__host__ __device__ inline TileConfig tile_config(int id) {
  switch (id) {
    case 1: return TileConfig{128, 1};
    case 2: return TileConfig{64, 0};
    case 3: return TileConfig{96, 0};
    default: return TileConfig{128, 0};
  }
}
constexpr int kWarpsPerCta = 4; // engine CTA = 4 independent warps

enum Kind : int { K_SL = 1, K_DL = 2, K_SLDL = 3 };

// Work item: up to 128 targets (sorted order) against a list of source segments.
struct Item {
  int32_t t0;       // first target (sorted order)
  int32_t tn_part;  // tn (1..128) | part << 8
  int32_t seg0;     // segment list range [seg0, seg1)
  int32_t seg1;
};

// Mixed-precision source record, 64 bytes, one per source (AoS so that one
// 1-D bulk copy stages a chunk).  Positions are split hi/lo relative to the
// frame centre c: y - c = yh + yl to about 2^-48 relative; the low parts ride
// in the .w lanes of the density and normal vectors.
struct __align__(16) SrcRec {
  float4 yh;  // fp32(y - c), hh = (alpha h)^2 clamped >= FLT_MIN
  float4 q;   // w f / (8 pi mu), .w = yl.x
  float4 n;   // outward unit normal, .w = yl.y
  float4 p;   // w phi * 6 / (8 pi), .w = yl.z
};
static_assert(sizeof(SrcRec) == 64, "SrcRec layout");

// FP64 source record for the FP64 path.
struct __align__(16) SrcRec64 {
  double y[3];
  double q[3];
  double n[3];
  double p[3];
};
static_assert(sizeof(SrcRec64) == 96, "SrcRec64 layout");

// Parameters of both engines.
struct EngineParams {
  const SrcRec *rec;         // mixed records (MIXED)
  const SrcRec64 *rec64;     // FP64 records (FP64)
  const double *src64;       // caller FP64 source positions [ns][3]
  const double *trg64;       // caller FP64 target positions [nt][3]
  const int32_t *tperm;      // sorted target -> caller index (NULL = identity)
  const Item *items;         // work items
  const int32_t *item_order; // processing order (NULL = identity)
  const int32_t *n_items;    // device count of items
  const int32_t *seg_list;   // segment ids (NULL = identity)
  const int64_t *range_ptr;  // source range of segment id s: [range_ptr[s], range_ptr[s+1])
  int32_t kind;              // K_SL / K_DL / K_SLDL for all segments
  int32_t kind_alternating;  // 1: segment id even -> SL, odd -> DL
  int32_t nt;                // number of targets
  int32_t self_index;        // 1: caller target index == source index means the same point
  int32_t policy;            // lane layout of the tile configuration
  double *part_out;          // [nparts][nt][3], sorted target order
  int32_t *item_counter;     // engine work queue head (zeroed before launch)
  int32_t *near_counter;     // k_near work queue head (zeroed before launch)
  float *frames;             // MIXED: per item, the engine's local frame (origin hi x3,
                             //   lo x3, target box lo x3, hi x3) for k_near
  float *xloc;               // MIXED: [nt][3] targets in their item's local frame
  int32_t *cand_list;        // MIXED: per item, up to cand_cap candidate sources (index | kind << 30)
  int32_t *cand_cnt;         // MIXED: per item, candidates listed (-1: more than cand_cap)
  int32_t cand_cap;
  int32_t *err_flag;         // device error word
  int64_t spin_limit;        // bounded mbarrier waits, in SM clock cycles
  int64_t drain_limit;       // bound of the wait for a warp's own copy after an expiry
  int32_t force_expire;      // 1: every item's first chunk wait reports expiry (failure-path tests)
};

__device__ __forceinline__ int seg_kind(const EngineParams &P, int32_t sid) {
  return P.kind_alternating ? ((sid & 1) ? K_DL : K_SL) : P.kind;
}

// FP64 <-> FP32 conversions on the integer pipe.  GB300 runs conversions
// that involve FP64 on its FP64 pipe (1/64 of the FP32 rate), where they were
// a third of the near pairs' FP64 operations and most of the packing's.  An
// FP64 instruction on a rarely taken path costs the same pipe time as a taken
// one when the compiler predicates it, so every finite input is handled here
// with integer operations, and only infinities and NaN (never met by the sums)
// reach the hardware conversion, through a call that runs only when made.
// f64_to_f32_rn rounds to nearest, ties to even (IEEE 754 binary64 to
// binary32): for a normal result the sign, the rebiased exponent and the top
// 23 of the 52 fraction bits, plus one when the 29 dropped bits are above half
// an FP32 ulp or exactly half with an odd kept fraction (a carry out of the
// fraction moves into the exponent, so a value just below 2^k rounds up to
// 2^k and one at or above FLT_MAX + ulp/2 to infinity); values of 2^128 and
// above give infinity; below 2^-126 the 53-bit significand is shifted to a
// multiple of 2^-149 with the same rounding (subnormal results, zero below
// 2^-150, the smallest normal when the rounding carries).  f32_to_f64 widens
// exactly: rebiased exponent and the fraction in the top of the 52 bits, a
// subnormal float normalised by its leading bit.
static __device__ __noinline__ float f64_to_f32_special(double v) { return __double2float_rn(v); }
static __device__ __noinline__ double f32_to_f64_special(float f) { return (double)f; }
// |v| < 2^-126 (out of line too: rare, and several 64-bit operations): k =
// 1.f x 2^(e + 149) rounded to nearest even, the result k x 2^-149.
static __device__ __noinline__ float f64_to_f32_small(unsigned long long u) {
  const int ef = (int)((u >> 52) & 0x7ffu), sh = -97 - (ef - 1023);  // shift >= 30
  unsigned k = 0u;
  if (ef != 0 && sh <= 53) {
    const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);
    const unsigned long long q = m >> sh, rest = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    k = (unsigned)q + ((rest > half || (rest == half && (q & 1ull))) ? 1u : 0u);
  }
  return __uint_as_float(((unsigned)(u >> 32) & 0x80000000u) | k);
}
// A subnormal float m x 2^-149 = 1.f x 2^(p - 149), p the index of m's leading bit.
static __device__ __noinline__ double f32_to_f64_small(unsigned b) {
  const unsigned m = b & 0x7fffffu, sign = b & 0x80000000u;
  const int p = 31 - __clz(m);
  const unsigned long long frac = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffull;
  return __hiloint2double((int)(sign | ((unsigned)(p + 874) << 20) | (unsigned)(frac >> 32)),
                          (int)(unsigned)frac);
}
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sign = hi & 0x80000000u;
  const int ef = (int)((hi >> 20) & 0x7ffu), e = ef - 1023;  // e: unbiased exponent
  if (ef == 0x7ff) return f64_to_f32_special(v);            // infinity or NaN
  if (e < -126)  // zero (common: the low part of an FP32-exact value) inline, the rest out of line
    return (u << 1) == 0ull ? __uint_as_float(sign) : f64_to_f32_small(u);
  if (e > 127) return __uint_as_float(sign | 0x7f800000u);
  const unsigned kept = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 fraction bits
  const unsigned dropped = lo & 0x1fffffffu;                    // the other 29
  const unsigned up =
      (dropped > 0x10000000u || (dropped == 0x10000000u && (kept & 1u))) ? 1u : 0u;
  return __uint_as_float((sign | ((unsigned)(e + 127) << 23) | kept) + up);
}
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu, sign = b & 0x80000000u;
  if (e == 0xffu) return f32_to_f64_special(f);  // infinity or NaN
  if (e != 0u) return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
  if (m == 0u) return __hiloint2double((int)sign, 0);
  return f32_to_f64_small(b);
}

// Exact-enough split of (x - c) into two floats; used identically for
// sources and targets so that coincident points get bit-identical local
// coordinates.
__device__ __forceinline__ void split_hl(double v, float &hi, float &lo) {
  hi = f64_to_f32_rn(v);
  lo = f64_to_f32_rn(v - f32_to_f64(hi));
}
__device__ __forceinline__ float to_local(float vh, float vl, float oh, float ol) {
  return __fadd_rn(__fsub_rn(vh, oh), __fsub_rn(vl, ol));
}

// ---------------------------------------------------------------------------
// Near/far decisions.  The mixed engine leaves a pair out of its FP32 sum when
// the pair is near in the item's local frame; k_near later finds the same
// pairs and adds them in FP64.  Both kernels compute the frame, the local
// coordinates, the box distance and |r|^2 with the functions below, built only
// from explicitly rounded operations (no contraction into FMAs the compiler
// might choose differently), so their decisions agree bit for bit.

// Item origin: centre of the targets' box, as an offset from the first target
// x0 (mn, mx: box of the targets' FP32 offsets from x0), split hi/lo about the
// frame centre c.
__device__ __forceinline__ void frame_origin(double x0, float mn, float mx, double c, float &oh,
                                             float &ol) {
  const double org = fma(0.5, __dadd_rn((double)mn, (double)mx), x0);
  split_hl(__dsub_rn(org, c), oh, ol);
}
// Local coordinate of a caller FP64 coordinate v (frame centre c).
__device__ __forceinline__ float local_coord(double v, double c, float oh, float ol) {
  float vh, vl;
  split_hl(__dsub_rn(v, c), vh, vl);
  return to_local(vh, vl, oh, ol);
}
// Squared distance from a local point to the box [lo, hi].
__device__ __forceinline__ float box_dist2(float y0, float y1, float y2, const float (&lo)[3],
                                           const float (&hi)[3]) {
  const float e0 = fmaxf(fmaxf(__fsub_rn(lo[0], y0), __fsub_rn(y0, hi[0])), 0.f);
  const float e1 = fmaxf(fmaxf(__fsub_rn(lo[1], y1), __fsub_rn(y1, hi[1])), 0.f);
  const float e2 = fmaxf(fmaxf(__fsub_rn(lo[2], y2), __fsub_rn(y2, hi[2])), 0.f);
  return __fmaf_rn(e0, e0, __fmaf_rn(e1, e1, __fmul_rn(e2, e2)));
}
// |r|^2 of a pair from its local difference.
__device__ __forceinline__ float pair_r2(float d0, float d1, float d2) {
  return __fmaf_rn(d0, d0, __fmaf_rn(d1, d1, __fmul_rn(d2, d2)));
}
// A staged source is a candidate for near pairs of an item unless its box
// distance reaches alpha h_j; a candidate pair is near when |r|^2 < (alpha h_j)^2.
__device__ __forceinline__ bool is_candidate(float bd2, float hh) { return !(bd2 >= hh); }
__device__ __forceinline__ bool is_near(float r2, float hh) { return r2 < hh; }

// 1/sqrt(x) by the hardware approximation (rsqrt.approx, relative error below
// 2^-22), with subnormal inputs flushed to zero.  The plain rsqrtf() keeps
// subnormals and pays for it with extra instructions around every call; the
// callers pass |r|^2 of pairs that are not near, which is at least
// (alpha h_j)^2 >= FLT_MIN, or +inf for pairs taken out of a sum.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Knuth two-sum accumulation of a partial into (hi, lo).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p) {
  float s = __fadd_rn(hi, p);
  float bb = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// The kernel products of a near pair in FP32 from its unit vector e = d/|r|
// and 1/|r| (q and psi carry the weight and kernel constant):
//   SL: (q + e (e.q)) / r      DL: e (e.psi)(e.n) / r^2
__device__ __forceinline__ float3 near_products(float ex, float ey, float ez, float ri, float4 q,
                                                float4 n, float4 p, int kind) {
  float3 c = make_float3(0.f, 0.f, 0.f);
  if (kind & K_SL) {
    const float eq = fmaf(ex, q.x, fmaf(ey, q.y, ez * q.z));
    c.x = fmaf(ex, eq, q.x) * ri;
    c.y = fmaf(ey, eq, q.y) * ri;
    c.z = fmaf(ez, eq, q.z) * ri;
  }
  if (kind & K_DL) {
    const float ep = fmaf(ex, p.x, fmaf(ey, p.y, ez * p.z));
    const float en = fmaf(ex, n.x, fmaf(ey, n.y, ez * n.z));
    const float cc = (ep * en) * (ri * ri);
    c.x = fmaf(ex, cc, c.x);
    c.y = fmaf(ey, cc, c.y);
    c.z = fmaf(ez, cc, c.z);
  }
  return c;
}

// A near pair whose r^2 in FP32 falls outside (1e-30, 1e30), where the FP32
// unit vector could underflow or the estimate overflow: 1/|r| and the unit
// vector from the FP64 values.  Out of line, so that its FP64 work runs only
// for such a pair (predicated into the common path it would hold the FP64
// pipe for every pair).
static __device__ __noinline__ float3 near_contrib_extreme(const double *x, const double *y, float4 q,
                                                    float4 n, float4 p, int kind) {
  const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  const double rid = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
  return near_products(f64_to_f32_rn(dx * rid), f64_to_f32_rn(dy * rid), f64_to_f32_rn(dz * rid),
                       f64_to_f32_rn(rid), q, n, p, kind);
}

// Near pair (|x - y| < alpha h_y): the difference x - y in FP64 from the FP64
// positions and 1/|r| to FP32 rounding from the FP64 r^2 (one Newton step on
// the FP32 estimate, its residual in FP64); the kernel products in FP32,
// written through the unit vector so that they stay in range however close
// the pair is (near_products).  Returns false for a pair at zero distance (no
// contribution).
__device__ __forceinline__ bool near_contrib(const double *x, const double *y, float4 q,
                                             float4 n, float4 p, int kind, float (&c)[3]) {
  // The FP64 instructions below run on GB300's FP64 pipe (1/64 of the FP32
  // rate), so there are as few as the FP64 difference and 1/|r| allow: 3
  // DADD, 3 for r^2, 2 for the Newton residual; the conversions run on the
  // integer pipe.
  const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  const float fx = f64_to_f32_rn(dx), fy = f64_to_f32_rn(dy), fz = f64_to_f32_rn(dz);
  if (fx == 0.f && fy == 0.f && fz == 0.f) return false;  // coincident (to 1e-45)
  const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
  float3 v;
  if (r2f > 1e-30f && r2f < 1e30f) {
    // One Newton step on the FP32 estimate y0 = rsqrt(r^2 in FP32):
    // 1/|r| = y0 (1 + e/2 + 3e^2/8 + ...) with the residual e = 1 - r^2 y0^2
    // (|e| < 2^-21), which cancels and so is formed in FP64 from the FP64
    // r^2; e/2 then needs only FP32, and the dropped 3e^2/8 < 2^-43.
    const double r2 = dx * dx + dy * dy + dz * dz;
    const float y0f = rsqrt_ftz(r2f);
    const double y0 = f32_to_f64(y0f);
    const float ri = fmaf(0.5f * y0f, f64_to_f32_rn(fma(-r2, y0 * y0, 1.0)), y0f);
    v = near_products(fx * ri, fy * ri, fz * ri, ri, q, n, p, kind);
  } else {
    v = near_contrib_extreme(x, y, q, n, p, kind);
  }
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
  return true;
}

__device__ __forceinline__ void set_error(int32_t *flag, int code) {
  if (flag) atomicCAS(flag, 0, code);
}

}  // namespace stk
