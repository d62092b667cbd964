// common.cuh -- types and device helpers shared by the library's kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace stk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarp = 32;
constexpr int kChunk = 64;      // sources staged per chunk (one bulk copy)
constexpr int kItemMax = 128;   // targets per work item (32 lanes x 4)
constexpr int kQCap = 16;       // near-pair queue entries per lane
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
  double *part_out;          // [nparts][nt][3], sorted target order
  int32_t *item_counter;     // work queue head (zeroed before launch)
  int32_t *err_flag;         // device error word
  int64_t spin_limit;        // bounded mbarrier waits, in SM clock cycles
};

__device__ __forceinline__ int seg_kind(const EngineParams &P, int32_t sid) {
  return P.kind_alternating ? ((sid & 1) ? K_DL : K_SL) : P.kind;
}

// Exact-enough split of (x - c) into two floats; used identically for
// sources and targets so that coincident points get bit-identical local
// coordinates.
__device__ __forceinline__ void split_hl(double v, float &hi, float &lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}
__device__ __forceinline__ float to_local(float vh, float vl, float oh, float ol) {
  return __fadd_rn(__fsub_rn(vh, oh), __fsub_rn(vl, ol));
}

// Knuth two-sum accumulation of a partial into (hi, lo).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p) {
  float s = __fadd_rn(hi, p);
  float bb = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ void set_error(int32_t *flag, int code) {
  if (flag) atomicCAS(flag, 0, code);
}

}  // namespace stk
