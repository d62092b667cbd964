// fmm_fast.cuh -- launch sequence of the CTA-blocked mixed far field
// (fmm_fast.cu) and the per-launch event hooks the far-field entry point
// offers for timing its passes.
#pragma once

#include <cuda_runtime.h>

#include "fmm_passes.cuh"

namespace stk {
namespace fmm {

constexpr int kFastMaxP = 8;  // the blocked mixed kernels take surfaces of order p <= 8

// While events != NULL, launch k of a far-field call records events[2k] before
// and events[2k + 1] after it on the call's stream (k < capacity / 2), names[k]
// receives the pass's name and *count the launches recorded.
struct FastHooks {
  cudaEvent_t *events = nullptr;
  int32_t capacity = 0;
  const char **names = nullptr;
  int32_t *count = nullptr;
  void before(int k, const char *name, cudaStream_t st) const {
    if (!events || 2 * k + 1 >= capacity) return;
    cudaEventRecord(events[2 * k], st);
    if (names) names[k] = name;
  }
  void after(int k, cudaStream_t st) const {
    if (!events || 2 * k + 1 >= capacity) return;
    cudaEventRecord(events[2 * k + 1], st);
    if (count) *count = k + 1;
  }
};

cudaError_t far_field_fast(const Pass &P, const int32_t *depth_ptr, int32_t max_depth, int sms,
                           cudaStream_t st, const FastHooks &hooks);

}  // namespace fmm
}  // namespace stk
