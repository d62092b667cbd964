// prep.cuh -- host-side launchers for the staging kernels and the engines.
#pragma once

#include "common.cuh"

namespace stk {

// Kernels launched by the calling thread through the library.
int64_t launch_count();
void count_launches(int n);

void launch_pack_mixed(int64_t ns, const double *src, const double *f, const double *nrm,
                       const double *phi, const double *w, const double *h, double alpha,
                       double csl, double cdl, const double *cen, SrcRec *rec, cudaStream_t st);
void launch_pack_fp64(int64_t ns, const double *src, const double *f, const double *nrm,
                      const double *phi, const double *w, double csl, double cdl, SrcRec64 *rec,
                      cudaStream_t st);
int bbox_partial_blocks(int64_t n);
void launch_bbox(int64_t n, const double *pts, double *partial, double *box, cudaStream_t st);
void launch_morton(int64_t n, const double *pts, const double *box, const int64_t *group_ptr,
                   int32_t ngroup, uint64_t *keys, int32_t *vals, cudaStream_t st);
void launch_scan(const int32_t *in, int64_t n, int32_t *out, int32_t *total, cudaStream_t st);
size_t radix_hist_entries(int64_t n);
int radix_sort(uint64_t *ka, int32_t *va, uint64_t *kb, int32_t *vb, int64_t n, int bits,
               int32_t *hist, int32_t *hist_scan, cudaStream_t st);
void launch_items_direct(int32_t nt, int64_t ns, int32_t nsplit, int32_t item_max, Item *items,
                         int64_t *range_ptr, int32_t *n_items, cudaStream_t st);
void launch_p2p_items(int32_t nleaf, const int32_t *leaf_ptr, const int32_t *ulist_ptr,
                      const int32_t *ulist_idx, int32_t item_max, int32_t *cnt, int32_t *offs,
                      int32_t *n_items, Item *items, uint64_t *keys, int32_t *vals,
                      cudaStream_t st);
void launch_batched_items(int32_t nsusp, const int64_t *susp_ptr, const int64_t *n_cell,
                          int32_t item_max, int32_t *cnt, int32_t *offs, int32_t *n_items,
                          Item *items, int64_t *range_ptr, uint64_t *keys, int32_t *vals,
                          cudaStream_t st);
// Item order by descending cost bucket (keys from the item builders; vals < 0
// marks unused slots); cnt and off hold 256 entries, rank and order n.
void launch_bucket_order(int64_t n, const uint64_t *keys, const int32_t *vals, int32_t *cnt,
                         int32_t *off, int32_t *rank, int32_t *order, cudaStream_t st);
// Near pairs of the mixed engine's items (near.cu); runs after the engine.
void launch_near(const EngineParams &P, int sms, int64_t max_items, cudaStream_t st);
// Small direct sums (direct_small.cu): one launch over blocks of targets x
// source splits writing part[split][target][3] (an FP32 (hi, lo) pair in
// each double's bytes); the last split of each block
// (counter blocks[block], zero before the launch and left zero) writes out.
constexpr int64_t kSmallPairs = (int64_t)1 << 26;  // targets x sources taking this form
int64_t direct_small_blocks(int64_t nt);
int direct_small_splits(int64_t ns, int64_t nt, int sms);
cudaError_t launch_direct_small(int kinds, const double *src, const double *f, const double *nrm,
                                const double *phi, const double *w, const double *h, int64_t ns,
                                const double *trg, int64_t nt, double alpha, double csl,
                                double cdl, int32_t nsplit, int32_t accumulate, double *part,
                                int32_t *blocks, double *out, cudaStream_t st);
void launch_finish(int64_t nt, int32_t nparts, const double *part_out, const int32_t *tperm,
                   int32_t accumulate, double *out, cudaStream_t st);
void launch_zero_ints(int32_t *p, int n, cudaStream_t st);
void launch_widen(int64_t n, const int32_t *in, int64_t *out, cudaStream_t st);

// Adjoint passes (adjoint.cu).
struct AdjParams {
  const void *out_rec;     // records of the output points (SrcRec or SrcRec64), caller order
  const void *in_rec;      // records of the input points
  const int32_t *operm;    // sorted -> caller index of the output points
  const int32_t *iperm;    // sorted -> caller index of the input points
  int64_t nout, nin;
  int32_t nsplit;
  int32_t has_sl, has_dl;
  const double *out64;     // caller FP64 positions of the output points
  const double *in64;      // caller FP64 positions of the input points
  double *partial;         // [nsplit][nout][12 or 3], caller order
  // mixed form: near pairs per output point (caller order), filled by the FP32
  // pass and evaluated in FP64 by k_adj_near
  int32_t *near_cnt;       // [nout], zeroed before the FP32 pass
  int32_t *near_idx;       // [nout][near_cap] input caller indices
  int32_t near_cap;
  float *oframe;           // [nout][9]: local coordinates and the CTA frame origin (hi, lo)
};
cudaError_t launch_adjoint(bool mixed, bool src_major, const AdjParams &A, cudaStream_t st);
constexpr int32_t kAdjNearCap = 32;  // near pairs listed per output point
void launch_adj_finish(bool src_major, int64_t n, int32_t nsplit, const double *part,
                       const double *w, double csl, double cdl, double *grad_f, double *grad_phi,
                       double *grad_n, double *grad_y, double *grad_x, cudaStream_t st);

size_t engine_mixed_smem_bytes();
cudaError_t launch_engine_mixed(const EngineParams &P, int grid, cudaStream_t stream);
cudaError_t engine_mixed_occupancy(int *blocks_per_sm);
cudaError_t launch_engine_fp64(const EngineParams &P, int grid, cudaStream_t stream);
cudaError_t engine_fp64_occupancy(int *blocks_per_sm);

}  // namespace stk
