// engine_fp64.cu -- FP64 evaluation of the Stokes single- and double-layer
// sums (Eq. "sl_stokes", the double-layer kernel of Sec. 2.1, summed as in
// Sec. 3.1).  Same work items as the mixed engine: a warp holds up to 128
// targets (T per lane) and walks the item's source segments; sources are
// 96-byte FP64 records read with warp-uniform (broadcast) loads.  On GB300
// the FP64 pipe issues about 1/64 of the FP32 rate, so this path is bound by
// DFMA throughput; it is the accuracy reference form on the GPU.
#include "common.cuh"
#include "prep.cuh"

namespace stk {

template <int T, int KIND>
__device__ __forceinline__ void seg64(const SrcRec64 *__restrict__ rec, int64_t s, int64_t e,
                                      int sg, int b, const double (&x)[T][3],
                                      double (&acc)[T][3]) {
  for (int64_t k = s + sg; k < e; k += b) {
    const SrcRec64 &R = rec[k];
    const double yx = R.y[0], yy = R.y[1], yz = R.y[2];
    double qx = 0, qy = 0, qz = 0, nx = 0, ny = 0, nz = 0, px = 0, py = 0, pz = 0;
    if (KIND & K_SL) { qx = R.q[0]; qy = R.q[1]; qz = R.q[2]; }
    if (KIND & K_DL) {
      nx = R.n[0]; ny = R.n[1]; nz = R.n[2];
      px = R.p[0]; py = R.p[1]; pz = R.p[2];
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const double dx = x[t][0] - yx, dy = x[t][1] - yy, dz = x[t][2] - yz;
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double ri = r2 > 0.0 ? rsqrt(r2) : 0.0;  // zero-distance pair contributes nothing
      const double ri2 = ri * ri;
      if (KIND == K_SL) {
        const double c = (dx * qx + dy * qy + dz * qz) * ri2;
        acc[t][0] += (qx + dx * c) * ri;
        acc[t][1] += (qy + dy * c) * ri;
        acc[t][2] += (qz + dz * c) * ri;
      } else if (KIND == K_DL) {
        const double c = (dx * px + dy * py + dz * pz) * (dx * nx + dy * ny + dz * nz) *
                         (ri2 * ri2 * ri);
        acc[t][0] += dx * c;
        acc[t][1] += dy * c;
        acc[t][2] += dz * c;
      } else {
        const double dq = dx * qx + dy * qy + dz * qz;
        const double dp = dx * px + dy * py + dz * pz;
        const double dn = dx * nx + dy * ny + dz * nz;
        const double c = (dq + dp * dn * ri2) * ri2;
        acc[t][0] += (qx + dx * c) * ri;
        acc[t][1] += (qy + dy * c) * ri;
        acc[t][2] += (qz + dz * c) * ri;
      }
    }
  }
}

template <int T>
__device__ void run_item64(const EngineParams &P, const Item &it, int b, int lane) {
  const int G = kWarp / b, tgl = lane % G, sg = lane / G;
  const int tn = it.tn_part & 0xFF, part = it.tn_part >> 8;
  double x[T][3], acc[T][3];
  bool valid[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int li = tgl + G * t;
    valid[t] = li < tn;
    const int gi = it.t0 + (valid[t] ? li : 0);
    const int ci = P.tperm ? P.tperm[gi] : gi;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      x[t][k] = valid[t] ? P.trg64[3 * (size_t)ci + k] : 1e300;
      acc[t][k] = 0.0;
    }
  }
  for (int e = it.seg0; e < it.seg1; ++e) {
    const int sid = P.seg_list ? P.seg_list[e] : e;
    const int64_t s = P.range_ptr[sid], en = P.range_ptr[sid + 1];
    const int kind = seg_kind(P, sid);
    if (kind == K_SL)
      seg64<T, K_SL>(P.rec64, s, en, sg, b, x, acc);
    else if (kind == K_DL)
      seg64<T, K_DL>(P.rec64, s, en, sg, b, x, acc);
    else
      seg64<T, K_SLDL>(P.rec64, s, en, sg, b, x, acc);
  }
  for (int o = G; o < kWarp; o <<= 1)
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[t][k] += __shfl_xor_sync(kFull, acc[t][k], o);
  if (sg == 0) {
    double *out = P.part_out + ((size_t)part * (size_t)P.nt + (size_t)it.t0) * 3;
#pragma unroll
    for (int t = 0; t < T; ++t)
      if (valid[t]) {
        const int li = tgl + G * t;
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * li + k] = acc[t][k];
      }
  }
}

__global__ void __launch_bounds__(kWarpsPerCta *kWarp, 4) k_engine_fp64(EngineParams P) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int n_items = *P.n_items;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(P.item_counter, 1);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= n_items) break;
    const int id = P.item_order ? P.item_order[idx] : idx;
    const Item it = P.items[id];
    const int tn = it.tn_part & 0xFF;
    if (P.policy == 1) {
      if (tn <= 32)
        run_item64<1>(P, it, 1, lane);
      else if (tn <= 64)
        run_item64<2>(P, it, 1, lane);
      else if (tn <= 96)
        run_item64<3>(P, it, 1, lane);
      else
        run_item64<4>(P, it, 1, lane);
    } else if (tn <= 8)
      run_item64<1>(P, it, 4, lane);
    else if (tn <= 16)
      run_item64<2>(P, it, 4, lane);
    else if (tn <= 24)
      run_item64<3>(P, it, 4, lane);
    else if (tn <= 32)
      run_item64<4>(P, it, 4, lane);
    else if (tn <= 48)
      run_item64<3>(P, it, 2, lane);
    else if (tn <= 64)
      run_item64<4>(P, it, 2, lane);
    else if (tn <= 96)
      run_item64<3>(P, it, 1, lane);
    else
      run_item64<4>(P, it, 1, lane);
  }
}

cudaError_t launch_engine_fp64(const EngineParams &P, int grid, cudaStream_t stream) {
  k_engine_fp64<<<grid, kWarpsPerCta * kWarp, 0, stream>>>(P);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t engine_fp64_occupancy(int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_engine_fp64,
                                                       kWarpsPerCta * kWarp, 0);
}

}  // namespace stk
