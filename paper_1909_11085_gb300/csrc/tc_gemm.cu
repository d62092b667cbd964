// tc_gemm.cu -- the three-term TF32 product of tc_gemm.cuh on the tensor
// cores: A streamed by TMA tile loads (128 rows x 128 bytes per chunk, landing
// in the 128-byte swizzle), split into TF32 hi + lo in shared memory, B tiles
// from the caller's table by bulk copies, tcgen05.mma into tensor memory.
#include "tc_gemm.cuh"

namespace stk {
namespace tc {
namespace {

constexpr int kThreads = 256;
constexpr int kRawStages = 4;   // A chunks in flight (FP32)
constexpr int kTileStages = 2;  // split A + B chunks ready for the MMAs
constexpr int kSplitters = 128;
constexpr int kRawBytes = kRows * kChunk * 4;          // 16 KB
constexpr int kBHalf = kCols * kChunk * 4;             // 8 KB: B hi or lo
constexpr int kTileBytes = 2 * kRawBytes + 2 * kBHalf;  // A hi, A lo, B hi, B lo
constexpr int kNumBars = 2 * kRawStages + 3 * kTileStages + 1;
constexpr size_t kSmem = 1024 + (size_t)kRawStages * kRawBytes + (size_t)kTileStages * kTileBytes +
                         8 * kNumBars + 16;
constexpr uint32_t kTmemCols = 2 * kCols;  // [0, 64): hi.hi + lo.hi, [64, 128): hi.lo
constexpr int kErrTimeout = 4;
static_assert(kRawBytes % 1024 == 0 && kTileBytes % 1024 == 0, "1024-byte aligned stages");

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity, int64_t limit) {
  if (try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void fail(const Args &g) {
  if (g.err) atomicCAS(g.err, 0, kErrTimeout);
}
__device__ __forceinline__ void arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   saddr(bar))
               : "memory");
}
__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// K-major, 128-byte swizzle, 8-row groups 1024 bytes apart, version 1.
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// Roles: warps 0-3 split A chunks (FP32 -> TF32 hi + lo, same swizzled
// offsets); thread 128 issues the copies (A tile loads, B bulk copies); thread
// 160 issues the MMAs; warps 4-7 then read the accumulators (one lane quarter
// each) and write D.  Every wait is bounded: on expiry the role records
// STK_ETIMEOUT and stops; the copies issued and the MMAs committed are waited
// for (bounded) before tensor memory is freed.
__global__ void __launch_bounds__(kThreads, 1) k_gemm3(const __grid_constant__ CUtensorMap amap,
                                                       const Args g) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *base = smem + ((1024u - (saddr(smem) & 1023u)) & 1023u);
  unsigned char *raw = base;                                   // [kRawStages][kRawBytes]
  unsigned char *tile = raw + (size_t)kRawStages * kRawBytes;  // [kTileStages][kTileBytes]
  uint64_t *bars = reinterpret_cast<uint64_t *>(tile + (size_t)kTileStages * kTileBytes);
  uint64_t *raw_full = bars, *raw_empty = raw_full + kRawStages;
  uint64_t *tile_full = raw_empty + kRawStages, *b_full = tile_full + kTileStages;
  uint64_t *tile_empty = b_full + kTileStages, *done = tile_empty + kTileStages;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kNumBars);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t row0 = (int32_t)blockIdx.x * kRows;
  const int nk = g.k_chunks;
  if (tid == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&raw_full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&raw_empty[s])),
                   "r"(kSplitters)
                   : "memory");
    }
    for (int s = 0; s < kTileStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&tile_full[s])),
                   "r"(kSplitters)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&b_full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&tile_empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp < 4) {
    // ----------------------------------------------------------- splitters
    for (int c = 0; c < nk; ++c) {
      const int rs = c % kRawStages, ts = c % kTileStages;
      if (!wait(&raw_full[rs], (uint32_t)((c / kRawStages) & 1), g.spin_limit) ||
          (c >= kTileStages &&
           !wait(&tile_empty[ts], (uint32_t)(((c / kTileStages) - 1) & 1), g.spin_limit))) {
        fail(g);
        break;
      }
      const float4 *src = reinterpret_cast<const float4 *>(raw + (size_t)rs * kRawBytes);
      float4 *hi = reinterpret_cast<float4 *>(tile + (size_t)ts * kTileBytes);
      float4 *lo = hi + kRawBytes / 16;
#pragma unroll
      for (int j = 0; j < kRawBytes / 16 / kSplitters; ++j) {
        const int e = tid + kSplitters * j;  // the same swizzled offset in every tile
        const float4 v = src[e];
        const float4 h = make_float4(tf32(v.x), tf32(v.y), tf32(v.z), tf32(v.w));
        hi[e] = h;
        lo[e] = make_float4(tf32(v.x - h.x), tf32(v.y - h.y), tf32(v.z - h.z), tf32(v.w - h.w));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      arrive(&tile_full[ts]);
      arrive(&raw_empty[rs]);
    }
  } else if (tid == 128) {
    // ------------------------------------------------------------ copies
    int issued = 0;
    for (int c = 0; c < nk; ++c) {
      const int rs = c % kRawStages, ts = c % kTileStages;
      if (c >= kRawStages &&
          !wait(&raw_empty[rs], (uint32_t)(((c / kRawStages) - 1) & 1), g.spin_limit)) {
        fail(g);
        break;
      }
      expect(&raw_full[rs], kRawBytes);
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(raw + (size_t)rs * kRawBytes)),
          "l"(reinterpret_cast<uint64_t>(&amap)), "r"(c * kChunk),
          "r"((int32_t)(g.a_row0 + row0)), "r"(saddr(&raw_full[rs]))
          : "memory");
      if (c >= kTileStages &&
          !wait(&tile_empty[ts], (uint32_t)(((c / kTileStages) - 1) & 1), g.spin_limit)) {
        fail(g);
        issued = -(c + 1);  // chunk c: A issued, B not
        break;
      }
      expect(&b_full[ts], 2 * kBHalf);
      const float *bsrc = g.btab + ((size_t)blockIdx.y * nk + c) * 2 * kCols * kChunk;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
              "r"(saddr(tile + (size_t)ts * kTileBytes + 2 * kRawBytes)),
          "l"(bsrc), "r"(2 * kBHalf), "r"(saddr(&b_full[ts]))
          : "memory");
      issued = c + 1;
    }
    // every copy issued has landed before the CTA goes on (at once where the
    // splitters and the MMAs consumed them)
    const int na = issued < 0 ? -issued : issued, nb = issued < 0 ? -issued - 1 : issued;
    for (int c = (na > kRawStages ? na - kRawStages : 0); c < na; ++c)
      if (!wait(&raw_full[c % kRawStages], (uint32_t)((c / kRawStages) & 1), g.spin_limit)) fail(g);
    for (int c = (nb > kTileStages ? nb - kTileStages : 0); c < nb; ++c)
      if (!wait(&b_full[c % kTileStages], (uint32_t)((c / kTileStages) & 1), g.spin_limit)) fail(g);
  } else if (tid == 160) {
    // --------------------------------------------------------------- MMAs
    // D F32, A and B TF32, K-major, M = 128; N = 128 (B hi then B lo) or 64
    const uint32_t id128 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * kCols >> 3) << 17) |
                           ((uint32_t)(kRows >> 4) << 24);
    const uint32_t id64 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kCols >> 3) << 17) |
                          ((uint32_t)(kRows >> 4) << 24);
    bool ok = true;
    int last = -1;
    for (int c = 0; c < nk; ++c) {
      const int ts = c % kTileStages;
      const uint32_t par = (uint32_t)((c / kTileStages) & 1);
      if (!wait(&tile_full[ts], par, g.spin_limit) || !wait(&b_full[ts], par, g.spin_limit)) {
        fail(g);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = saddr(tile + (size_t)ts * kTileBytes), al = ah + kRawBytes;
      const uint32_t bh = ah + 2 * kRawBytes;
#pragma unroll
      for (int ks = 0; ks < kChunk / 8; ++ks) {
        const uint32_t kb = 32u * ks;
        mma(tmem, desc(ah + kb), desc(bh + kb), id128, (c > 0 || ks > 0) ? 1u : 0u);
        mma(tmem, desc(al + kb), desc(bh + kb), id64, 1u);
      }
      commit(&tile_empty[ts]);
      last = c;
    }
    if (ok) {
      commit(done);
    } else if (last >= 0 &&
               !wait(&tile_empty[last % kTileStages], (uint32_t)((last / kTileStages) & 1),
                     g.spin_limit)) {
      fail(g);
    }
  }
  if (warp >= 4) {
    // ----------------------------------------------------------- epilogue
    __syncwarp();
    const bool fin = wait(done, 0, g.spin_limit);
    if (!fin && lane == 0) fail(g);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__all_sync(0xffffffffu, fin)) {
      const int quarter = warp & 3;
      const int32_t r = row0 + quarter * 32 + lane;
      float d[kCols];
#pragma unroll
      for (int part = 0; part < 2 * kCols / 16; ++part) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(part * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int col = part * 16 + e;
          if (col < kCols)
            d[col] = __uint_as_float(v[e]);
          else
            d[col - kCols] += __uint_as_float(v[e]);
        }
      }
      if (r < g.m) {
        float *o = g.out + (size_t)r * g.ldo;
        const int c0 = (int)blockIdx.y * kCols;
#pragma unroll
        for (int c = 0; c < kCols; ++c)
          if (c0 + c < g.n) o[c0 + c] = d[c];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library does not link libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

}  // namespace

cudaError_t encode_a(CUtensorMap *map, const float *a, uint64_t rows, uint64_t k, uint64_t ld) {
  const EncodeTiledFn f = encode_tiled();
  if (!f) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a) & 15) != 0 || (ld & 3) != 0 || k > ld || rows == 0 || k == 0)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {k, rows};
  const cuuint64_t strides[1] = {ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)kRows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = f(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a), dims,
                       strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t gemm3(const CUtensorMap &a_map, const Args &g, cudaStream_t st) {
  if (g.m <= 0 || g.n_tiles <= 0) return cudaSuccess;
  if (g.k_chunks <= 0 || !g.btab || !g.out) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_gemm3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((g.m + kRows - 1) / kRows), (unsigned)g.n_tiles);
  k_gemm3<<<grid, kThreads, kSmem, st>>>(a_map, g);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace stk
