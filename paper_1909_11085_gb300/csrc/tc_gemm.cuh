// tc_gemm.cuh -- a dense FP32-accurate product on the tensor cores (tcgen05,
// kind::tf32, three TF32 terms): D[M][N] = A[M][K] B[N][K]^T with A an FP32
// row-major array in global memory (K contiguous) and B a table prepared by the
// caller in the operand layout, split into TF32 hi + lo parts.  Used for the
// inverse lattice DFT of the FMM's Fourier-space M2L (Sec. 3.1, "Far
// evaluation"), a dense contraction of every box's check spectrum with the
// inverse-DFT matrix.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace stk {
namespace tc {

constexpr int kRows = 128;   // rows of A (and D) per CTA
constexpr int kCols = 64;    // columns of D per CTA (rows of a B tile)
constexpr int kChunk = 32;   // K per chunk: 128 bytes of FP32

// B table of n_tiles x k_chunks tiles: tile (t, c) holds B[t kCols + n][c kChunk + k]
// for n < kCols, k < kChunk as TF32 hi then lo, each kCols rows of 128 bytes in
// the 128-byte swizzle (piece j of row n at position j ^ (n mod 8)); missing
// rows and columns are zero.  Floats in the table:
inline size_t b_table_floats(int n_tiles, int k_chunks) {
  return (size_t)n_tiles * k_chunks * 2 * kCols * kChunk;
}
// Float offset of entry (n, k) of one tile half (n < kCols, k < kChunk).
__host__ __device__ inline uint32_t b_table_offset(int n, int k) {
  return (uint32_t)(((n >> 3) << 8) + ((n & 7) << 5) + ((((k >> 2) ^ (n & 7)) & 7) << 2) + (k & 3));
}

struct Args {
  int64_t a_row0;     // first row of A in the tensor map
  int32_t m;          // rows of D to compute (rows a_row0 .. a_row0 + m - 1)
  int32_t k_chunks;   // K / kChunk, rounded up (A's columns past K read as zero)
  int32_t n_tiles;    // B tiles along N (grid.y)
  int32_t n;          // columns of D written (< n_tiles kCols)
  const float *btab;  // the B table
  float *out;         // D[r][c] at out[r ldo + c], r < m, c < n
  int64_t ldo;
  int32_t *err;       // device error word: STK_ETIMEOUT (4) when a wait expires
  int64_t spin_limit; // SM cycles a wait may take
};

// The tensor map of A (rows x k FP32, row stride ld floats, a multiple of 4)
// for the product's loads.
cudaError_t encode_a(CUtensorMap *map, const float *a, uint64_t rows, uint64_t k, uint64_t ld);

// Launches the product on st: ceil(m / kRows) x n_tiles CTAs.
cudaError_t gemm3(const CUtensorMap &a_map, const Args &g, cudaStream_t st);

}  // namespace tc
}  // namespace stk
