// Tensor-core (tcgen05, kind::tf32) real GEMM with split-precision operands:
//   C[m][n] = sum_k A[m][k] B[n][k],  A = Ahi + Alo, B = Bhi + Blo (TF32 pairs),
//   evaluated as Ahi.Bhi + Ahi.Blo + Alo.Bhi with FP32 accumulation in TMEM
//   (the lo.lo term is below FP32 resolution; Ootomo & Yokota, IJHPCA 2022).
// Operands are K-major FP32 arrays padded to the tile sizes (rows to 128,
// K to 32) and staged into shared memory by TMA with 128-byte swizzle; one
// elected thread issues the MMAs; four warps drain the accumulator.  Every
// mbarrier wait is bounded: on time-out the kernel records an error code,
// waits (bounded) for its own copies in flight, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qe {

constexpr int TC_BM = 128;      // rows of A per CTA (TMEM lanes)
constexpr int TC_BN = 128;      // rows of B per CTA (TMEM columns)
constexpr int TC_BK = 32;       // K per stage: one 128-byte swizzle row of FP32
constexpr int TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;           // 16 KiB per operand tile
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;          // Ahi, Alo, Bhi, Blo
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;

// Error codes written to the status word.
enum { TC_OK = 0, TC_TIMEOUT_FULL = 1, TC_TIMEOUT_EMPTY = 2, TC_TIMEOUT_ACC = 3 };

}  // namespace qe
