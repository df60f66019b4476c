// BF16 tensor-core GEMM (tcgen05 + TMEM accumulators, operands staged by TMA)
// for the model's Linear layers and their adjoints in BF16 mode.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace edpc {

// C[m][n] = sum_k A[m][k] B[n][k] (+ bias[n]) (+ R[m][n]); A is M x K and B is
// N x K, both BF16 and K-contiguous; accumulation is FP32 in TMEM.
struct TcGemm {
  CUtensorMap ta;  // A: box 64 (K) x 128 (M), 128-byte swizzle
  CUtensorMap tb;  // B: box 64 (K) x bn (N), 128-byte swizzle
  int M = 0, N = 0, K = 0;
  int bn = 64;     // N tile: 64, 128 or 256
  float* C = nullptr;
  int ldc = 0;
  int epi = 0;     // Epi of kernels.cuh
  const float* bias = nullptr;
  const float* R = nullptr;
  int ldr = 0;
  int* err = nullptr;  // set to kErrTcTimeout if a bounded wait expired
};

constexpr int kErrTcTimeout = 4;

// Tensor map of a row-major BF16 matrix [rows][cols] with row stride ld
// elements, for boxes of 64 columns x box_rows rows. Returns 0 or an EDPC code.
int make_tmap_bf16(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint32_t box_rows);

cudaError_t launch_gemm_tc(const TcGemm& g, cudaStream_t st);

// One tcgen05 GEMM per call site of the step (maps are bound to fixed buffers).
struct TcPlan {
  static constexpr int kMaxSites = 8 * kMaxBlocks + 16;
  TcGemm site[kMaxSites];
  bool ready = false;
};

}  // namespace edpc
