// BF16 tensor-core GEMM (tcgen05 + TMEM accumulators, operands staged by TMA)
// for the model's Linear layers and their adjoints in BF16 mode.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace edpc {

// Epilogue modes.
//   TC_PLAIN     v = acc (+ bias[n]) (+ R[m][n]); writes C (FP32), Cb (BF16,
//                row-major) and CbT (BF16, transposed [n][m]) when non-null.
//   TC_BRANCH    MBRB Eqs. 10-12: the N tile holds the same 32 hidden units of
//                each of the k branches (B is loaded in k sections of 32 rows).
//                X_i = acc_i + bias[i*H + h] is stored to C (FP32, [m][i*H+h]);
//                G = GELU(prod_i X_i) goes to Cb ([m][h]) and CbT ([h][m]).
//   TC_BRANCH_BWD adjoint of Eqs. 11-12 on dG = acc: with X_i read from Aux
//                ([m][i*H+h]), dX_i = dG * GELU'(prod X) * prod_{l!=i} X_l is
//                stored to C (FP32), Cb (BF16) and CbT (BF16, [i*H+h][m]).
enum TcMode { TC_PLAIN = 0, TC_BRANCH = 1, TC_BRANCH_BWD = 2 };

// C[m][n] = sum_k A[m][k] B[n][k] (+ epilogue); A is M x K and B is N x K,
// both BF16 (or both FP8 e4m3 with power-of-two per-tensor scales) and
// K-contiguous; accumulation is FP32 in TMEM.
struct TcGemm {
  CUtensorMap ta;  // A: box 128 bytes of K x 128 (M), 128-byte swizzle
  CUtensorMap tb;  // B: box 128 bytes of K x bn (N) (TC_BRANCH: x 32 per section)
  int M = 0, N = 0, K = 0;
  int bn = 64;     // N tile: 32, 64 or 128 (TC_BRANCH: 32 * k); must equal tb's box rows
  int box_b = 0;   // rows of tb's box, recorded by the plan (checked at launch)
  int mode = TC_PLAIN;
  int H = 0, k = 1;        // TC_BRANCH / TC_BRANCH_BWD: hidden width and branch count
  float* C = nullptr;
  int ldc = 0;
  __nv_bfloat16* Cb = nullptr;
  int ldcb = 0;
  __nv_bfloat16* CbT = nullptr;
  int ldct = 0;
  const float* bias = nullptr;
  const float* R = nullptr;
  int ldr = 0;
  const float* Aux = nullptr;
  int ldaux = 0;
  int* err = nullptr;  // set to kErrTcTimeout if a bounded wait expired
  bool fp8 = false;    // operands are e4m3; acc is multiplied by inv_a[0] * inv_b[0]
  bool b_early = true; // B was written two or more launches back: prefetch it before the PDL wait
  const float* inv_a = nullptr;
  const float* inv_b = nullptr;
};

constexpr int kErrTcTimeout = 4;

// Tensor map of a row-major BF16 matrix [rows][cols] with row stride ld
// elements, for boxes of 64 columns x box_rows rows. Returns 0 or an EDPC code.
int make_tmap_bf16(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint32_t box_rows);
// The same for a byte matrix (FP8 e4m3) with row stride ld bytes and boxes of
// 128 columns x box_rows rows.
int make_tmap_u8(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows);

cudaError_t launch_gemm_tc(const TcGemm& g, cudaStream_t st);

// One tcgen05 GEMM per call site of the step (maps are bound to fixed buffers).
struct TcPlan {
  static constexpr int kMaxSites = 8 * kMaxBlocks + 16;
  TcGemm site[kMaxSites];
  bool ready = false;
};

}  // namespace edpc
