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
  int bn = 64;     // N tile: 32, 64, 128 or 256 (TC_BRANCH: k * section, section 32, 64 or 128)
  int box_b = 0;   // rows of tb's box, recorded by the plan (checked at launch): bn, or
                   // the section width in TC_BRANCH mode
  // Split-K (TC_PLAIN with no bias, residual or BF16 outputs): grid.z = splitk
  // CTAs per output tile each take a contiguous range of K blocks and write
  // their FP32 partial tile to ws ([splitk][M][N]); the last CTA of a tile to
  // arrive (counter cnt[tile], zero between launches) adds the partials in
  // split order and writes C. Launches that share ws and cnt must not overlap.
  int splitk = 1;
  float* ws = nullptr;
  unsigned* cnt = nullptr;
  // Persistent kernel: one CTA per SM walks the output tiles, with two TMEM
  // accumulators so that a tile's epilogue overlaps the next tile's MMAs.
  // Same K order and epilogue arithmetic as the one-tile kernel, so the
  // results are identical for the same bn.
  bool persistent = false;
  // Output tensor maps (FP32 C and BF16 Cb, boxes of 32 x 32, built by
  // tc_build_out_maps when the outputs are 16-byte aligned): whole 32 x 32
  // chunks are written by TMA stores from shared memory.
  CUtensorMap tmc, tmcb;
  bool has_tmc = false, has_tmcb = false;
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
  // Grouped mode (independent per-file models; BF16, one-tile kernel only):
  //   mt  forward / dX GEMMs: nmt M tiles {m0, m_end, group, 0}: the tile
  //       covers rows [m0, m_end) (rows from m_end to m0 + 128 belong to the
  //       next group and are neither stored nor read back); tb is a 3-D map
  //       over the groups' B matrices (group coordinate z) and the bias of
  //       the tile's group starts at bias + group * gs.
  //   gk  weight-gradient GEMMs (K = streams): ngk groups {k0, nkb, 0, 0}:
  //       grid.z runs over the groups, group g contracts K elements
  //       [k0, k0 + 64 nkb) and writes C + g * gs.
  const int4* mt = nullptr;
  int nmt = 0;
  const int4* gk = nullptr;
  int ngk = 0;
  size_t gs = 0;
};

constexpr int kErrTcTimeout = 4;

// Tensor map of a row-major BF16 matrix [rows][cols] with row stride ld
// elements, for boxes of 64 columns x box_rows rows. Returns 0 or an EDPC code.
int make_tmap_bf16(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint32_t box_rows);
// The same for a byte matrix (FP8 e4m3) with row stride ld bytes and boxes of
// 128 columns x box_rows rows.
int make_tmap_u8(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows);
// A 3-D BF16 map over `groups` row-major matrices [rows][cols] (row stride ld
// elements), matrix g at base + g * gstride elements, boxes of 64 columns x
// box_rows rows of one matrix.
int make_tmap_bf16_groups(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                          uint64_t groups, uint64_t gstride, uint32_t box_rows);

cudaError_t launch_gemm_tc(const TcGemm& g, cudaStream_t st);
// The persistent kernel (g.persistent), dispatched by launch_gemm_tc.
cudaError_t launch_gemm_tcp(const TcGemm& g, cudaStream_t st);

// Builds g's output tensor maps (C over its logical columns: N for TC_PLAIN,
// k * H for the branch modes; Cb likewise, H for TC_BRANCH). Returns 0 or an
// EDPC code; an unaligned output simply gets no map.
int tc_build_out_maps(TcGemm* g);

// Split-K factor of a TC_PLAIN GEMM with an N tile of bn: up to about 64 CTAs
// in all (the split GEMMs run on a side stream beside the step's critical
// path), at least 8 K blocks (of 64) per CTA, at most 32 splits.
int tc_splitk(int M, int N, int K, int bn);
// Output tiles of a launch (the size of its counter array when split).
inline int tc_tiles(int M, int N, int bn) { return ((M + 127) / 128) * ((N + bn - 1) / bn); }

// One tcgen05 GEMM per call site of the step (maps are bound to fixed buffers).
struct TcPlan {
  static constexpr int kMaxSites = 8 * kMaxBlocks + 16;
  TcGemm site[kMaxSites];
  bool ready = false;
};

}  // namespace edpc
