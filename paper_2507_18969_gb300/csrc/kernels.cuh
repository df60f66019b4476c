// Kernel launchers of the EDPC library. Every launcher is asynchronous on
// `st` and returns the launch status.
#pragma once

#include "common.cuh"

namespace edpc {

// ---- initial values -------------------------------------------------------------------
// dst[j] = value (start + j) of tensor `tid` (SplitMix64 counter rule), or `fill`
// when bound < 0.
cudaError_t launch_init_values(float* dst, size_t n, uint64_t seed, int tid, float bound,
                               size_t start, float fill, cudaStream_t st);

// ---- forward ------------------------------------------------------------------------------
// X[s][k*D + d] = E[ctx(s,k)][d]. With data != nullptr the context is gathered
// from the stream bytes at the step's position and also written to ctx;
// otherwise ctx (b x K) is read.
// Grouped mode (rg != nullptr): row s reads the table of its group, E + rg[s] * gs.
cudaError_t launch_embed(const uint8_t* data, Split sp, const StepCtl* ctl, const float* E, int b,
                         int K, int D, float* X, uint8_t* ctx, cudaStream_t st, const int* rg = nullptr,
                         size_t gs = 0);
// Row-wise LayerNorm: xhat, rstd, X0 = g * xhat + beta.
cudaError_t launch_ln_fwd(const float* X, const float* g, const float* be, float* xhat, float* rstd,
                          float* X0, int b, int F, cudaStream_t st);
// G = GELU(prod_i A[:, iH:(i+1)H]).
cudaError_t launch_branch_gelu(const float* A, int b, int H, int k, float* G, cudaStream_t st);
// Which streams of a step are active: `active` (model API) if set, else
// the stream still has bytes at time index ctl->i. ctl == nullptr: all.
struct FdmAct {
  const StepCtl* ctl = nullptr;
  Split sp{0, 0, 0};
  const uint8_t* active = nullptr;
};
// Per-stream FDM product y_s = x'_s U_s (and optional BF16 copies of Y);
// inactive streams get y_s = 0 without reading U_s.
// err (optional) gets bit 8 if a bounded wait for a bulk copy expired.
cudaError_t launch_fdm_fwd(const float* Xp, const float* U, float* Y, int b, int Fp, cudaStream_t st,
                           __nv_bfloat16* Yb = nullptr, __nv_bfloat16* YbT = nullptr, int ldT = 0,
                           int* err = nullptr, FdmAct act = FdmAct{});

// Softmax, CDF quantization, coding and the CE gradient of one step.
struct HeadArgs {
  const float* z;            // b x 256 logits
  int b;
  const StepCtl* ctl;
  Split sp;
  int mode;                  // 0 encode, 1 decode, 2 model API (targets/active given)
  uint8_t* data;             // stream bytes (read at encode, written at decode)
  const uint8_t* targets;    // mode 2
  const uint8_t* active;     // mode 2
  float* p;                  // b x 256 out (may be null)
  float* dz;                 // b x 256 out
  uint32_t* ring;            // mode 0: ring[slot*b + s] = cum | (f-1) << 16 or kSkip
  DecState* dec;             // mode 1
  const uint8_t* bits;       // mode 1: concatenated substreams
  const unsigned long long* bits_off;
  const uint32_t* bits_len;
  uint32_t* freq_out;        // optional b x 256
  uint32_t* cum_out;         // optional b x 257
  __nv_bfloat16* dzb;        // optional b x 256 BF16 copy of dz
  __nv_bfloat16* dzbT;       // optional 256 x ldT transposed BF16 copy of dz
  int ldT;
  int* err;
  // grouped mode: row s belongs to group rg[s]; its CE gradient is divided by
  // the count of that group's active streams (group_active(gi[rg[s]], i))
  const int* rg = nullptr;
  const GroupInfo* gi = nullptr;
};
cudaError_t launch_head(const HeadArgs& a, cudaStream_t st);

// ---- backward -----------------------------------------------------------------------------
cudaError_t launch_branch_gelu_bwd(const float* dG, const float* A, int b, int H, int k, float* dA,
                                   cudaStream_t st);
// out[c] = sum_r X[r][c] (or sum_r X[r][c] * Y[r][c] when Y != nullptr), fixed order.
cudaError_t launch_colsum(const float* X, const float* Y, int rows, int cols, int ld, float* out,
                          cudaStream_t st);
// dX = dRes + LN backward of dX0.
cudaError_t launch_ln_bwd(const float* dX0, const float* xhat, const float* rstd, const float* g,
                          const float* dRes, float* dX, int b, int F, cudaStream_t st);
// FDM adjoint: dx'_s = U_s dy_s with the pre-update U, then (update=1) Adam on
// U_s, m, v with the rank-1 gradient x'_s dy_s^T; inactive streams are skipped.
// With update=0 the gradient is written to gU instead (no state change).
struct FdmBwdArgs {
  const float* Xp;
  const float* dY;
  float* U;
  float* Um;
  float* Uv;
  float* dXp;
  float* gU;
  const StepCtl* ctl;
  Split sp;
  const uint8_t* active;     // optional mask; else active = (ctl->i < len_s)
  int b, Fp;
  int update;
  __nv_bfloat16* dXpb;       // optional BF16 copies of dx'
  __nv_bfloat16* dXpbT;
  int ldT;
};
cudaError_t launch_fdm_bwd(const FdmBwdArgs& a, cudaStream_t st);

// The FDM adjoint split in two, so that the update leaves the critical path:
//   fdm_dx    dx'_s = U_s dy_s with the pre-update U (the only part the rest of
//             the adjoint waits for); also saves x'_s, dy_s and the step's Adam
//             scalars in a pending record;
//   fdm_adam  the Adam update of U, m, v from the pending record, on a side
//             stream while the rest of the step (and the next step's layers up
//             to Eq. 14) run; it must finish before the next FDM forward.
// Together they compute exactly what fdm_bwd computes (same operations, same
// order) at the cost of one more read of U.
struct FdmPend {
  int i;
  float lr, bc1, bc2;
};
struct FdmSplitArgs {
  const float* Xp;
  const float* dY;
  float* U;
  float* Um;
  float* Uv;
  float* dXp;
  __nv_bfloat16* dXpb;
  __nv_bfloat16* dXpbT;
  int ldT;
  float* xp_pend;   // b x F' copy of x'
  float* dy_pend;   // b x F' copy of dy
  FdmPend* pend;
  const StepCtl* ctl;
  Split sp;
  const uint8_t* active;
  int b, Fp;
  const float* Ub;  // fdm_adam: the Adam base (nullptr: U, in place); the delayed
                    // update reads the next step's U there and writes U, whose
                    // values fdm_dx has already consumed
};
cudaError_t launch_fdm_dx(const FdmSplitArgs& a, cudaStream_t st);
// persistent: one resident CTA per SM (else a CTA per 32 FDM rows, which the
// block scheduler interleaves with other streams' CTAs as they retire).
cudaError_t launch_fdm_adam(const FdmSplitArgs& a, cudaStream_t st, bool persistent = true);
// dE[c][d] = sum over positions with ctx == c of dX[s][k*D + d], fixed order
// (CTAs per byte value c and chunk of kEmbChunkPos positions); D <= 64. With
// more than one chunk, part (256 * chunks * D floats) and cnt (256 counters,
// zero between launches) hold the chunk partials; launches sharing them must
// not overlap.
constexpr int kEmbChunkPos = 16384;
int embed_bwd_chunks(int b, int K);
cudaError_t launch_embed_bwd(const uint8_t* ctx, const float* dX, int b, int K, int D, float* dE, float* part,
                             unsigned* cnt, cudaStream_t st);
// Grouped mode: dE of group g (at dE + g * gs) sums the positions of its
// stream rows [gi[g].r0, gi[g].r0 + gi[g].s) only, in a fixed order that
// depends on the group alone (four quarters of the positions, each summed in
// increasing order, then added in order); CTAs per group and pair of byte
// values (ctx 4-byte aligned).
cudaError_t launch_embed_bwd_groups(const uint8_t* ctx, const float* dX, int K, int D, float* dE,
                                    const GroupInfo* gi, int ngroups, size_t gs, cudaStream_t st);

// Adam over the flat shared parameters; bf16 != nullptr also refreshes the BF16 copy.
// Pin: the parameters read (nullptr: P itself, an in-place update).
cudaError_t launch_adam(float* P, const float* G, float* M, float* V, size_t n, const StepCtl* ctl,
                        cudaStream_t st, const float* Pin = nullptr);
// i += 1 and the derived per-step scalars.
// dst: where the next step's control goes (nullptr: ctl itself).
cudaError_t launch_step_advance(StepCtl* ctl, Split sp, int K, int ring_slots, int b, cudaStream_t st,
                                StepCtl* dst = nullptr);

// ---- coder --------------------------------------------------------------------------------
cudaError_t launch_prefix_encode(EncState* es, const uint8_t* data, Split sp, int K, int b,
                                 uint8_t* out, const unsigned long long* out_off,
                                 const uint32_t* out_cap, cudaStream_t st);
cudaError_t launch_range_encode(EncState* es, const uint32_t* ring, int ring_slots, int slot0,
                                int nsteps, int b, uint8_t* out, const unsigned long long* out_off,
                                const uint32_t* out_cap, cudaStream_t st);
cudaError_t launch_encode_flush(EncState* es, int b, uint8_t* out, const unsigned long long* out_off,
                                const uint32_t* out_cap, uint32_t* out_len, cudaStream_t st);
cudaError_t launch_dec_init(DecState* ds, const uint8_t* bits, const unsigned long long* off,
                            const uint32_t* len, int b, cudaStream_t st);
cudaError_t launch_prefix_decode(DecState* ds, const uint8_t* bits, const unsigned long long* off,
                                 const uint32_t* len, Split sp, int K, int b, uint8_t* data,
                                 cudaStream_t st);
// Standalone quantizer (one warp per row).
cudaError_t launch_cdf_quantize(const float* p, int rows, uint32_t* freq, uint32_t* cum,
                                cudaStream_t st);

// ---- GEMM (FP32 SIMT) ------------------------------------------------------------------------
// C[m][n] = sum_k A(m,k) B(n,k) (+ bias[n]) (+ R[m][n]).
// A(m,k) = a_kcont ? A[m*lda + k] : A[k*lda + m];  B(n,k) = b_kcont ? B[n*ldb + k] : B[k*ldb + n].
enum Epi { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RESID = 2 };
struct GemmF32 {
  int M, N, K;
  const float* A; int lda; bool a_kcont;
  const float* B; int ldb; bool b_kcont;
  float* C; int ldc;
  int epi;
  const float* bias;
  const float* R; int ldr;
};
cudaError_t launch_gemm_f32(const GemmF32& g, cudaStream_t st);

// ---- BF16 path: fused operand production -----------------------------------------------------
// Rows are processed 16 per CTA so that the transposed copy YT[c][r] (ld ldT, a
// multiple of 16; padding rows are written as zero) goes out in 32-byte runs.
constexpr int kRowsT = 16;
// LayerNorm forward writing xhat, rstd and the BF16 copies of X0 (row-major and transposed).
// Grouped mode (rg != nullptr): row r uses g + rg[r] * gs and be + rg[r] * gs.
cudaError_t launch_ln_fwd_bf16(const float* X, const float* g, const float* be, float* xhat, float* rstd,
                               __nv_bfloat16* X0b, __nv_bfloat16* X0bT, int b, int F, int ldT, cudaStream_t st,
                               const int* rg = nullptr, size_t gs = 0);
// Embedding and the first block's LayerNorm forward in one launch (F = K * D
// in {128, 256, 512, 1024}; otherwise cudaErrorInvalidValue): X and ctx as
// launch_embed, xhat, rstd, X0b, X0bT as launch_ln_fwd_bf16, same arithmetic.
cudaError_t launch_embed_ln_bf16(const uint8_t* data, Split sp, const StepCtl* ctl, const float* E, int b, int K,
                                 int D, float* X, uint8_t* ctx, const float* g, const float* be, float* xhat,
                                 float* rstd, __nv_bfloat16* X0b, __nv_bfloat16* X0bT, int ldT, cudaStream_t st,
                                 const int* rg = nullptr, size_t gs = 0);
// LayerNorm backward: dX = dRes + LN adjoint; also the BF16 copies of dX when non-null.
cudaError_t launch_ln_bwd_bf16(const float* dX0, const float* xhat, const float* rstd, const float* g,
                               const float* dRes, float* dX, __nv_bfloat16* dXb, __nv_bfloat16* dXbT, int b, int F,
                               int ldT, cudaStream_t st, const int* rg = nullptr, size_t gs = 0);
// Batched deterministic column sums: one launch for up to kMaxColsumJobs tensors.
constexpr int kMaxColsumJobs = 8;
struct ColsumJob {
  const float* X;
  const float* Y;  // optional: sum of X * Y
  int rows, cols, ld;
  float* out;
};
// With chunk_rows > 0 the rows are cut into chunks of chunk_rows (one CTA per
// 32-column tile and chunk); each CTA writes its partial sums to `part` and the
// last CTA of a tile to arrive adds the chunks' partials in chunk order, so the
// result does not depend on which CTA finishes last. `part` holds
// colsum_tiles(jobs) * chunks * (tile width) floats and `cnt` one zero-initialised counter
// per tile; the last CTA sets its counter back to zero. Launches that share
// part and cnt must not overlap (they run on one stream).
struct ColsumJobs {
  ColsumJob job[kMaxColsumJobs];
  int n;
  float* part = nullptr;
  unsigned* cnt = nullptr;
  int chunk_rows = 0;
};
// Tiles of a launch: 128-column tiles when colsum_vec (every job's columns,
// row stride and pointers allow 16-byte loads), else 32-column tiles.
bool colsum_vec(const ColsumJobs& jobs);
int colsum_tiles(const ColsumJobs& jobs);
// Rows per chunk for a column sum over `rows` rows and `tiles` 32-column
// tiles (0: one chunk).
int colsum_chunk_rows(int rows, int tiles);
constexpr int kColsumMaxChunks = 64;
cudaError_t launch_colsum_multi(const ColsumJobs& jobs, cudaStream_t st);
// Grouped column sums: for each job and group g, out[g * gs + c] = sum over
// the group's stream rows r in [gi[g].r0, gi[g].r0 + gi[g].s) of X[r][c]
// (* Y[r][c]) in a fixed order that depends on the group alone (its padding
// rows hold zero gradients; chunk fields of jobs unused).
cudaError_t launch_colsum_groups(const ColsumJobs& jobs, const GroupInfo* gi, int ngroups, size_t gs,
                                 cudaStream_t st);
// Adam that also writes the BF16 copy Pb of every updated parameter (same flat layout).
cudaError_t launch_adam_bf16(float* P, const float* G, float* M, float* V, __nv_bfloat16* Pb, size_t n,
                             const StepCtl* ctl, cudaStream_t st, const float* Pin = nullptr);
// Transposed BF16 copies of several matrices in one launch: PbT[off + c*rows + r] = Pb[off + r*cols + c].
struct TransposeTile {
  unsigned long long off;
  int rows, cols, r0, c0;
};
cudaError_t launch_transpose_tiles(const __nv_bfloat16* Pb, __nv_bfloat16* PbT, const TransposeTile* tiles,
                                   int ntiles, cudaStream_t st);

// ---- BF16 operands ------------------------------------------------------------------------------
// Y[r][c] = bf16(X[r][c]) (ld ldy) and/or YT[c][r] = bf16(X[r][c]) (ld ldt).
cudaError_t launch_to_bf16(const float* X, int rows, int cols, int ldx, __nv_bfloat16* Y, int ldy,
                           __nv_bfloat16* YT, int ldt, cudaStream_t st);

// ---- FP8 e4m3 operands (per-tensor power-of-two scales) --------------------------------------
// Each job quantizes a BF16 matrix src [rows][ld] (cols used) into e4m3 bytes
// dst [rows][ld8] with scale s = 2^k, k the largest integer with
// amax * 2^k <= 448 (amax = max |src|; k = 0 when amax = 0). inv[slot]
// receives 2^-k. amax[slot] (float bits, non-negative) must start at 0: the
// max is taken with integer atomicMax, which gives the same result in any
// order.
constexpr int kMaxFp8Jobs = 16;
struct Fp8Job {
  const __nv_bfloat16* src;
  int rows, cols, ld;
  uint8_t* dst;
  int ld8;
  int slot;
};
struct Fp8Jobs {
  Fp8Job job[kMaxFp8Jobs];
  int n;
  unsigned* amax;
  float* inv;
};
cudaError_t launch_fp8_quantize(const Fp8Jobs& jobs, cudaStream_t st);  // two launches: amax, convert
cudaError_t launch_zero_u32(unsigned* p, int n, cudaStream_t st);

}  // namespace edpc
