// Device state of the EDPC model for b streams and the launch sequence of one
// step of Algorithm 1 (Model() forward, coding, cross-entropy adjoint, Adam).
#pragma once

#include <vector>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "kernels.cuh"

namespace edpc {

struct BlockAct {
  float* xhat;  // b x F  normalised input
  float* rstd;  // b
  float* X0;    // b x F  LN output (Eq. 9), FP32 path
  float* A;     // b x kH branch outputs [X_1 | ... | X_k] (Eq. 10)
  float* G;     // b x H  GELU(X_fused) (Eq. 12), FP32 path
};

// BF16-path buffers of one MBRB block. "T" buffers are transposed copies
// [feature][ldT], the K-major operands of the dW GEMMs (contraction over streams).
struct BlockBf16 {
  __nv_bfloat16 *X0b, *X0bT;      // LN output
  __nv_bfloat16 *Gb, *GbT;        // GELU output
  float* dOut;                    // gradient w.r.t. the block output (b x F)
  __nv_bfloat16 *dOutb, *dOutbT;
  float* dA;                      // gradient w.r.t. the branch outputs (b x kH)
  __nv_bfloat16 *dAb, *dAbT;
  float* dX0;                     // gradient w.r.t. the LN output (b x F)
};

class Model {
 public:
  Dims d{};
  ParamOff po{};
  uint32_t precision = EDPC_FP32;
  uint64_t seed = 0;
  float lr = 1e-3f;
  size_t nparam = 0;

  // parameters and Adam state
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  float *U = nullptr, *Um = nullptr, *Uv = nullptr, *gU = nullptr;
  StepCtl* ctl = nullptr;

  // activations
  uint8_t* ctx = nullptr;                 // b x K context bytes of the step
  float* S[kMaxBlocks + 2] = {};          // residual-stream stages, b x F
  BlockAct ba[kMaxBlocks] = {};
  float *Xp = nullptr, *Y = nullptr, *z = nullptr, *p = nullptr, *dz = nullptr;
  float *dXa = nullptr, *dXb = nullptr, *dX0 = nullptr, *dA = nullptr, *dG = nullptr;
  float *dY = nullptr, *dXp = nullptr;
  float* emb_part = nullptr;              // embedding-adjoint chunk partials (many positions)
  unsigned* emb_cnt = nullptr;            // their arrival counters, one per byte value
  float* cs_part = nullptr;               // column-sum chunk partials (side stream)
  unsigned* cs_cnt = nullptr;             // column-sum arrival counters, one per 32-column tile
  int cs_tiles = 0;                       // tiles cs_cnt is sized for
  int cs_cols = 0;                        // tile columns (per chunk) cs_part is sized for
  float* sk_ws = nullptr;                 // split-K partial tiles of the dW GEMMs (side stream)
  unsigned* sk_cnt = nullptr;             // split-K arrival counters
  size_t sk_ws_floats = 0;
  static constexpr int kSplitCounters = 1024;

  // BF16 mode
  __nv_bfloat16* Pb = nullptr;   // row-major weight copies (flat layout of P)
  __nv_bfloat16* PbT = nullptr;  // transposed weight copies (same offsets)
  TransposeTile* tiles = nullptr;
  int ntiles = 0;
  BlockBf16 bb[kMaxBlocks] = {};
  __nv_bfloat16 *Slte_b = nullptr, *Slte_bT = nullptr;    // LTE-down input copies
  __nv_bfloat16 *Shead_b = nullptr, *Shead_bT = nullptr;  // head input copies
  __nv_bfloat16 *Yb = nullptr, *YbT = nullptr;
  __nv_bfloat16 *dzb = nullptr, *dzbT = nullptr;
  float* dLte = nullptr;                                   // gradient w.r.t. the LTE-up output
  __nv_bfloat16 *dLteb = nullptr, *dLtebT = nullptr;
  __nv_bfloat16 *dXpb = nullptr, *dXpbT = nullptr;
  float* dh0 = nullptr;                                    // gradient w.r.t. the embedding output
  TcPlan tcp;
  cudaStream_t side = nullptr;                             // dW GEMMs and column sums
  static constexpr int kForks = 4 * kMaxBlocks + 8;
  cudaEvent_t fork[kForks] = {};
  cudaEvent_t join_ev = nullptr;
  cudaEvent_t tr_ev = nullptr;                             // transposed weight copies ready
  cudaEvent_t fdm_join_ev = nullptr;                       // side stream caught up before the FDM adjoint
  // FDM update off the critical path (BF16/FP8): dx' on the step's stream, the
  // Adam update of U, m, v on side_fdm from the pending copies; the next FDM
  // forward waits for adam_ev.
  cudaStream_t side_fdm = nullptr;
  cudaEvent_t dx_ev = nullptr, adam_ev = nullptr;
  float *xp_pend = nullptr, *dy_pend = nullptr;
  FdmPend* pend = nullptr;
  bool fdm_pending = false;                                // an update was launched and not yet waited for

  // FDM kernel timing (optional): forward [0,1], adjoint dx' [2,3], update [4,5]
  cudaEvent_t ev_fdm[6] = {};
  bool timing = false;

  // Delayed-update schedule (EDPC_FLAG_DELAYED_UPDATE): two copies ("parities")
  // of the parameters, the FDMs, the step control and every buffer that the
  // forward pass and the head write. Step s predicts with parity s % 2 while
  // the adjoint of step s - 1 runs with parity (s - 1) % 2 (its parameters,
  // activations and control) on bwd_st; Adam then writes the parameters of
  // step s + 1 into parity (s + 1) % 2. The FDM adjoint's dx' reads parity
  // (s - 1) % 2's FDMs, and its update (on side_fdm, off the adjoint's
  // critical path) writes the FDMs of step s + 1 over them, from those of
  // step s; the FDM forward of step s + 1 waits for it. Before the first
  // step parity 1 is the zero state, whose adjoint is zero: its updates copy
  // parity 0 exactly.
  struct Parity {
    float *P = nullptr, *U = nullptr;
    __nv_bfloat16 *Pb = nullptr, *PbT = nullptr;
    StepCtl* ctl = nullptr;
    uint8_t* ctx = nullptr;
    float* S[kMaxBlocks + 2] = {};
    BlockAct ba[kMaxBlocks] = {};
    __nv_bfloat16 *X0b[kMaxBlocks] = {}, *X0bT[kMaxBlocks] = {}, *Gb[kMaxBlocks] = {}, *GbT[kMaxBlocks] = {};
    __nv_bfloat16 *Slte_b = nullptr, *Slte_bT = nullptr, *Shead_b = nullptr, *Shead_bT = nullptr;
    __nv_bfloat16 *Yb = nullptr, *YbT = nullptr, *dzb = nullptr, *dzbT = nullptr;
    float *Xp = nullptr, *Y = nullptr, *z = nullptr, *p = nullptr, *dz = nullptr;
    float *xp_pend = nullptr, *dy_pend = nullptr;  // the FDM update's inputs
    FdmPend* pend = nullptr;
    TcPlan tcp;  // GEMM sites bound to this parity's buffers
  };
  bool delayed = false;
  Parity par[2];
  int cur = 0;                    // the parity the members above point into
  float* U_base = nullptr;        // delayed: the other parity's U (Adam base of the FDM adjoint)
  cudaStream_t bwd_st = nullptr;  // delayed: the adjoint of the previous step
  cudaEvent_t tick_ev = nullptr, bwd_ev = nullptr;
  void select(int q);             // points the members at parity q
  StepCtl* ctl_of(int q) const { return delayed ? par[q].ctl : par[0].ctl; }

  // Grouped mode: independent per-file models in one batch (BF16, Algorithm
  // 1's schedule). Group g owns rows [r0, r1) and its own parameters, Adam
  // moments and BF16 copies at offset g * gstride of every parameter buffer;
  // every GEMM runs over all groups in one launch (tile lists with the
  // group's weights, or the group's own K range for weight gradients).
  int ngroups = 0;
  size_t gstride = 0;               // floats between consecutive groups' parameters
  size_t np_all = 0;                // parameter floats of all groups (nparam when not grouped)
  int* row_grp = nullptr;           // device, b: group of each row
  GroupInfo* ginfo = nullptr;       // device, ngroups
  int4* gtiles = nullptr;           // device: M tiles {m0, m_end, group, 0} of forward / dX GEMMs
  int ngtiles = 0;
  int4* gkr = nullptr;              // device, ngroups: {k0, K blocks of 64, 0, 0} of weight gradients
  std::vector<GroupInfo> groups_h;

  ~Model();
  int init(const edpc_cfg& cfg, int streams, const std::vector<GroupInfo>* groups = nullptr);
  int set_ctl_for_step(int i, int t, int bact, int ring_slots, cudaStream_t st);

  // One model step. mode: 0 encode, 1 decode, 2 model API.
  struct StepIO {
    int mode = 0;
    uint8_t* data = nullptr;
    Split sp{};
    uint32_t* ring = nullptr;
    int ring_slots = 1;
    DecState* dec = nullptr;
    const uint8_t* bits = nullptr;
    const unsigned long long* bits_off = nullptr;
    const uint32_t* bits_len = nullptr;
    const uint8_t* targets = nullptr;  // mode 2
    const uint8_t* active = nullptr;   // mode 2
    int update = 1;                    // 0: gradient only (FDM grad to gU, no Adam)
    bool advance = true;               // launch the step-control advance at the end
    int tick = 0;                      // delayed update: the step's index (its parity is tick & 1)
  };
  int forward(const StepIO& io, cudaStream_t st);
  int head(const StepIO& io, cudaStream_t st);
  int backward(const StepIO& io, cudaStream_t st);
  int adam(cudaStream_t st);
  int step(const StepIO& io, cudaStream_t st);
  int step_delayed(const StepIO& io, cudaStream_t st);
  // Makes `st` wait for a pending FDM update (call before reading U, and before
  // ending a graph capture).
  int flush(cudaStream_t st);
  int launches_per_step() const;
  int refresh_bf16_weights(cudaStream_t st);
  size_t device_bytes() const { return arena_bytes_; }

  // GEMM N tile per tcgen05 site: 32 * code (0 = size heuristic). The codes
  // change the accumulation layout, so a bitstream records the ones its
  // encoder used and the decoder sets the same.
  uint8_t tile_code[TcPlan::kMaxSites] = {};
  int set_tiles(const uint8_t* code, int n);  // codes 0, 1, 2, 4 or 8; rebuilds the plan

  // FP8 e4m3 mode: one e4m3 shadow per distinct BF16 GEMM operand, with a
  // per-tensor power-of-two scale computed every step (amax slot + inverse).
  struct Fp8Shadow {
    const __nv_bfloat16* src = nullptr;
    int rows = 0, cols = 0, ld = 0;
    uint8_t* dst = nullptr;
    int ld8 = 0;
    int qcols = 0;            // columns quantized (cols rounded up to 8, within ld)
    bool weight = false;      // a weight copy (Pb / PbT): quantized once at the step's start
    bool transposed = false;  // a PbT weight copy
  };
  std::vector<Fp8Shadow> f8;
  uint8_t* f8_arena = nullptr;
  unsigned* f8_amax = nullptr;
  float* f8_inv = nullptr;
  std::vector<char> f8_done;
  int site_fa[TcPlan::kMaxSites] = {}, site_fb[TcPlan::kMaxSites] = {};
  int tune_tiles(cudaStream_t st);            // times the N tiles of every tcgen05 site
  void tunable_sites(std::vector<int>* ids) const;
  bool tile_code_ok(int id, uint8_t code) const;
  // CUDA-event time of each tcgen05 site launched alone (mean of `reps`
  // launches after one warm-up; like tune_tiles it overwrites per-step outputs),
  // its FLOP count 2*M*N*K and its compulsory bytes (operands and epilogue
  // inputs read once, outputs written once); unused sites get 0.
  int time_sites(cudaStream_t st, int reps, double* ms, double* flop, double* bytes, int cap);

 private:
  void* arena_ = nullptr;
  size_t arena_bytes_ = 0;
  int nfork_ = 0;
  // FP32 path
  int block_fwd(int j, const float* Xin, float* Xout, cudaStream_t st);
  int block_bwd(int j, const float* dOut, float* dXnew, cudaStream_t st);
  int forward_f32(const StepIO& io, cudaStream_t st);
  int backward_f32(const StepIO& io, cudaStream_t st);
  int linear_fwd(const float* X, int rows, int in, size_t w_off, size_t b_off, int out, const float* resid, float* Yo,
                 cudaStream_t st);
  int linear_dx(const float* dOut, int rows, int out, size_t w_off, int in, float* dX, cudaStream_t st);
  int linear_dw(const float* dOut, int rows, int out, const float* X, int in, size_t w_off, cudaStream_t st);
  // BF16 path
  int forward_bf16(const StepIO& io, cudaStream_t st);
  int backward_bf16(const StepIO& io, cudaStream_t st);
  int build_tc_plan();
  int build_tc_sites();
  int fp8_shadow(const void* src, int rows, int cols, int ld);
  int quantize_weights(bool transposed, cudaStream_t st);
  int quantize_site(int site, cudaStream_t st);
  bool f8_collect = false;
  int run_tc(int site, cudaStream_t st);
  int fork_side(cudaStream_t st);  // the side stream waits for the work issued so far on st
  int colsums(ColsumJobs cj, cudaStream_t st);  // column sums with the model's chunk scratch
  int fdm_fwd_call(const StepIO& io, cudaStream_t st);
  int fdm_bwd_call(const StepIO& io, cudaStream_t st);
  int fdm_bwd_joined(const StepIO& io, cudaStream_t st);  // waits for the side stream from 2048 streams on
  int build_tc_plan_one();
  void save_parity(int q);                                 // parity q <- the members
  const TcPlan& plan() const { return delayed ? par[cur].tcp : tcp; }
};

}  // namespace edpc
