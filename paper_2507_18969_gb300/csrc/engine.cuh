// Device state of the EDPC model for b streams and the launch sequence of one
// step of Algorithm 1 (Model() forward, coding, cross-entropy adjoint, Adam).
#pragma once

#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "gemm_tc.cuh"

namespace edpc {

struct BlockAct {
  float* xhat;  // b x F  normalised input
  float* rstd;  // b
  float* X0;    // b x F  LN output (Eq. 9)
  float* A;     // b x kH branch outputs [X_1 | ... | X_k] (Eq. 10)
  float* G;     // b x H  GELU(X_fused) (Eq. 12)
};

// BF16 copies of GEMM operands (BF16 mode only). Row-major copies are
// K-major A operands of forward/dX GEMMs; transposed copies [feature][b]
// are the K-major operands of the dW GEMMs (contraction over streams).
struct Bf16Ops {
  __nv_bfloat16* P;    // weights, row-major, same flat layout as the FP32 params
  __nv_bfloat16* PT;   // weights, transposed per matrix (same offsets)
  __nv_bfloat16* act;  // activation copies (arena)
  __nv_bfloat16* actT;
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

  // BF16 mode
  __nv_bfloat16* Pb = nullptr;   // row-major weight copies
  __nv_bfloat16* PbT = nullptr;  // transposed weight copies
  __nv_bfloat16 *xa = nullptr, *xaT = nullptr, *xb = nullptr, *xbT = nullptr;  // activation operand copies
  TcPlan tc;                     // tensor maps and tile choices of every tcgen05 GEMM

  // FDM kernel timing (optional)
  cudaEvent_t ev_fdm[4] = {};
  bool timing = false;

  ~Model();
  int init(const edpc_cfg& cfg, int streams);
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
  };
  int forward(const StepIO& io, cudaStream_t st);
  int head(const StepIO& io, cudaStream_t st);
  int backward(const StepIO& io, cudaStream_t st);
  int adam(cudaStream_t st);
  int step(const StepIO& io, cudaStream_t st);
  int launches_per_step() const;
  int refresh_bf16_weights(cudaStream_t st);

 private:
  void* arena_ = nullptr;
  size_t arena_bytes_ = 0;
  int block_fwd(int j, const float* Xin, float* Xout, cudaStream_t st);
  int block_bwd(int j, const float* dOut, const float* Xin, float* dXnew, cudaStream_t st);
  // GEMM dispatch: FP32 SIMT or BF16 tcgen05 by precision. `site` names a
  // tensor-map slot of the BF16 plan.
  int linear_fwd(int site, const float* X, int rows, int in, size_t w_off, size_t b_off, int out,
                 const float* resid, float* Y, cudaStream_t st);
  int linear_dx(int site, const float* dOut, int rows, int out, size_t w_off, int in, float* dX,
                cudaStream_t st);
  int linear_dw(int site, const float* dOut, int rows, int out, const float* X, int in, size_t w_off,
                cudaStream_t st);
  int build_tc_plan();
};

}  // namespace edpc
