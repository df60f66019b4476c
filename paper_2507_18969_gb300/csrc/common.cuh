// Shared definitions of the EDPC CUDA library (device and host).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/edpc.h"

namespace edpc {

constexpr int kT = 1 << 16;          // CDF total (quantized probabilities sum to 2^16)
constexpr int kTBits = 16;
constexpr uint32_t kTop = 1u << 24;  // range coder renormalisation threshold
constexpr uint32_t kSkip = 0xFFFFFFFFu;
constexpr int kMaxBlocks = 16;
constexpr uint32_t kMaxStreams = 65535;  // streams index grid dimension y of the FDM adjoint
constexpr float kLnEps = 1e-5f;
constexpr float kB1 = 0.9f, kB2 = 0.999f, kAdamEps = 1e-8f;
constexpr int kFdmTid = 1023;        // tensor id of the FDM in the initial-value rule

// Error bits written by kernels into StepCtl::err.
constexpr int kErrCoderOverflow = 1;
constexpr int kErrDecodeOverrun = 2;

// Model dimensions of one session (derived from edpc_cfg).
struct Dims {
  int b;      // rows = streams
  int K, D, F;
  int Fp, H, n, nloc, k;  // Fp: side of each stream's FDM (F' with the LTE, F without)
  bool lte;   // false: the "w/o LTE" ablation (cfg latent = 0), no W1, b1, W2, b2
  int ldT;    // leading dimension of transposed [feature][row] operands (b rounded up to 8)
};

// Offsets (in floats) of each shared tensor inside the flat parameter buffer.
// Order: E, blocks 0..n-1 (ln_g, ln_b, W, c, Wo, co), LTE (W1, b1, W2, b2), head (Wh, bh).
struct BlockOff {
  size_t ln_g, ln_b, W, c, Wo, co;
};
struct ParamOff {
  size_t E;
  BlockOff blk[kMaxBlocks];
  size_t W1, b1, W2, b2, Wh, bh;
  size_t total;
};

// Per-step scalars, read by every kernel of a step from device memory so the
// step's launches are identical from step to step (CUDA-graph friendly).
struct StepCtl {
  int i;          // time index of the current step (0-based position in each stream)
  int t;          // Adam step number of the current step (1-based)
  int bact;       // streams active at this step
  int slot;       // coder ring slot of this step
  float inv_bact; // 1 / bact
  float bc1;      // 1 - beta1^t
  float bc2;      // 1 - beta2^t
  float lr;
  int err;        // sticky error bits
  int cpi;        // next entry of the active-count table (uneven splits)
  int pad[6];
};

// Change point of the active-stream count: from time index i on, bact
// streams are active (uneven splits; see ActiveTable).
struct ActivePoint {
  int i;
  int bact;
};

// Split of the input into b streams.
//   Balanced (seg == nullptr): n bytes into b streams of q or q+1 bytes.
//   Explicit (seg != nullptr): stream s is bytes [seg[s], seg[s+1]) of the
//   input (device array of b+1 offsets); cp[0..ncp) lists, in increasing i,
//   the time indices at which the count of active streams changes.
// off/len dereference seg, so the explicit form is for device code; host
// code keeps its own copy of the offsets.
struct Split {
  long long n;
  long long q;
  int rem;
  const unsigned long long* seg = nullptr;
  const ActivePoint* cp = nullptr;
  int ncp = 0;
  __host__ __device__ long long off(int s) const {
    return seg ? (long long)seg[s] : (long long)s * q + (s < rem ? s : rem);
  }
  __host__ __device__ long long len(int s) const {
    return seg ? (long long)(seg[s + 1] - seg[s]) : q + (s < rem ? 1 : 0);
  }
};

// Independent per-file models in one batch ("grouped" mode): group g owns
// rows [r0, r1) (r0, r1 multiples of 64): its file's s streams, the first rem
// of q + 1 bytes and the others of q bytes (the balanced split of the file),
// then r1 - r0 - s padding rows that never hold a byte. Each group has its own
// parameters, `gstride` floats after the previous group's.
struct GroupInfo {
  int r0, r1, s, rem;
  long long q;
};
// Streams of a group active at time index i (K <= i): the mean of Eq. 2 over
// the group's own active streams.
__host__ __device__ inline int group_active(const GroupInfo& g, long long i) {
  return i < g.q ? g.s : (i < g.q + 1 ? g.rem : 0);
}
constexpr int kGroupAlign = 64;  // rows per group are padded to a multiple of this

// Range coder states (one per stream), kept in device memory between launches.
struct EncState {
  unsigned long long low;
  uint32_t range;
  uint32_t cache;
  uint32_t pending;
  uint32_t started;
  uint32_t pos;
  uint32_t err;
};
struct DecState {
  uint32_t code;
  uint32_t range;
  uint32_t pos;
  uint32_t err;
};

Dims make_dims(const edpc_cfg& c, int b);
ParamOff make_offsets(const Dims& d);

// ---- error plumbing (host) ----------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define EDPC_CUDA(call)                                                                \
  do {                                                                                 \
    cudaError_t e__ = (call);                                                          \
    if (e__ != cudaSuccess)                                                            \
      return ::edpc::fail(EDPC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
  } while (0)

#define EDPC_TRY(expr)             \
  do {                             \
    int r__ = (expr);              \
    if (r__ != EDPC_OK) return r__; \
  } while (0)

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }
inline long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

}  // namespace edpc
