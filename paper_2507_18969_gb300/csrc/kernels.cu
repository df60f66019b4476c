// Row-wise, element-wise and coder kernels of the EDPC step.
//
// Every reduction runs in a fixed order (warp xor-butterflies, then shared
// memory in warp order), and nothing is accumulated with floating-point
// atomics. So the encoder and the decoder, which launch the same kernels on
// the same values, compute bit-identical probabilities and CDFs.
#include <cuda_fp8.h>

#include <algorithm>

#include <mutex>

#include "kernels.cuh"
#include "launch.cuh"

namespace edpc {

// ============================================================================================
// Initial values: SplitMix64 counter streams (Steele, Lea, Flood, OOPSLA 2014).
// Value idx of tensor tid is output idx+1 of the stream seeded with
// seed + G * tid * 2^32; its top 24 bits k give w = (2k + 1 - 2^24) / 2^24 in
// (-1, 1), exact in FP32, and the value is the FP32 product bound * w.
// ============================================================================================
__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void init_values_kernel(float* dst, size_t n, unsigned long long seed, int tid, float bound,
                                   size_t start, float fill) {
  pdl_wait();
  pdl_launch();
  const unsigned long long G = 0x9E3779B97F4A7C15ull;
  const unsigned long long base = seed + G * ((unsigned long long)tid << 32);
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    if (bound < 0.f) {
      dst[j] = fill;
      continue;
    }
    unsigned long long z = sm64_mix(base + G * (start + j + 1));
    int k = (int)(z >> 40);
    float w = (float)(2 * k + 1 - (1 << 24)) * (1.0f / 16777216.0f);
    dst[j] = __fmul_rn(bound, w);
  }
}

cudaError_t launch_init_values(float* dst, size_t n, uint64_t seed, int tid, float bound, size_t start,
                               float fill, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
  return launch_k(init_values_kernel, dim3(grid), dim3(256), 0, st, dst, n, seed, tid, bound, start, fill);
}

// ============================================================================================
// Warp helpers
// ============================================================================================
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ============================================================================================
// Embedding: h0 = concat_k E[x_{i-K+k}] (the model input of Algorithm 1's Model()).
// ============================================================================================
__global__ void embed_kernel(const uint8_t* __restrict__ data, Split sp, const StepCtl* __restrict__ ctl,
                             const float* __restrict__ E, int K, int D, float* __restrict__ X,
                             uint8_t* __restrict__ ctx, const int* __restrict__ rg, size_t gs) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.x;
  if (rg) E += (size_t)rg[s] * gs;  // grouped mode: the row's own model
  const int F = K * D;
  // A stream past its end (inactive) keeps its last context: its bytes
  // [i - K, i) would run beyond the stream, and its outputs are masked.
  if (data && ctl->i <= sp.len(s)) {
    const long long base = sp.off(s) + ctl->i - K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) ctx[(size_t)s * K + k] = data[base + k];
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < F; idx += blockDim.x) {
    int k = idx / D, d = idx - k * D;
    int c = ctx[(size_t)s * K + k];
    X[(size_t)s * F + idx] = E[c * D + d];
  }
}

cudaError_t launch_embed(const uint8_t* data, Split sp, const StepCtl* ctl, const float* E, int b, int K,
                         int D, float* X, uint8_t* ctx, cudaStream_t st, const int* rg, size_t gs) {
  return launch_k(embed_kernel, dim3(b), dim3(128), 0, st, data, sp, ctl, E, K, D, X, ctx, rg, gs);
}

// ============================================================================================
// LayerNorm forward (Eq. 9), one warp per row, two-pass statistics.
// ============================================================================================
__global__ void ln_fwd_kernel(const float* __restrict__ X, const float* __restrict__ g,
                              const float* __restrict__ be, float* __restrict__ xhat,
                              float* __restrict__ rstd, float* __restrict__ X0, int b, int F) {
  pdl_wait();
  pdl_launch();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= b) return;
  const float* x = X + (size_t)row * F;
  float s = 0.f;
  for (int c = lane; c < F; c += 32) s += x[c];
  const float mean = warp_sum(s) / (float)F;
  float q = 0.f;
  for (int c = lane; c < F; c += 32) {
    float d = x[c] - mean;
    q += d * d;
  }
  const float var = warp_sum(q) / (float)F;
  const float r = 1.0f / sqrtf(var + kLnEps);
  for (int c = lane; c < F; c += 32) {
    float h = (x[c] - mean) * r;
    xhat[(size_t)row * F + c] = h;
    X0[(size_t)row * F + c] = h * g[c] + be[c];
  }
  if (lane == 0) rstd[row] = r;
}

cudaError_t launch_ln_fwd(const float* X, const float* g, const float* be, float* xhat, float* rstd,
                          float* X0, int b, int F, cudaStream_t st) {
  return launch_k(ln_fwd_kernel, dim3(div_up(b, 8)), dim3(256), 0, st, X, g, be, xhat, rstd, X0, b, F);
}

// ============================================================================================
// MBRB branch fusion (Eqs. 11-12): G = GELU(X_1 * ... * X_k), exact erf GELU.
// ============================================================================================
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void branch_gelu_kernel(const float* __restrict__ A, int b, int H, int k, float* __restrict__ G) {
  pdl_wait();
  pdl_launch();
  const size_t n = (size_t)b * H;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    size_t r = e / H, h = e - r * H;
    const float* a = A + r * (size_t)k * H + h;
    float f = a[0];
    for (int i = 1; i < k; ++i) f *= a[(size_t)i * H];
    G[e] = gelu_f(f);
  }
}

cudaError_t launch_branch_gelu(const float* A, int b, int H, int k, float* G, cudaStream_t st) {
  size_t n = (size_t)b * H;
  int grid = (int)((n + 255) / 256);
  return launch_k(branch_gelu_kernel, dim3(grid), dim3(256), 0, st, A, b, H, k, G);
}

__global__ void branch_gelu_bwd_kernel(const float* __restrict__ dG, const float* __restrict__ A, int b, int H,
                                       int k, float* __restrict__ dA) {
  pdl_wait();
  pdl_launch();
  const size_t n = (size_t)b * H;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    size_t r = e / H, h = e - r * H;
    const float* a = A + r * (size_t)k * H + h;
    float* da = dA + r * (size_t)k * H + h;
    float f = a[0];
    for (int i = 1; i < k; ++i) f *= a[(size_t)i * H];
    float df = dG[e] * gelu_grad_f(f);
    for (int i = 0; i < k; ++i) {
      float o = 1.0f;
      for (int l = 0; l < k; ++l)
        if (l != i) o *= a[(size_t)l * H];
      da[(size_t)i * H] = df * o;
    }
  }
}

cudaError_t launch_branch_gelu_bwd(const float* dG, const float* A, int b, int H, int k, float* dA,
                                   cudaStream_t st) {
  size_t n = (size_t)b * H;
  int grid = (int)((n + 255) / 256);
  return launch_k(branch_gelu_bwd_kernel, dim3(grid), dim3(256), 0, st, dG, A, b, H, k, dA);
}

// ============================================================================================
// Column sums over rows (bias and LN-affine gradients), fixed order:
// warp w sums rows w, w+8, ... for 32 columns; then warps are added in order.
// ============================================================================================
__global__ void colsum_kernel(const float* __restrict__ X, const float* __restrict__ Y, int rows, int cols,
                              int ld, float* __restrict__ out) {
  pdl_wait();
  pdl_launch();
  __shared__ float part[8][33];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (c < cols) {
    if (Y) {
      for (int r = w; r < rows; r += 8) s += X[(size_t)r * ld + c] * Y[(size_t)r * ld + c];
    } else {
      for (int r = w; r < rows; r += 8) s += X[(size_t)r * ld + c];
    }
  }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && c < cols) {
    float t = part[0][lane];
#pragma unroll
    for (int i = 1; i < 8; ++i) t += part[i][lane];
    out[c] = t;
  }
}

cudaError_t launch_colsum(const float* X, const float* Y, int rows, int cols, int ld, float* out,
                          cudaStream_t st) {
  return launch_k(colsum_kernel, dim3(div_up(cols, 32)), dim3(256), 0, st, X, Y, rows, cols, ld, out);
}

// ============================================================================================
// LayerNorm backward: dX = dRes + rstd * (dxh - mean(dxh) - xhat * mean(dxh * xhat)),
// dxh = dX0 * g; one warp per row.
// ============================================================================================
__global__ void ln_bwd_kernel(const float* __restrict__ dX0, const float* __restrict__ xhat,
                              const float* __restrict__ rstd, const float* __restrict__ g,
                              const float* __restrict__ dRes, float* __restrict__ dX, int b, int F) {
  pdl_wait();
  pdl_launch();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= b) return;
  const size_t o = (size_t)row * F;
  float s1 = 0.f, s2 = 0.f;
  for (int c = lane; c < F; c += 32) {
    float d = dX0[o + c] * g[c];
    s1 += d;
    s2 += d * xhat[o + c];
  }
  const float m1 = warp_sum(s1) / (float)F;
  const float m2 = warp_sum(s2) / (float)F;
  const float r = rstd[row];
  for (int c = lane; c < F; c += 32) {
    float d = dX0[o + c] * g[c];
    dX[o + c] = dRes[o + c] + r * (d - m1 - xhat[o + c] * m2);
  }
}

cudaError_t launch_ln_bwd(const float* dX0, const float* xhat, const float* rstd, const float* g,
                          const float* dRes, float* dX, int b, int F, cudaStream_t st) {
  return launch_k(ln_bwd_kernel, dim3(div_up(b, 8)), dim3(256), 0, st, dX0, xhat, rstd, g, dRes, dX, b, F);
}

// ============================================================================================
// FDM forward (Eq. 15): y_s[j] = sum_i x'_s[i] U_s[i][j]. One CTA per stream;
// threads own 4 consecutive columns and a row group; row groups are added in order.
// ============================================================================================
// A stream that is past its end (or masked in the model API) has no
// prediction to make: its y is written as zeros and its U_s is not read.
__device__ __forceinline__ bool fdm_row_active(const FdmAct& a, int s) {
  if (!a.ctl) return true;
  return a.active ? a.active[s] != 0 : (long long)a.ctl->i < a.sp.len(s);
}

__device__ __forceinline__ void fdm_zero_row(float* Y, __nv_bfloat16* Yb, __nv_bfloat16* YbT, int ldT, int s,
                                             int Fp) {
  for (int j = threadIdx.x; j < Fp; j += blockDim.x) {
    Y[(size_t)s * Fp + j] = 0.f;
    if (Yb) Yb[(size_t)s * Fp + j] = __float2bfloat16_rn(0.f);
    if (YbT) YbT[(size_t)j * ldT + s] = __float2bfloat16_rn(0.f);
  }
}

__global__ void __launch_bounds__(256) fdm_fwd_kernel(const float* __restrict__ Xp, const float* __restrict__ U,
                                                      float* __restrict__ Y, int Fp, __nv_bfloat16* Yb,
                                                      __nv_bfloat16* YbT, int ldT, FdmAct act) {
  pdl_wait();
  pdl_launch();
  extern __shared__ float sm[];
  float* xs = sm;              // Fp
  float* part = sm + Fp;       // groups x Fp
  const int s = blockIdx.x;
  if (!fdm_row_active(act, s)) {
    fdm_zero_row(Y, Yb, YbT, ldT, s, Fp);
    return;
  }
  const int cols4 = Fp >> 2;
  const int groups = blockDim.x / cols4;
  const int cg = threadIdx.x % cols4, rg = threadIdx.x / cols4;
  for (int i = threadIdx.x; i < Fp; i += blockDim.x) xs[i] = Xp[(size_t)s * Fp + i];
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (rg < groups) {
    const float4* u = reinterpret_cast<const float4*>(U + (size_t)s * Fp * Fp) + cg;
    int i = rg;
#pragma unroll 4
    for (; i < Fp; i += groups) {
      float4 v = __ldcs(u + (size_t)i * cols4);
      float x = xs[i];
      acc.x += x * v.x;
      acc.y += x * v.y;
      acc.z += x * v.z;
      acc.w += x * v.w;
    }
    float* p = part + (size_t)rg * Fp + cg * 4;
    p[0] = acc.x; p[1] = acc.y; p[2] = acc.z; p[3] = acc.w;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < Fp; j += blockDim.x) {
    float t = part[j];
    for (int g = 1; g < groups; ++g) t += part[(size_t)g * Fp + j];
    Y[(size_t)s * Fp + j] = t;
    if (Yb) Yb[(size_t)s * Fp + j] = __float2bfloat16_rn(t);
    if (YbT) YbT[(size_t)j * ldT + s] = __float2bfloat16_rn(t);
  }
}

// Streamed FDM forward helpers (F' in {128, 256, 512, 1024}): TMA bulk copies
// of 16 KB (consecutive rows of U_s are contiguous) into a ring of shared
// memory slots, each with an mbarrier; every wait is bounded.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <int FP>
struct FdmRing {
  static constexpr int NT = FP < 256 ? FP : 256;     // threads
  static constexpr int CPT = FP / NT;                 // columns per thread
  static constexpr int SROWS = 4096 / FP;             // rows per 16 KB stage
  static constexpr int NST = FP / SROWS;              // stages per stream
  static constexpr int RING = NST < 3 ? NST : 3;
  static constexpr size_t kSmem = (size_t)RING * 16384 + (size_t)FP * 4 + 64;
};

// Persistent FDM forward: kFdmPersistPerSm CTAs per SM walk the streams s =
// blockIdx.x, blockIdx.x + gridDim.x, ...; thread 0 keeps kFdmPersistRing
// 16 KB copies in flight across stream boundaries (no drain between streams,
// no partial last wave). Thread t owns columns t, t + NT, ... of the stream's
// y and sums its rows in increasing i (deterministic, no cross-thread
// reduction).
constexpr int kFdmPersistRing = 6;
constexpr int kFdmPersistPerSm = 2;

template <int FP>
__global__ void __launch_bounds__(FdmRing<FP>::NT)
    fdm_fwd_persist_kernel(const float* __restrict__ Xp, const float* __restrict__ U, float* __restrict__ Y,
                           __nv_bfloat16* Yb, __nv_bfloat16* YbT, int ldT, int* err, FdmAct act, int b) {
  using R = FdmRing<FP>;
  constexpr int RING = kFdmPersistRing;
  extern __shared__ __align__(128) float smf[];
  float* buf = smf;                         // RING x 16 KB
  float* xs = smf + (size_t)RING * 4096;    // FP
  uint64_t* bars = reinterpret_cast<uint64_t*>(xs + FP);
  const int t = threadIdx.x;
  if (t == 0) {
    for (int q = 0; q < RING; ++q) bar_init(&bars[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // producer cursor (thread 0): next stream and stage to copy, copies issued
  int ps = blockIdx.x, pst = 0;
  uint32_t issued = 0;
  auto next_active = [&](int s0) {
    int s1 = s0;
    while (s1 < b && !fdm_row_active(act, s1)) s1 += gridDim.x;
    return s1;
  };
  auto issue_one = [&]() {
    if (ps >= b) return;
    const float* src = U + (size_t)ps * FP * FP + (size_t)pst * 4096;
    bulk_load(buf + (size_t)(issued % RING) * 4096, src, 16384u, &bars[issued % RING]);
    ++issued;
    if (++pst == R::NST) {
      pst = 0;
      ps = next_active(ps + gridDim.x);
    }
  };
  // The first copies go out before the dependent-launch wait: U and the step
  // control were written by launches that completed before the preceding
  // launch (whose own wait this one follows) could start; only x' comes from
  // the preceding launch, and every thread reads it after the wait below.
  if (t == 0) {
    ps = next_active(ps);
    for (int q = 0; q < RING; ++q) issue_one();
  }
  pdl_wait();
  pdl_launch();
  uint32_t used = 0;  // copies consumed (same sequence as issued)
  bool ok = true;
  for (int s = blockIdx.x; s < b; s += gridDim.x) {
    if (!fdm_row_active(act, s)) {  // CTA-uniform
      fdm_zero_row(Y, Yb, YbT, ldT, s, FP);
      continue;
    }
    __syncthreads();  // the previous stream's readers are done with xs
    for (int i = t; i < FP; i += R::NT) xs[i] = Xp[(size_t)s * FP + i];
    __syncthreads();
    float acc[R::CPT];
#pragma unroll
    for (int j = 0; j < R::CPT; ++j) acc[j] = 0.f;
    for (int st = 0; st < R::NST; ++st, ++used) {
      const int q = (int)(used % RING);
      ok = bar_wait(&bars[q], (used / RING) & 1u) && ok;
      const float* u = buf + (size_t)q * 4096;
      const float* xv = xs + st * R::SROWS;
#pragma unroll
      for (int r = 0; r < R::SROWS; ++r) {
        const float xr = xv[r];
#pragma unroll
        for (int j = 0; j < R::CPT; ++j) acc[j] += xr * u[r * FP + t + j * R::NT];
      }
      __syncthreads();  // slot q consumed by every thread
      if (t == 0) issue_one();
    }
#pragma unroll
    for (int j = 0; j < R::CPT; ++j) {
      const int c = t + j * R::NT;
      Y[(size_t)s * FP + c] = acc[j];
      if (Yb) Yb[(size_t)s * FP + c] = __float2bfloat16_rn(acc[j]);
      if (YbT) YbT[(size_t)c * ldT + s] = __float2bfloat16_rn(acc[j]);
    }
  }
  if (!ok && t == 0 && err) atomicOr(err, 8);
}

template <int FP>
cudaError_t launch_fdm_fwd_persist(const float* Xp, const float* U, float* Y, int b, __nv_bfloat16* Yb,
                                   __nv_bfloat16* YbT, int ldT, int* err, const FdmAct& act, cudaStream_t st) {
  const size_t smem = (size_t)kFdmPersistRing * 16384 + (size_t)FP * 4 + 64 + 64;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int grid = 0;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(fdm_fwd_persist_kernel<FP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0;
    if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
    if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = sms * kFdmPersistPerSm;
  });
  if (attr != cudaSuccess) return attr;
  const int g = b < grid ? b : grid;
  return launch_k(fdm_fwd_persist_kernel<FP>, dim3(g), dim3(FdmRing<FP>::NT), smem, st, Xp, U, Y, Yb, YbT, ldT, err,
                  act, b);
}

cudaError_t launch_fdm_fwd(const float* Xp, const float* U, float* Y, int b, int Fp, cudaStream_t st,
                           __nv_bfloat16* Yb, __nv_bfloat16* YbT, int ldT, int* err, FdmAct act) {
  switch (Fp) {
    case 128: return launch_fdm_fwd_persist<128>(Xp, U, Y, b, Yb, YbT, ldT, err, act, st);
    case 256: return launch_fdm_fwd_persist<256>(Xp, U, Y, b, Yb, YbT, ldT, err, act, st);
    case 512: return launch_fdm_fwd_persist<512>(Xp, U, Y, b, Yb, YbT, ldT, err, act, st);
    case 1024: return launch_fdm_fwd_persist<1024>(Xp, U, Y, b, Yb, YbT, ldT, err, act, st);
    default: break;
  }
  const int cols4 = Fp / 4;
  const int threads = cols4 >= 256 ? cols4 : (256 / cols4) * cols4;
  const int groups = threads / cols4;
  size_t smem = (size_t)(Fp + groups * Fp) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fdm_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_k(fdm_fwd_kernel, dim3(b), dim3(threads), smem, st, Xp, U, Y, Fp, Yb, YbT, ldT, act);
}

// ============================================================================================
// FDM adjoint + Adam (the per-stream HBM-bound update). One warp per FDM row i;
// lanes own float4 column chunks. For row i of stream s:
//   dx'_s[i] = sum_j U[i][j] dy[j]   (pre-update U, warp reduction in fixed order)
//   g[i][j]  = x'_s[i] dy[j]         (rank-1 gradient of Eq. 15)
//   m, v, U  <- Adam(g)              (bias-corrected, lr from the step control)
// ============================================================================================
constexpr int kFdmRowsPerCta = 32;

__device__ __forceinline__ void adam1(float& p, float& m, float& v, float g, float lr, float bc1, float bc2) {
  m = kB1 * m + (1.0f - kB1) * g;
  v = kB2 * v + (1.0f - kB2) * g * g;
  float mh = m / bc1;
  float vh = v / bc2;
  p = p - lr * mh / (sqrtf(vh) + kAdamEps);
}

__device__ __forceinline__ void store_dxp(const FdmBwdArgs& a, int s, int i, float v) {
  a.dXp[(size_t)s * a.Fp + i] = v;
  if (a.dXpb) a.dXpb[(size_t)s * a.Fp + i] = __float2bfloat16_rn(v);
  if (a.dXpbT) a.dXpbT[(size_t)i * a.ldT + s] = __float2bfloat16_rn(v);
}

template <int NCH>  // float4 chunks per lane per row: Fp = 128 * NCH
__global__ void __launch_bounds__(256) fdm_bwd_kernel(FdmBwdArgs a) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StepCtl c = *a.ctl;
  bool act = a.active ? (a.active[s] != 0) : ((long long)c.i < a.sp.len(s));
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  if (!act) {
    // dy is zero for an inactive stream, so dx' = 0 and its FDM state is left as is.
    for (int r = warp; r < kFdmRowsPerCta; r += 8)
      if (lane == 0 && row0 + r < Fp) store_dxp(a, s, row0 + r, 0.f);
    if (!a.update) {
      for (int r = warp; r < kFdmRowsPerCta; r += 8) {
        int i = row0 + r;
        if (i >= Fp) break;
        float4* gu = reinterpret_cast<float4*>(a.gU + ((size_t)s * Fp + i) * Fp);
#pragma unroll
        for (int q = 0; q < NCH; ++q) gu[lane + 32 * q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    return;
  }
  float4 dy[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) dy[q] = reinterpret_cast<const float4*>(a.dY + (size_t)s * Fp)[lane + 32 * q];
  for (int r = warp; r < kFdmRowsPerCta; r += 8) {
    const int i = row0 + r;
    if (i >= Fp) break;
    const float xi = a.Xp[(size_t)s * Fp + i];
    const size_t ro = ((size_t)s * Fp + i) * Fp;
    float4* U4 = reinterpret_cast<float4*>(a.U + ro);
    float dot = 0.f;
    if (a.update) {
      float4* M4 = reinterpret_cast<float4*>(a.Um + ro);
      float4* V4 = reinterpret_cast<float4*>(a.Uv + ro);
      float4 u[NCH], m[NCH], v[NCH];
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        u[q] = __ldcs(U4 + lane + 32 * q);
        m[q] = __ldcs(M4 + lane + 32 * q);
        v[q] = __ldcs(V4 + lane + 32 * q);
      }
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        dot += u[q].x * dy[q].x;
        dot += u[q].y * dy[q].y;
        dot += u[q].z * dy[q].z;
        dot += u[q].w * dy[q].w;
        adam1(u[q].x, m[q].x, v[q].x, xi * dy[q].x, c.lr, c.bc1, c.bc2);
        adam1(u[q].y, m[q].y, v[q].y, xi * dy[q].y, c.lr, c.bc1, c.bc2);
        adam1(u[q].z, m[q].z, v[q].z, xi * dy[q].z, c.lr, c.bc1, c.bc2);
        adam1(u[q].w, m[q].w, v[q].w, xi * dy[q].w, c.lr, c.bc1, c.bc2);
        __stcs(U4 + lane + 32 * q, u[q]);
        __stcs(M4 + lane + 32 * q, m[q]);
        __stcs(V4 + lane + 32 * q, v[q]);
      }
    } else {
      float4* G4 = reinterpret_cast<float4*>(a.gU + ro);
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        float4 u = U4[lane + 32 * q];
        dot += u.x * dy[q].x;
        dot += u.y * dy[q].y;
        dot += u.z * dy[q].z;
        dot += u.w * dy[q].w;
        G4[lane + 32 * q] = make_float4(xi * dy[q].x, xi * dy[q].y, xi * dy[q].z, xi * dy[q].w);
      }
    }
    dot = warp_sum(dot);
    if (lane == 0) store_dxp(a, s, i, dot);
  }
}

// ---- split form: dx' on the critical path, the update on a side stream ------------------------
__device__ __forceinline__ bool fdm_split_active(const FdmSplitArgs& a, int s, long long i) {
  return a.active ? (a.active[s] != 0) : (i < a.sp.len(s));
}

template <int NCH>
__global__ void __launch_bounds__(256) fdm_dx_kernel(FdmSplitArgs a) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StepCtl c = *a.ctl;
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  if (blockIdx.x == 0 && s == 0 && threadIdx.x == 0) *a.pend = FdmPend{c.i, c.lr, c.bc1, c.bc2};
  const bool act = fdm_split_active(a, s, c.i);
  if (blockIdx.x == 0 && act) {  // the update's inputs, kept past this step's x' and dy
    for (int j = threadIdx.x; j < Fp; j += blockDim.x) {
      a.xp_pend[(size_t)s * Fp + j] = a.Xp[(size_t)s * Fp + j];
      a.dy_pend[(size_t)s * Fp + j] = a.dY[(size_t)s * Fp + j];
    }
  }
  FdmBwdArgs o{};
  o.dXp = a.dXp;
  o.dXpb = a.dXpb;
  o.dXpbT = a.dXpbT;
  o.ldT = a.ldT;
  o.Fp = Fp;
  if (!act) {
    for (int r = warp; r < kFdmRowsPerCta; r += 8)
      if (lane == 0 && row0 + r < Fp) store_dxp(o, s, row0 + r, 0.f);
    return;
  }
  float4 dy[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) dy[q] = reinterpret_cast<const float4*>(a.dY + (size_t)s * Fp)[lane + 32 * q];
  for (int r = warp; r < kFdmRowsPerCta; r += 8) {
    const int i = row0 + r;
    if (i >= Fp) break;
    const float4* U4 = reinterpret_cast<const float4*>(a.U + ((size_t)s * Fp + i) * Fp);
    float4 u[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) u[q] = __ldcs(U4 + lane + 32 * q);
    float dot = 0.f;
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      dot += u[q].x * dy[q].x;
      dot += u[q].y * dy[q].y;
      dot += u[q].z * dy[q].z;
      dot += u[q].w * dy[q].w;
    }
    dot = warp_sum(dot);
    if (lane == 0) store_dxp(o, s, i, dot);
  }
}

template <int NCH>
__global__ void __launch_bounds__(256) fdm_adam_kernel(FdmSplitArgs a) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const FdmPend pd = *a.pend;
  if (!fdm_split_active(a, s, pd.i)) return;  // a finished stream's FDM is left as is
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  float4 dy[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) dy[q] = reinterpret_cast<const float4*>(a.dy_pend + (size_t)s * Fp)[lane + 32 * q];
  for (int r = warp; r < kFdmRowsPerCta; r += 8) {
    const int i = row0 + r;
    if (i >= Fp) break;
    const float xi = a.xp_pend[(size_t)s * Fp + i];
    const size_t ro = ((size_t)s * Fp + i) * Fp;
    float4* U4 = reinterpret_cast<float4*>(a.U + ro);
    const float4* B4 = reinterpret_cast<const float4*>((a.Ub ? a.Ub : a.U) + ro);
    float4* M4 = reinterpret_cast<float4*>(a.Um + ro);
    float4* V4 = reinterpret_cast<float4*>(a.Uv + ro);
    float4 u[NCH], m[NCH], v[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      u[q] = __ldcs(B4 + lane + 32 * q);
      m[q] = __ldcs(M4 + lane + 32 * q);
      v[q] = __ldcs(V4 + lane + 32 * q);
    }
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      adam1(u[q].x, m[q].x, v[q].x, xi * dy[q].x, pd.lr, pd.bc1, pd.bc2);
      adam1(u[q].y, m[q].y, v[q].y, xi * dy[q].y, pd.lr, pd.bc1, pd.bc2);
      adam1(u[q].z, m[q].z, v[q].z, xi * dy[q].z, pd.lr, pd.bc1, pd.bc2);
      adam1(u[q].w, m[q].w, v[q].w, xi * dy[q].w, pd.lr, pd.bc1, pd.bc2);
      __stcs(U4 + lane + 32 * q, u[q]);
      __stcs(M4 + lane + 32 * q, m[q]);
      __stcs(V4 + lane + 32 * q, v[q]);
    }
  }
}

// Persistent form of the update, built to run beside the step's other kernels:
// one CTA of 512 threads per SM, at most 80 registers a thread and no shared
// memory, so the step's tensor-core GEMM CTAs still fit on every SM. The FDM
// rows are cut into units of 32 lanes x NU float4 (NU = min(NCH, 2)); warp w of
// CTA c owns units u = c * 16 + w, u + W, u + 2W, ... (W = 16 * grid) and
// updates two units per iteration, so every lane has 6 NU independent
// 16-byte loads in flight. Warps never synchronise.
constexpr int kAdamWarps = 16;

template <int NCH>
__global__ void __maxnreg__(80) fdm_adam_persist_kernel(FdmSplitArgs a) {
  constexpr int FP = 128 * NCH;
  constexpr int NU = NCH < 2 ? NCH : 2;  // float4 per lane per unit
  constexpr int UPR = NCH / NU;          // units per FDM row
  pdl_wait();
  pdl_launch();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const FdmPend pd = *a.pend;
  const float* src = a.Ub ? a.Ub : a.U;  // Adam base (the delayed update reads the other parity)
  const int units = a.b * FP * UPR;      // < 2^31: at most 65535 x 1024 x 4
  const int W = gridDim.x * kAdamWarps;
  for (int u0 = blockIdx.x * kAdamWarps + warp; u0 < units; u0 += 2 * W) {
    const int un[2] = {u0, u0 + W};
    bool act[2];
    float xi[2];
    size_t base[2];
    int dyo[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = un[h] / UPR;  // global FDM row: stream g / F', row g % F'
      const int part = un[h] % UPR;
      const int s = g / FP;
      act[h] = un[h] < units && fdm_split_active(a, s, pd.i);
      xi[h] = act[h] ? a.xp_pend[g] : 0.f;
      base[h] = (size_t)g * FP + (size_t)part * 128 * NU;
      dyo[h] = s * FP + part * 128 * NU;
    }
    float4 u[2][NU], m[2][NU], v[2][NU];
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (act[h]) {
#pragma unroll
        for (int q = 0; q < NU; ++q) {
          u[h][q] = __ldcs(reinterpret_cast<const float4*>(src + base[h]) + lane + 32 * q);
          m[h][q] = __ldcs(reinterpret_cast<const float4*>(a.Um + base[h]) + lane + 32 * q);
          v[h][q] = __ldcs(reinterpret_cast<const float4*>(a.Uv + base[h]) + lane + 32 * q);
        }
      }
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (act[h]) {
#pragma unroll
        for (int q = 0; q < NU; ++q) {
          const float4 dy = reinterpret_cast<const float4*>(a.dy_pend + dyo[h])[lane + 32 * q];
          adam1(u[h][q].x, m[h][q].x, v[h][q].x, xi[h] * dy.x, pd.lr, pd.bc1, pd.bc2);
          adam1(u[h][q].y, m[h][q].y, v[h][q].y, xi[h] * dy.y, pd.lr, pd.bc1, pd.bc2);
          adam1(u[h][q].z, m[h][q].z, v[h][q].z, xi[h] * dy.z, pd.lr, pd.bc1, pd.bc2);
          adam1(u[h][q].w, m[h][q].w, v[h][q].w, xi[h] * dy.w, pd.lr, pd.bc1, pd.bc2);
          __stcs(reinterpret_cast<float4*>(a.U + base[h]) + lane + 32 * q, u[h][q]);
          __stcs(reinterpret_cast<float4*>(a.Um + base[h]) + lane + 32 * q, m[h][q]);
          __stcs(reinterpret_cast<float4*>(a.Uv + base[h]) + lane + 32 * q, v[h][q]);
        }
      }
  }
}

// Generic fallback for F' not a multiple of 128: one element per lane step.
__global__ void __launch_bounds__(256) fdm_bwd_generic_kernel(FdmBwdArgs a) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StepCtl c = *a.ctl;
  bool act = a.active ? (a.active[s] != 0) : ((long long)c.i < a.sp.len(s));
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  for (int r = warp; r < kFdmRowsPerCta; r += 8) {
    const int i = row0 + r;
    if (i >= Fp) break;
    const size_t ro = ((size_t)s * Fp + i) * Fp;
    if (!act) {
      if (lane == 0) store_dxp(a, s, i, 0.f);
      if (!a.update)
        for (int j = lane; j < Fp; j += 32) a.gU[ro + j] = 0.f;
      continue;
    }
    const float xi = a.Xp[(size_t)s * Fp + i];
    float dot = 0.f;
    for (int j = lane; j < Fp; j += 32) {
      float dyj = a.dY[(size_t)s * Fp + j];
      float u = a.U[ro + j];
      dot += u * dyj;
      if (a.update) {
        float m = a.Um[ro + j], v = a.Uv[ro + j];
        adam1(u, m, v, xi * dyj, c.lr, c.bc1, c.bc2);
        a.U[ro + j] = u;
        a.Um[ro + j] = m;
        a.Uv[ro + j] = v;
      } else {
        a.gU[ro + j] = xi * dyj;
      }
    }
    dot = warp_sum(dot);
    if (lane == 0) store_dxp(a, s, i, dot);
  }
}

cudaError_t launch_fdm_bwd(const FdmBwdArgs& a, cudaStream_t st) {
  dim3 grid(div_up(a.Fp, kFdmRowsPerCta), a.b);
  cudaError_t e = cudaSuccess;
  switch (a.Fp) {
    case 128: e = launch_k(fdm_bwd_kernel<1>, dim3(grid), dim3(256), 0, st, a); break;
    case 256: e = launch_k(fdm_bwd_kernel<2>, dim3(grid), dim3(256), 0, st, a); break;
    case 384: e = launch_k(fdm_bwd_kernel<3>, dim3(grid), dim3(256), 0, st, a); break;
    case 512: e = launch_k(fdm_bwd_kernel<4>, dim3(grid), dim3(256), 0, st, a); break;
    case 1024: e = launch_k(fdm_bwd_kernel<8>, dim3(grid), dim3(256), 0, st, a); break;
    default: e = launch_k(fdm_bwd_generic_kernel, dim3(grid), dim3(256), 0, st, a); break;
  }
  return e;
}

__global__ void __launch_bounds__(256) fdm_dx_generic_kernel(FdmSplitArgs a) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StepCtl c = *a.ctl;
  if (blockIdx.x == 0 && s == 0 && threadIdx.x == 0) *a.pend = FdmPend{c.i, c.lr, c.bc1, c.bc2};
  const bool act = fdm_split_active(a, s, c.i);
  if (blockIdx.x == 0 && act)
    for (int j = threadIdx.x; j < Fp; j += blockDim.x) {
      a.xp_pend[(size_t)s * Fp + j] = a.Xp[(size_t)s * Fp + j];
      a.dy_pend[(size_t)s * Fp + j] = a.dY[(size_t)s * Fp + j];
    }
  FdmBwdArgs o{};
  o.dXp = a.dXp;
  o.dXpb = a.dXpb;
  o.dXpbT = a.dXpbT;
  o.ldT = a.ldT;
  o.Fp = Fp;
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  for (int r = warp; r < kFdmRowsPerCta; r += 8) {
    const int i = row0 + r;
    if (i >= Fp) break;
    float dot = 0.f;
    if (act)
      for (int j = lane; j < Fp; j += 32) dot += a.U[((size_t)s * Fp + i) * Fp + j] * a.dY[(size_t)s * Fp + j];
    dot = warp_sum(dot);
    if (lane == 0) store_dxp(o, s, i, act ? dot : 0.f);
  }
}

__global__ void __launch_bounds__(256) fdm_adam_generic_kernel(FdmSplitArgs a) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const FdmPend pd = *a.pend;
  if (!fdm_split_active(a, s, pd.i)) return;
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  for (int r = warp; r < kFdmRowsPerCta; r += 8) {
    const int i = row0 + r;
    if (i >= Fp) break;
    const size_t ro = ((size_t)s * Fp + i) * Fp;
    const float xi = a.xp_pend[(size_t)s * Fp + i];
    const float* src = a.Ub ? a.Ub : a.U;
    for (int j = lane; j < Fp; j += 32) {
      float u = src[ro + j], m = a.Um[ro + j], v = a.Uv[ro + j];
      adam1(u, m, v, xi * a.dy_pend[(size_t)s * Fp + j], pd.lr, pd.bc1, pd.bc2);
      a.U[ro + j] = u;
      a.Um[ro + j] = m;
      a.Uv[ro + j] = v;
    }
  }
}

cudaError_t launch_fdm_dx(const FdmSplitArgs& a, cudaStream_t st) {
  dim3 grid(div_up(a.Fp, kFdmRowsPerCta), a.b);
  switch (a.Fp) {
    case 128: return launch_k(fdm_dx_kernel<1>, grid, dim3(256), 0, st, a);
    case 256: return launch_k(fdm_dx_kernel<2>, grid, dim3(256), 0, st, a);
    case 384: return launch_k(fdm_dx_kernel<3>, grid, dim3(256), 0, st, a);
    case 512: return launch_k(fdm_dx_kernel<4>, grid, dim3(256), 0, st, a);
    case 1024: return launch_k(fdm_dx_kernel<8>, grid, dim3(256), 0, st, a);
    default: return launch_k(fdm_dx_generic_kernel, grid, dim3(256), 0, st, a);
  }
}

template <int NCH>
cudaError_t launch_adam_persist(const FdmSplitArgs& a, cudaStream_t st) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // The CTA stays resident for the whole update: keep its SM configured for
    // the largest shared-memory carveout, so GEMM CTAs still fit beside it.
    e = cudaFuncSetAttribute(fdm_adam_persist_kernel<NCH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return launch_k(fdm_adam_persist_kernel<NCH>, dim3(sms), dim3(32 * kAdamWarps), 0, st, a);
}

cudaError_t launch_fdm_adam(const FdmSplitArgs& a, cudaStream_t st, bool persistent) {
  if (persistent) switch (a.Fp) {
      case 128: return launch_adam_persist<1>(a, st);
      case 256: return launch_adam_persist<2>(a, st);
      case 384: return launch_adam_persist<3>(a, st);
      case 512: return launch_adam_persist<4>(a, st);
      case 1024: return launch_adam_persist<8>(a, st);
      default: break;
    }
  dim3 grid(div_up(a.Fp, kFdmRowsPerCta), a.b);
  switch (a.Fp) {
    case 128: return launch_k(fdm_adam_kernel<1>, grid, dim3(256), 0, st, a);
    case 256: return launch_k(fdm_adam_kernel<2>, grid, dim3(256), 0, st, a);
    case 384: return launch_k(fdm_adam_kernel<3>, grid, dim3(256), 0, st, a);
    case 512: return launch_k(fdm_adam_kernel<4>, grid, dim3(256), 0, st, a);
    case 1024: return launch_k(fdm_adam_kernel<8>, grid, dim3(256), 0, st, a);
    default: return launch_k(fdm_adam_generic_kernel, grid, dim3(256), 0, st, a);
  }
}

// ============================================================================================
// Embedding backward: scatter-add of dh0 into E's rows, owner computes.
// CTA (c, q) owns byte value c and chunk q of kEmbChunkPos consecutive
// positions. Warp w of 8 takes a contiguous eighth of the chunk, read 128
// positions at a time (one 32-bit word per lane, coalesced, four words
// prefetched); ballots find the positions p with ctx[p] == c, which the warp
// visits in increasing p: lane d adds dh0[p][d] (and d + 32 when D > 32),
// eight rows' loads in flight at a time. The 8 warp sums are added in warp
// order. With one chunk that is dE[c]; with several, each CTA writes its
// partial and the last CTA of c to arrive adds the chunks' partials in chunk
// order (a fence precedes the arrival counter), so the result does not depend
// on timing. Position p = s*K + k has its D gradient values at dX[p*D ..).
// ============================================================================================
__global__ void __launch_bounds__(256) embed_bwd_owner_kernel(const uint8_t* __restrict__ ctx,
                                                              const float* __restrict__ dX, int P, int D,
                                                              float* __restrict__ dE, float* __restrict__ part,
                                                              unsigned* __restrict__ cnt) {
  pdl_wait();
  pdl_launch();
  __shared__ float wsum[8][64];
  __shared__ int is_last;
  const uint32_t c = blockIdx.x;
  const int nq = gridDim.y, q = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c_lo = min(P, q * kEmbChunkPos), c_hi = min(P, c_lo + kEmbChunkPos);
  const int per = ((c_hi - c_lo + 8 * 128 - 1) / (8 * 128)) * 128;  // positions per warp, a multiple of 128
  const int p_lo = min(c_hi, c_lo + w * per), p_hi = min(c_hi, p_lo + per);
  const bool al4 = (reinterpret_cast<uintptr_t>(ctx) & 3) == 0;
  float a0 = 0.f, a1 = 0.f;  // dims lane and lane + 32
  int pend[8];
  int np = 0;
  auto flush = [&]() {
    float v0[8], v1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v0[k] = (k < np && lane < D) ? dX[(size_t)pend[k] * D + lane] : 0.f;
      v1[k] = (k < np && lane + 32 < D) ? dX[(size_t)pend[k] * D + lane + 32] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k < np) {
        a0 += v0[k];
        a1 += v1[k];
      }
    }
    np = 0;
  };
  auto word = [&](int pw) -> uint32_t {  // positions pw..pw+3 (a non-matching byte past p_hi)
    if (al4 && pw + 4 <= p_hi) return *reinterpret_cast<const uint32_t*>(ctx + pw);
    uint32_t x = 0;
    for (int u = 0; u < 4; ++u) x |= (uint32_t)(pw + u < p_hi ? ctx[pw + u] : (uint8_t)(c ^ 1u)) << (8 * u);
    return x;
  };
  for (int pb = p_lo; pb < p_hi; pb += 4 * 128) {
    uint32_t xs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xs[k] = (pb + k * 128 < p_hi) ? word(pb + k * 128 + 4 * lane) : (c ^ 1u) * 0x01010101u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int p0 = pb + k * 128;
      uint32_t m[4], any = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        m[u] = __ballot_sync(0xffffffffu, ((xs[k] >> (8 * u)) & 0xffu) == c);
        any |= m[u];
      }
      while (any) {  // warp-uniform: lanes l in increasing order, then their bytes u
        const int l = __ffs(any) - 1;
        any &= any - 1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if ((m[u] >> l) & 1u) {
            pend[np++] = p0 + 4 * l + u;
            if (np == 8) flush();
          }
        }
      }
    }
  }
  flush();
  wsum[w][lane] = a0;
  wsum[w][lane + 32] = a1;
  __syncthreads();
  const int t = threadIdx.x;
  float sum = 0.f;
  if (t < D) {
    sum = wsum[0][t];
#pragma unroll
    for (int ww = 1; ww < 8; ++ww) sum += wsum[ww][t];
  }
  if (nq == 1) {
    if (t < D) dE[(size_t)c * D + t] = sum;
    return;
  }
  if (t < D) {
    part[((size_t)c * nq + q) * D + t] = sum;
    __threadfence();
  }
  __syncthreads();
  if (t == 0) is_last = (atomicAdd(&cnt[c], 1u) == (unsigned)(nq - 1));
  __syncthreads();
  if (is_last && t < D) {
    __threadfence();
    const float* src = part + (size_t)c * nq * D + t;
    float acc = 0.f;
    for (int k = 0; k < nq; ++k) acc += __ldcg(src + (size_t)k * D);
    dE[(size_t)c * D + t] = acc;
    if (t == 0) cnt[c] = 0u;
  }
}

int embed_bwd_chunks(int b, int K) { return (b * K + kEmbChunkPos - 1) / kEmbChunkPos; }

cudaError_t launch_embed_bwd(const uint8_t* ctx, const float* dX, int b, int K, int D, float* dE, float* part,
                             unsigned* cnt, cudaStream_t st) {
  if (D > 64) return cudaErrorInvalidValue;
  const int nq = embed_bwd_chunks(b, K);
  if (nq > 1 && (!part || !cnt)) return cudaErrorInvalidValue;
  return launch_k(embed_bwd_owner_kernel, dim3(256, nq < 1 ? 1 : nq), dim3(256), 0, st, ctx, dX, b * K, D, dE, part,
                  cnt);
}

// Grouped embedding adjoint: CTA (group g, pair of byte values); warps 4v to
// 4v + 3 own byte value 2 cb + v, each one quarter of the group's context
// positions (in blocks of 512). A warp walks its quarter in increasing order,
// 512 positions at a time (four 32-bit words of 4 positions per lane, loaded
// together), finds the value's positions by ballot and adds their gradient
// rows (lane d: dimensions d and d + 32) in position order, eight rows'
// loads in flight at a time; the four quarter sums are then added in order.
// So each dE[g][c] is a fixed-order sum that depends on the group alone.
__global__ void __launch_bounds__(256) embed_bwd_groups_kernel(const uint8_t* __restrict__ ctx,
                                                               const float* __restrict__ dX, int K, int D,
                                                               float* __restrict__ dE,
                                                               const GroupInfo* __restrict__ gi, size_t gs) {
  pdl_wait();
  pdl_launch();
  __shared__ float part[8][64];
  const GroupInfo g = gi[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t c = blockIdx.y * 2 + (w >> 2);
  // the group's streams only: its padding rows never hold a byte (their
  // gradient is zero) and their all-zero contexts would all match byte 0
  const int g_lo = g.r0 * K, g_hi = (g.r0 + g.s) * K;
  const int per = ((g_hi - g_lo + 4 * 512 - 1) / (4 * 512)) * 512;  // a quarter, whole 512-position blocks
  const int p_lo = min(g_hi, g_lo + (w & 3) * per), p_hi = min(g_hi, p_lo + per);
  float a0 = 0.f, a1 = 0.f;
  int pend[8];
  int np = 0;
  auto flush = [&]() {
    float v0[8], v1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v0[k] = (k < np && lane < D) ? dX[(size_t)pend[k] * D + lane] : 0.f;
      v1[k] = (k < np && lane + 32 < D) ? dX[(size_t)pend[k] * D + lane + 32] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k < np) {
        a0 += v0[k];
        a1 += v1[k];
      }
    }
    np = 0;
  };
  for (int pb = p_lo; pb < p_hi; pb += 4 * 128) {
    uint32_t xs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // positions pw..pw+3 (p_lo is a multiple of 4; bytes at or past p_hi never match)
      const int pw = pb + k * 128 + 4 * lane;
      uint32_t x = pw < p_hi ? *reinterpret_cast<const uint32_t*>(ctx + pw) : (c ^ 1u) * 0x01010101u;
      for (int u = 0; u < 4; ++u)
        if (pw + u >= p_hi) x = (x & ~(0xFFu << (8 * u))) | ((c ^ 1u) & 0xFFu) << (8 * u);
      xs[k] = x;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int p0 = pb + k * 128;
      uint32_t m[4], any = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        m[u] = __ballot_sync(0xffffffffu, ((xs[k] >> (8 * u)) & 0xffu) == c);
        any |= m[u];
      }
      while (any) {  // warp-uniform: lanes in increasing order, then their bytes
        const int l = __ffs(any) - 1;
        any &= any - 1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if ((m[u] >> l) & 1u) {
            pend[np++] = p0 + 4 * l + u;
            if (np == 8) flush();
          }
        }
      }
    }
  }
  flush();
  part[w][lane] = a0;
  part[w][lane + 32] = a1;
  __syncthreads();
  if ((w & 3) == 0) {
    float* out = dE + (size_t)blockIdx.x * gs + (size_t)c * D;
    if (lane < D) out[lane] = ((part[w][lane] + part[w + 1][lane]) + part[w + 2][lane]) + part[w + 3][lane];
    if (lane + 32 < D)
      out[lane + 32] = ((part[w][lane + 32] + part[w + 1][lane + 32]) + part[w + 2][lane + 32]) + part[w + 3][lane + 32];
  }
}

cudaError_t launch_embed_bwd_groups(const uint8_t* ctx, const float* dX, int K, int D, float* dE,
                                    const GroupInfo* gi, int ngroups, size_t gs, cudaStream_t st) {
  if (D > 64 || ngroups < 1 || ngroups > 65535 || !gi || (reinterpret_cast<uintptr_t>(ctx) & 3))
    return cudaErrorInvalidValue;
  return launch_k(embed_bwd_groups_kernel, dim3(ngroups, 128), dim3(256), 0, st, ctx, dX, K, D, dE, gi, gs);
}

// ============================================================================================
// Adam on the shared parameters (Sec. 4.1: lr 1e-3; beta, eps as documented).
// ============================================================================================
// P is read from Pin and written to P (Pin == P: in place; the delayed-update
// schedule writes the next parameters beside the current ones).
__global__ void adam_kernel(float* P, const float* Pin, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, size_t n, const StepCtl* __restrict__ ctl) {
  pdl_wait();
  pdl_launch();
  const StepCtl c = *ctl;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float p = Pin[e], m = M[e], v = V[e];
    const float gr = G[e];
    adam1(p, m, v, gr, c.lr, c.bc1, c.bc2);
    P[e] = p;
    M[e] = m;
    V[e] = v;
  }
}

cudaError_t launch_adam(float* P, const float* G, float* M, float* V, size_t n, const StepCtl* ctl,
                        cudaStream_t st, const float* Pin) {
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  return launch_k(adam_kernel, dim3(grid), dim3(256), 0, st, P, Pin ? Pin : P, G, M, V, n, ctl);
}

// ============================================================================================
// Step control: advance to the next time index and derive its scalars.
// ============================================================================================
// Reads the step control of the current step from `src` and writes the next
// step's to `dst` (the same record, or the other of the delayed-update
// schedule's two, whose sticky error bits are kept).
// The control record of the next step (i + 1) from that of the current one.
__device__ __forceinline__ StepCtl advance_ctl(StepCtl c, int dst_err, Split sp, int K, int ring_slots, int b) {
  c.err |= dst_err;
  c.i += 1;
  c.t += 1;
  long long i = c.i;
  int bact;
  if (sp.cp) {
    // uneven split: the count changes only at the table's time indices
    bact = c.bact;
    while (c.cpi < sp.ncp && sp.cp[c.cpi].i <= i) bact = sp.cp[c.cpi++].bact;
  } else {
    bact = (i < sp.q) ? b : (i == sp.q ? sp.rem : 0);
  }
  c.bact = bact;
  c.inv_bact = bact > 0 ? 1.0f / (float)bact : 0.f;
  c.bc1 = 1.0f - powf(kB1, (float)c.t);
  c.bc2 = 1.0f - powf(kB2, (float)c.t);
  c.slot = (int)((i - K) % ring_slots);
  return c;
}

__global__ void step_advance_kernel(const StepCtl* src, StepCtl* dst, Split sp, int K, int ring_slots, int b) {
  pdl_wait();
  pdl_launch();
  *dst = advance_ctl(*src, dst->err, sp, K, ring_slots, b);
}
cudaError_t launch_step_advance(StepCtl* ctl, Split sp, int K, int ring_slots, int b, cudaStream_t st,
                                StepCtl* dst) {
  return launch_k(step_advance_kernel, dim3(1), dim3(1), 0, st, (const StepCtl*)ctl, dst ? dst : ctl, sp, K,
                  ring_slots, b);
}

// ============================================================================================
// Range coder (32-bit, carry-propagating). See the oracle's coder for the
// same rule: r = R >> 16; low += r*cum; R = r*f (or R - r*cum for the last
// symbol); renormalise bytewise below 2^24 with cache + pending 0xFF bytes.
// ============================================================================================
struct EncIO {
  uint8_t* out;
  uint32_t cap;
};

__device__ __forceinline__ void enc_emit(EncState& s, EncIO& io, uint32_t byte) {
  if (s.pos < io.cap) {
    io.out[s.pos++] = (uint8_t)byte;
  } else {
    s.err = 1;
  }
}

__device__ __forceinline__ void enc_shift_low(EncState& s, EncIO& io) {
  if (s.low < 0xFF000000ull || s.low >= (1ull << 32)) {
    uint32_t carry = (uint32_t)(s.low >> 32);
    if (s.started) enc_emit(s, io, (s.cache + carry) & 0xFF);
    for (; s.pending; --s.pending) enc_emit(s, io, (0xFF + carry) & 0xFF);
    s.cache = (uint32_t)(s.low >> 24) & 0xFF;
    s.started = 1;
  } else {
    s.pending++;
  }
  s.low = (s.low & 0x00FFFFFFull) << 8;
}

__device__ __forceinline__ void enc_symbol(EncState& s, EncIO& io, uint32_t cum, uint32_t f) {
  uint32_t r = s.range >> kTBits;
  s.low += (unsigned long long)r * cum;
  if (cum + f == (uint32_t)kT)
    s.range -= r * cum;
  else
    s.range = r * f;
  while (s.range < kTop) {
    s.range <<= 8;
    enc_shift_low(s, io);
  }
}

__device__ __forceinline__ void enc_init(EncState& s) {
  s.low = 0;
  s.range = 0xFFFFFFFFu;
  s.cache = 0;
  s.pending = 0;
  s.started = 0;
  s.pos = 0;
  s.err = 0;
}

__global__ void prefix_encode_kernel(EncState* es, const uint8_t* __restrict__ data, Split sp, int K, int b,
                                     uint8_t* out, const unsigned long long* out_off, const uint32_t* out_cap) {
  pdl_wait();
  pdl_launch();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= b) return;
  EncState st;
  enc_init(st);
  EncIO io{out + out_off[s], out_cap[s]};
  long long n = sp.len(s) < K ? sp.len(s) : K;
  const uint8_t* x = data + sp.off(s);
  for (long long i = 0; i < n; ++i) enc_symbol(st, io, 256u * x[i], 256u);
  es[s] = st;
}

cudaError_t launch_prefix_encode(EncState* es, const uint8_t* data, Split sp, int K, int b, uint8_t* out,
                                 const unsigned long long* out_off, const uint32_t* out_cap, cudaStream_t st) {
  return launch_k(prefix_encode_kernel, dim3(div_up(b, 128)), dim3(128), 0, st, es, data, sp, K, b, out, out_off, out_cap);
}

// One thread per stream codes `nsteps` consecutive ring slots. Reads of a slot
// are coalesced across the streams of a warp.
__global__ void range_encode_kernel(EncState* es, const uint32_t* __restrict__ ring, int ring_slots, int slot0,
                                    int nsteps, int b, uint8_t* out, const unsigned long long* out_off,
                                    const uint32_t* out_cap) {
  pdl_wait();
  pdl_launch();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= b) return;
  EncState st = es[s];
  EncIO io{out + out_off[s], out_cap[s]};
  int slot = slot0;
  for (int t = 0; t < nsteps; ++t) {
    uint32_t w = ring[(size_t)slot * b + s];
    if (w != kSkip) enc_symbol(st, io, w & 0xFFFFu, (w >> 16) + 1u);
    if (++slot == ring_slots) slot = 0;
  }
  es[s] = st;
}

cudaError_t launch_range_encode(EncState* es, const uint32_t* ring, int ring_slots, int slot0, int nsteps, int b,
                                uint8_t* out, const unsigned long long* out_off, const uint32_t* out_cap,
                                cudaStream_t st) {
  if (nsteps <= 0) return cudaSuccess;
  return launch_k(range_encode_kernel, dim3(div_up(b, 128)), dim3(128), 0, st, es, ring, ring_slots, slot0, nsteps, b, out, out_off,
                                                       out_cap);
}

__global__ void encode_flush_kernel(EncState* es, int b, uint8_t* out, const unsigned long long* out_off,
                                    const uint32_t* out_cap, uint32_t* out_len) {
  pdl_wait();
  pdl_launch();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= b) return;
  EncState st = es[s];
  EncIO io{out + out_off[s], out_cap[s]};
  // The value low rounded up to a multiple of 2^24 lies in [low, low + R).
  st.low = (st.low + (kTop - 1)) & ~(unsigned long long)(kTop - 1);
  enc_shift_low(st, io);
  enc_shift_low(st, io);
  uint32_t n = st.pos;
  while (n > 0 && io.out[n - 1] == 0) --n;  // the decoder reads missing bytes as zero
  out_len[s] = st.err ? 0xFFFFFFFFu : n;
  es[s] = st;
}

cudaError_t launch_encode_flush(EncState* es, int b, uint8_t* out, const unsigned long long* out_off,
                                const uint32_t* out_cap, uint32_t* out_len, cudaStream_t st) {
  return launch_k(encode_flush_kernel, dim3(div_up(b, 128)), dim3(128), 0, st, es, b, out, out_off, out_cap, out_len);
}

__device__ __forceinline__ uint32_t dec_byte(const uint8_t* in, uint32_t len, uint32_t& pos) {
  uint32_t v = pos < len ? in[pos] : 0u;
  ++pos;
  return v;
}

__device__ __forceinline__ void dec_update(DecState& d, const uint8_t* in, uint32_t len, uint32_t r, uint32_t c,
                                           uint32_t f) {
  d.code -= r * c;
  d.range = (c + f == (uint32_t)kT) ? d.range - r * c : r * f;
  while (d.range < kTop) {
    d.code = (d.code << 8) | dec_byte(in, len, d.pos);
    d.range <<= 8;
  }
}

__global__ void dec_init_kernel(DecState* ds, const uint8_t* bits, const unsigned long long* off,
                                const uint32_t* len, int b) {
  pdl_wait();
  pdl_launch();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= b) return;
  DecState d;
  d.pos = 0;
  d.range = 0xFFFFFFFFu;
  d.code = 0;
  d.err = 0;
  const uint8_t* in = bits + off[s];
  for (int k = 0; k < 4; ++k) d.code = (d.code << 8) | dec_byte(in, len[s], d.pos);
  ds[s] = d;
}

cudaError_t launch_dec_init(DecState* ds, const uint8_t* bits, const unsigned long long* off, const uint32_t* len,
                            int b, cudaStream_t st) {
  return launch_k(dec_init_kernel, dim3(div_up(b, 128)), dim3(128), 0, st, ds, bits, off, len, b);
}

__global__ void prefix_decode_kernel(DecState* ds, const uint8_t* bits, const unsigned long long* off,
                                     const uint32_t* len, Split sp, int K, int b, uint8_t* data) {
  pdl_wait();
  pdl_launch();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= b) return;
  DecState d = ds[s];
  const uint8_t* in = bits + off[s];
  const uint32_t L = len[s];
  long long n = sp.len(s) < K ? sp.len(s) : K;
  uint8_t* x = data + sp.off(s);
  for (long long i = 0; i < n; ++i) {
    uint32_t r = d.range >> kTBits;
    uint32_t target = d.code / r;
    if (target > (uint32_t)kT - 1) target = kT - 1;
    uint32_t sym = target >> 8;
    dec_update(d, in, L, r, sym << 8, 256u);
    x[i] = (uint8_t)sym;
  }
  ds[s] = d;
}

cudaError_t launch_prefix_decode(DecState* ds, const uint8_t* bits, const unsigned long long* off,
                                 const uint32_t* len, Split sp, int K, int b, uint8_t* data, cudaStream_t st) {
  return launch_k(prefix_decode_kernel, dim3(div_up(b, 128)), dim3(128), 0, st, ds, bits, off, len, sp, K, b, data);
}

// ============================================================================================
// Head: softmax -> integer CDF -> (encode slot | decode symbol) -> CE gradient.
// One warp per stream; lane l owns symbols 8l..8l+7.
// CDF rule: f_j = 1 + floor(fl32(p_j * 65280)); the remainder 2^16 - sum f goes
// to the first largest f; cum is the exclusive prefix sum.
// ============================================================================================
struct RowCdf {
  uint32_t f[8];
  uint32_t cum[8];  // exclusive prefix within the whole row
};

__device__ __forceinline__ void row_cdf(const float (&p)[8], int lane, RowCdf& o) {
  int fsum = 0;
  uint32_t best = 0;
  int bidx = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    o.f[q] = 1u + (uint32_t)floorf(__fmul_rn(p[q], (float)(kT - 256)));
    fsum += (int)o.f[q];
    if (o.f[q] > best) {
      best = o.f[q];
      bidx = lane * 8 + q;
    }
  }
  const int total = warp_isum(fsum);
  // argmax of f, lowest index on ties
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    uint32_t ob = __shfl_xor_sync(0xffffffffu, best, off);
    int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
    if (ob > best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  const int rem = kT - total;
  if ((bidx >> 3) == lane) o.f[bidx & 7] = (uint32_t)((int)o.f[bidx & 7] + rem);
  uint32_t run = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    o.cum[q] = run;
    run += o.f[q];
  }
  // exclusive scan of lane totals
  uint32_t incl = run;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  const uint32_t excl = incl - run;
#pragma unroll
  for (int q = 0; q < 8; ++q) o.cum[q] += excl;
}

// Transposed BF16 store of an [R][cols] tile held in shared memory:
// YT[c][r0 + r] for r < R, as 16-byte stores (R = 8 or 16).
template <int R>
__device__ __forceinline__ void store_tile_T(const __nv_bfloat16* tile, int ld_s, int cols, int r0,
                                             __nv_bfloat16* YT, int ldT) {
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    __align__(16) __nv_bfloat16 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tile[r * ld_s + c];
    uint4* dst = reinterpret_cast<uint4*>(YT + (size_t)c * ldT + r0);
#pragma unroll
    for (int q = 0; q < R / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(v)[q];
  }
}

__global__ void __launch_bounds__(32 * kRowsT) head_kernel(HeadArgs a) {
  pdl_wait();
  pdl_launch();
  __shared__ __nv_bfloat16 tile[kRowsT][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kRowsT + warp;
  const bool valid = s < a.b;  // warp-uniform
  const StepCtl c = *a.ctl;
  float dzv[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) dzv[q] = 0.f;
  if (valid) {
    const float* z = a.z + (size_t)s * 256 + lane * 8;
    float zz[8], p[8];
    float4 z0 = reinterpret_cast<const float4*>(z)[0], z1 = reinterpret_cast<const float4*>(z)[1];
    zz[0] = z0.x; zz[1] = z0.y; zz[2] = z0.z; zz[3] = z0.w;
    zz[4] = z1.x; zz[5] = z1.y; zz[6] = z1.z; zz[7] = z1.w;
    float mx = zz[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) mx = fmaxf(mx, zz[q]);
    mx = warp_max(mx);
    float se = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      p[q] = expf(zz[q] - mx);
      se += p[q];
    }
    se = warp_sum(se);
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = p[q] / se;

    bool active;
    if (a.mode == 2)
      active = a.active[s] != 0;
    else
      active = (long long)c.i < a.sp.len(s);

    RowCdf cdf;
    row_cdf(p, lane, cdf);
    if (a.freq_out) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        a.freq_out[(size_t)s * 256 + lane * 8 + q] = cdf.f[q];
        a.cum_out[(size_t)s * 257 + lane * 8 + q] = cdf.cum[q];
      }
      if (lane == 31) a.cum_out[(size_t)s * 257 + 256] = (uint32_t)kT;
    }

    int x = -1;
    if (active) {
      if (a.mode == 0) {
        x = a.data[a.sp.off(s) + c.i];  // warp-uniform
        uint32_t cx = __shfl_sync(0xffffffffu, cdf.cum[x & 7], x >> 3);
        uint32_t fx = __shfl_sync(0xffffffffu, cdf.f[x & 7], x >> 3);
        if (lane == 0) a.ring[(size_t)c.slot * a.b + s] = cx | ((fx - 1u) << 16);
      } else if (a.mode == 1) {
        DecState d;
        uint32_t target = 0, r = 0;
        if (lane == 0) {
          d = a.dec[s];
          r = d.range >> kTBits;
          target = d.code / r;
          if (target > (uint32_t)kT - 1) target = kT - 1;
        }
        target = __shfl_sync(0xffffffffu, target, 0);
        unsigned ball = __ballot_sync(0xffffffffu, cdf.cum[0] <= target);
        int L = 31 - __clz(ball);
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) cnt += (cdf.cum[q] <= target) ? 1 : 0;
        cnt = __shfl_sync(0xffffffffu, cnt, L);
        x = L * 8 + cnt - 1;
        uint32_t cx = __shfl_sync(0xffffffffu, cdf.cum[x & 7], L);
        uint32_t fx = __shfl_sync(0xffffffffu, cdf.f[x & 7], L);
        if (lane == 0) {
          dec_update(d, a.bits + a.bits_off[s], a.bits_len[s], r, cx, fx);
          a.dec[s] = d;
          a.data[a.sp.off(s) + c.i] = (uint8_t)x;
        }
      } else {
        x = a.targets[s];
      }
    } else if (a.mode == 0 && lane == 0) {
      a.ring[(size_t)c.slot * a.b + s] = kSkip;
    }

    float* dz = a.dz + (size_t)s * 256 + lane * 8;
    float* po = a.p ? a.p + (size_t)s * 256 + lane * 8 : nullptr;
    float inv = c.inv_bact;
    if (a.rg) {  // grouped mode: the mean over the row's own group (as set_ctl / step_advance form it)
      const int n = group_active(a.gi[a.rg[s]], c.i);
      inv = n > 0 ? 1.0f / (float)n : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int j = lane * 8 + q;
      dzv[q] = active ? (p[q] - (j == x ? 1.0f : 0.0f)) * inv : 0.f;
      dz[q] = dzv[q];
      if (po) po[q] = p[q];
    }
    if (a.dzb) {
      __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) hb[q] = __float2bfloat16_rn(dzv[q]);
      *reinterpret_cast<uint4*>(a.dzb + (size_t)s * 256 + lane * 8) = *reinterpret_cast<const uint4*>(hb);
    }
  }
  if (a.dzbT) {
#pragma unroll
    for (int q = 0; q < 8; ++q) tile[warp][lane * 8 + q] = __float2bfloat16_rn(dzv[q]);
    __syncthreads();
    store_tile_T<kRowsT>(&tile[0][0], 256, 256, blockIdx.x * kRowsT, a.dzbT, a.ldT);
  }
}

cudaError_t launch_head(const HeadArgs& a, cudaStream_t st) {
  return launch_k(head_kernel, dim3(div_up(a.b, kRowsT)), dim3(32 * kRowsT), 0, st, a);
}

__global__ void cdf_quantize_kernel(const float* __restrict__ P, int rows, uint32_t* freq, uint32_t* cum) {
  pdl_wait();
  pdl_launch();
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= rows) return;
  float p[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) p[q] = P[(size_t)s * 256 + lane * 8 + q];
  RowCdf cdf;
  row_cdf(p, lane, cdf);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    freq[(size_t)s * 256 + lane * 8 + q] = cdf.f[q];
    cum[(size_t)s * 257 + lane * 8 + q] = cdf.cum[q];
  }
  if (lane == 31) cum[(size_t)s * 257 + 256] = (uint32_t)kT;
}

cudaError_t launch_cdf_quantize(const float* p, int rows, uint32_t* freq, uint32_t* cum, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  return launch_k(cdf_quantize_kernel, dim3(div_up(rows, 8)), dim3(256), 0, st, p, rows, freq, cum);
}

// ============================================================================================
// BF16 path: LayerNorm forward / backward with fused BF16 operand copies.
// kRowsLN warps per CTA, one row each; the BF16 rows are staged in shared memory
// and written transposed ([c][row], 16-byte runs) for the dW GEMMs.
// ============================================================================================
constexpr int kRowsLN = 8;  // rows (warps) per CTA of the LayerNorm kernels

// NPL = F / 32 values per lane held in registers (all loads issued up front);
// NPL = 0 is the generic loop for any F.
template <int NPL>
__global__ void __launch_bounds__(32 * kRowsLN)
    ln_fwd_bf16_kernel(const float* __restrict__ X, const float* __restrict__ g, const float* __restrict__ be,
                       float* __restrict__ xhat, float* __restrict__ rstd, __nv_bfloat16* __restrict__ X0b,
                       __nv_bfloat16* __restrict__ X0bT, int b, int F, int ldT, const int* __restrict__ rg,
                       size_t gs) {
  pdl_wait();
  pdl_launch();
  extern __shared__ __nv_bfloat16 tile_dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsLN + warp;
  __nv_bfloat16* trow = tile_dyn + (size_t)warp * F;
  if (row < b) {
    if (rg) {  // grouped mode: the row's own gamma and beta
      g += (size_t)rg[row] * gs;
      be += (size_t)rg[row] * gs;
    }
    const float* x = X + (size_t)row * F;
    if (NPL > 0) {
      float v[NPL > 0 ? NPL : 1];
#pragma unroll
      for (int q = 0; q < NPL; ++q) v[q] = x[lane + 32 * q];
      float sm = 0.f;
#pragma unroll
      for (int q = 0; q < NPL; ++q) sm += v[q];
      const float mean = warp_sum(sm) / (float)F;
      float qv = 0.f;
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        const float d = v[q] - mean;
        qv += d * d;
      }
      const float r = 1.0f / sqrtf(warp_sum(qv) / (float)F + kLnEps);
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        const int c = lane + 32 * q;
        const float h = (v[q] - mean) * r;
        xhat[(size_t)row * F + c] = h;
        const __nv_bfloat16 o = __float2bfloat16_rn(h * g[c] + be[c]);
        X0b[(size_t)row * F + c] = o;
        trow[c] = o;
      }
      if (lane == 0) rstd[row] = r;
    } else {
      float sm = 0.f;
      for (int c = lane; c < F; c += 32) sm += x[c];
      const float mean = warp_sum(sm) / (float)F;
      float qv = 0.f;
      for (int c = lane; c < F; c += 32) {
        const float d = x[c] - mean;
        qv += d * d;
      }
      const float r = 1.0f / sqrtf(warp_sum(qv) / (float)F + kLnEps);
      for (int c = lane; c < F; c += 32) {
        const float h = (x[c] - mean) * r;
        xhat[(size_t)row * F + c] = h;
        const __nv_bfloat16 o = __float2bfloat16_rn(h * g[c] + be[c]);
        X0b[(size_t)row * F + c] = o;
        trow[c] = o;
      }
      if (lane == 0) rstd[row] = r;
    }
  } else {
    for (int c = lane; c < F; c += 32) trow[c] = __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  store_tile_T<kRowsLN>(tile_dyn, F, F, blockIdx.x * kRowsLN, X0bT, ldT);
}

cudaError_t launch_ln_fwd_bf16(const float* X, const float* g, const float* be, float* xhat, float* rstd,
                               __nv_bfloat16* X0b, __nv_bfloat16* X0bT, int b, int F, int ldT, cudaStream_t st,
                               const int* rg, size_t gs) {
  const size_t smem = (size_t)kRowsLN * F * sizeof(__nv_bfloat16);
  const dim3 grid(div_up(b, kRowsLN)), block(32 * kRowsLN);
  switch (F) {
    case 128:
      return launch_k(ln_fwd_bf16_kernel<4>, grid, block, smem, st, X, g, be, xhat, rstd, X0b, X0bT, b, F, ldT, rg, gs);
    case 256:
      return launch_k(ln_fwd_bf16_kernel<8>, grid, block, smem, st, X, g, be, xhat, rstd, X0b, X0bT, b, F, ldT, rg, gs);
    case 512:
      return launch_k(ln_fwd_bf16_kernel<16>, grid, block, smem, st, X, g, be, xhat, rstd, X0b, X0bT, b, F, ldT, rg,
                      gs);
    case 1024:
      return launch_k(ln_fwd_bf16_kernel<32>, grid, block, smem, st, X, g, be, xhat, rstd, X0b, X0bT, b, F, ldT, rg,
                      gs);
    default:
      return launch_k(ln_fwd_bf16_kernel<0>, grid, block, smem, st, X, g, be, xhat, rstd, X0b, X0bT, b, F, ldT, rg, gs);
  }
}

// Embedding (the model input) and the first block's LayerNorm in one launch:
// warp w of the CTA gathers row s's context (as embed_kernel does), holds
// X[s][c] for c = lane + 32 q in registers, writes X (FP32) and then runs
// exactly the arithmetic of ln_fwd_bf16_kernel<NPL> on those values.
template <int NPL>
__global__ void __launch_bounds__(32 * kRowsLN)
    embed_ln_bf16_kernel(const uint8_t* __restrict__ data, Split sp, const StepCtl* __restrict__ ctl,
                         const float* __restrict__ E, int K, int D, float* __restrict__ X, uint8_t* __restrict__ ctx,
                         const float* __restrict__ g, const float* __restrict__ be, float* __restrict__ xhat,
                         float* __restrict__ rstd, __nv_bfloat16* __restrict__ X0b, __nv_bfloat16* __restrict__ X0bT,
                         int b, int ldT, const int* __restrict__ rg, size_t gs) {
  pdl_wait();
  pdl_launch();
  constexpr int F = 32 * NPL;
  extern __shared__ __nv_bfloat16 tile_dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kRowsLN + warp;
  __nv_bfloat16* trow = tile_dyn + (size_t)warp * F;
  if (s < b) {
    if (rg) {  // grouped mode: the row's own model
      const size_t o = (size_t)rg[s] * gs;
      E += o;
      g += o;
      be += o;
    }
    const int i = ctl->i;
    // A stream past its end (inactive) keeps its last context, as in embed_kernel.
    if (data && i <= sp.len(s)) {
      const long long base = sp.off(s) + i - K;
      for (int k = lane; k < K; k += 32) ctx[(size_t)s * K + k] = data[base + k];
    }
    __syncwarp();
    float v[NPL];
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const int c = lane + 32 * q, k = c / D, dd = c - k * D;
      v[q] = E[(int)ctx[(size_t)s * K + k] * D + dd];
      X[(size_t)s * F + c] = v[q];
    }
    float sm = 0.f;
#pragma unroll
    for (int q = 0; q < NPL; ++q) sm += v[q];
    const float mean = warp_sum(sm) / (float)F;
    float qv = 0.f;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const float d = v[q] - mean;
      qv += d * d;
    }
    const float r = 1.0f / sqrtf(warp_sum(qv) / (float)F + kLnEps);
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const int c = lane + 32 * q;
      const float h = (v[q] - mean) * r;
      xhat[(size_t)s * F + c] = h;
      const __nv_bfloat16 o = __float2bfloat16_rn(h * g[c] + be[c]);
      X0b[(size_t)s * F + c] = o;
      trow[c] = o;
    }
    if (lane == 0) rstd[s] = r;
  } else {
    for (int c = lane; c < F; c += 32) trow[c] = __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  store_tile_T<kRowsLN>(tile_dyn, F, F, blockIdx.x * kRowsLN, X0bT, ldT);
}

cudaError_t launch_embed_ln_bf16(const uint8_t* data, Split sp, const StepCtl* ctl, const float* E, int b, int K,
                                 int D, float* X, uint8_t* ctx, const float* g, const float* be, float* xhat,
                                 float* rstd, __nv_bfloat16* X0b, __nv_bfloat16* X0bT, int ldT, cudaStream_t st,
                                 const int* rg, size_t gs) {
  const int F = K * D;
  const size_t smem = (size_t)kRowsLN * F * sizeof(__nv_bfloat16);
  const dim3 grid(div_up(b, kRowsLN)), block(32 * kRowsLN);
#define EDPC_ELN(NPL) \
  launch_k(embed_ln_bf16_kernel<NPL>, grid, block, smem, st, data, sp, ctl, E, K, D, X, ctx, g, be, xhat, rstd, X0b, \
           X0bT, b, ldT, rg, gs)
  switch (F) {
    case 128: return EDPC_ELN(4);
    case 256: return EDPC_ELN(8);
    case 512: return EDPC_ELN(16);
    case 1024: return EDPC_ELN(32);
    default: return cudaErrorInvalidValue;
  }
#undef EDPC_ELN
}

template <int NPL>
__global__ void __launch_bounds__(32 * kRowsLN)
    ln_bwd_bf16_kernel(const float* __restrict__ dX0, const float* __restrict__ xhat, const float* __restrict__ rstd,
                       const float* __restrict__ g, const float* __restrict__ dRes, float* __restrict__ dX,
                       __nv_bfloat16* __restrict__ dXb, __nv_bfloat16* __restrict__ dXbT, int b, int F, int ldT,
                       const int* __restrict__ rg, size_t gs) {
  pdl_wait();
  pdl_launch();
  extern __shared__ __nv_bfloat16 tile_dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsLN + warp;
  __nv_bfloat16* trow = tile_dyn + (size_t)warp * F;
  if (row < b) {
    if (rg) g += (size_t)rg[row] * gs;  // grouped mode: the row's own gamma
    const size_t o = (size_t)row * F;
    const float r = rstd[row];
    if (NPL > 0) {
      float d[NPL > 0 ? NPL : 1], xh[NPL > 0 ? NPL : 1], rs[NPL > 0 ? NPL : 1];
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        const int c = lane + 32 * q;
        d[q] = dX0[o + c] * g[c];
        xh[q] = xhat[o + c];
        rs[q] = dRes[o + c];
      }
      float s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        s1 += d[q];
        s2 += d[q] * xh[q];
      }
      const float m1 = warp_sum(s1) / (float)F;
      const float m2 = warp_sum(s2) / (float)F;
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        const int c = lane + 32 * q;
        const float v = rs[q] + r * (d[q] - m1 - xh[q] * m2);
        dX[o + c] = v;
        if (dXb) {
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          dXb[o + c] = h;
          trow[c] = h;
        }
      }
    } else {
      float s1 = 0.f, s2 = 0.f;
      for (int c = lane; c < F; c += 32) {
        const float dd = dX0[o + c] * g[c];
        s1 += dd;
        s2 += dd * xhat[o + c];
      }
      const float m1 = warp_sum(s1) / (float)F;
      const float m2 = warp_sum(s2) / (float)F;
      for (int c = lane; c < F; c += 32) {
        const float dd = dX0[o + c] * g[c];
        const float v = dRes[o + c] + r * (dd - m1 - xhat[o + c] * m2);
        dX[o + c] = v;
        if (dXb) {
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          dXb[o + c] = h;
          trow[c] = h;
        }
      }
    }
  } else if (dXbT) {
    for (int c = lane; c < F; c += 32) trow[c] = __float2bfloat16_rn(0.f);
  }
  if (dXbT) {
    __syncthreads();
    store_tile_T<kRowsLN>(tile_dyn, F, F, blockIdx.x * kRowsLN, dXbT, ldT);
  }
}

cudaError_t launch_ln_bwd_bf16(const float* dX0, const float* xhat, const float* rstd, const float* g,
                               const float* dRes, float* dX, __nv_bfloat16* dXb, __nv_bfloat16* dXbT, int b, int F,
                               int ldT, cudaStream_t st, const int* rg, size_t gs) {
  const size_t smem = dXbT ? (size_t)kRowsLN * F * sizeof(__nv_bfloat16) : 0;
  const dim3 grid(div_up(b, kRowsLN)), block(32 * kRowsLN);
#define EDPC_LNB(NPL)                                                                                      \
  launch_k(ln_bwd_bf16_kernel<NPL>, grid, block, smem, st, dX0, xhat, rstd, g, dRes, dX, dXb, dXbT, b, F, ldT, rg, \
           gs)
  switch (F) {
    case 128: return EDPC_LNB(4);
    case 256: return EDPC_LNB(8);
    case 512: return EDPC_LNB(16);
    case 1024: return EDPC_LNB(32);
    default: return EDPC_LNB(0);
  }
#undef EDPC_LNB
}

// ============================================================================================
// Batched column sums (bias and LN-affine gradients), fixed order: CTA = one
// tile of TW columns of one job and one chunk of rows; warp w sums the chunk's
// rows w, w+16, ...; warps are then added in order. TW = 32 (one column per
// lane, four interleaved row accumulators) below 2048 rows; from there, when
// every job allows 16-byte loads, TW = 128 (four columns per lane, eight
// interleaved row accumulators: rows r, r+16, ..., r+112 of each pass). With
// several chunks, the last CTA of a tile to arrive adds the chunk partials in
// chunk order (a fence before the arrival counter makes the partials visible
// to it).
// ============================================================================================
template <bool VEC>
__global__ void __launch_bounds__(512) colsum_multi_kernel(ColsumJobs jobs) {
  pdl_wait();
  pdl_launch();
  constexpr int TW = VEC ? 128 : 32;
  constexpr int CPL = VEC ? 4 : 1;  // columns per lane
  __shared__ float part[16][TW + 1];
  __shared__ int is_last;
  const int tile = blockIdx.x;
  int t = blockIdx.x, j = 0;
  while (j < jobs.n - 1 && t >= (jobs.job[j].cols + TW - 1) / TW) {
    t -= (jobs.job[j].cols + TW - 1) / TW;
    ++j;
  }
  const ColsumJob jb = jobs.job[j];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = t * TW + lane * CPL;
  const int nch = gridDim.y;
  const int r_lo = (nch > 1) ? blockIdx.y * jobs.chunk_rows : 0;
  const int r_hi = (nch > 1) ? min(jb.rows, r_lo + jobs.chunk_rows) : jb.rows;
  float a[8][CPL];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int q = 0; q < CPL; ++q) a[k][q] = 0.f;
  auto load = [&](int r, float (&v)[CPL]) {
    const size_t o = (size_t)r * jb.ld + c;
    if (VEC) {
      float4 x = *reinterpret_cast<const float4*>(jb.X + o);
      if (jb.Y) {
        const float4 y = *reinterpret_cast<const float4*>(jb.Y + o);
        x.x *= y.x;
        x.y *= y.y;
        x.z *= y.z;
        x.w *= y.w;
      }
      v[0] = x.x;
      if (CPL > 1) {
        v[CPL > 1 ? 1 : 0] = x.y;
        v[CPL > 2 ? 2 : 0] = x.z;
        v[CPL > 3 ? 3 : 0] = x.w;
      }
    } else {
      v[0] = jb.Y ? jb.X[o] * jb.Y[o] : jb.X[o];
    }
  };
  if (!VEC && c < jb.cols) {
    // rows w, w+16, ... with four interleaved accumulators
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int r = r_lo + w;
    if (jb.Y) {
      for (; r + 48 < r_hi; r += 64) {
        a0 += jb.X[(size_t)r * jb.ld + c] * jb.Y[(size_t)r * jb.ld + c];
        a1 += jb.X[(size_t)(r + 16) * jb.ld + c] * jb.Y[(size_t)(r + 16) * jb.ld + c];
        a2 += jb.X[(size_t)(r + 32) * jb.ld + c] * jb.Y[(size_t)(r + 32) * jb.ld + c];
        a3 += jb.X[(size_t)(r + 48) * jb.ld + c] * jb.Y[(size_t)(r + 48) * jb.ld + c];
      }
      for (; r < r_hi; r += 16) a0 += jb.X[(size_t)r * jb.ld + c] * jb.Y[(size_t)r * jb.ld + c];
    } else {
      for (; r + 48 < r_hi; r += 64) {
        a0 += jb.X[(size_t)r * jb.ld + c];
        a1 += jb.X[(size_t)(r + 16) * jb.ld + c];
        a2 += jb.X[(size_t)(r + 32) * jb.ld + c];
        a3 += jb.X[(size_t)(r + 48) * jb.ld + c];
      }
      for (; r < r_hi; r += 16) a0 += jb.X[(size_t)r * jb.ld + c];
    }
    a[0][0] = (a0 + a1) + (a2 + a3);
  }
  if (VEC && c < jb.cols) {
    int r = r_lo + w;
    for (; r + 112 < r_hi; r += 128) {
      float v[8][CPL];
#pragma unroll
      for (int k = 0; k < 8; ++k) load(r + 16 * k, v[k]);
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int q = 0; q < CPL; ++q) a[k][q] += v[k][q];
    }
    for (; r < r_hi; r += 16) {
      float v[CPL];
      load(r, v);
#pragma unroll
      for (int q = 0; q < CPL; ++q) a[0][q] += v[q];
    }
  }
#pragma unroll
  for (int q = 0; q < CPL; ++q)
    part[w][lane * CPL + q] =
        VEC ? ((a[0][q] + a[1][q]) + (a[2][q] + a[3][q])) + ((a[4][q] + a[5][q]) + (a[6][q] + a[7][q])) : a[0][q];
  __syncthreads();
  const int tc = threadIdx.x;  // column of the tile handled in the final sums
  const int cc = t * TW + tc;
  float sum = 0.f;
  if (tc < TW) {
    sum = part[0][tc];
#pragma unroll
    for (int i = 1; i < 16; ++i) sum += part[i][tc];
  }
  if (nch == 1) {
    if (tc < TW && cc < jb.cols) jb.out[cc] = sum;
    return;
  }
  if (tc < TW) {
    jobs.part[((size_t)tile * nch + blockIdx.y) * TW + tc] = sum;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&jobs.cnt[tile], 1u) == (unsigned)(nch - 1));
  __syncthreads();
  if (is_last && tc < TW) {
    __threadfence();
    const float* src = jobs.part + (size_t)tile * nch * TW + tc;
    float acc = 0.f;
    for (int k = 0; k < nch; ++k) acc += __ldcg(src + (size_t)k * TW);
    if (cc < jb.cols) jb.out[cc] = acc;
    if (tc == 0) jobs.cnt[tile] = 0u;
  }
}

bool colsum_vec(const ColsumJobs& jobs) {
  // 128-column tiles only from 2048 rows on: below that the 32-column grid's
  // parallelism matters more (the sums end the side stream before Adam)
  for (int j = 0; j < jobs.n; ++j) {
    const ColsumJob& b = jobs.job[j];
    if (b.rows < 2048) return false;
    if ((b.cols & 3) || (b.ld & 3) || (reinterpret_cast<uintptr_t>(b.X) & 15) ||
        (b.Y && (reinterpret_cast<uintptr_t>(b.Y) & 15)))
      return false;
  }
  return true;
}

int colsum_tiles(const ColsumJobs& jobs) {
  const int tw = colsum_vec(jobs) ? 128 : 32;
  int tiles = 0;
  for (int j = 0; j < jobs.n; ++j) tiles += (jobs.job[j].cols + tw - 1) / tw;
  return tiles;
}

int colsum_chunk_rows(int rows, int tiles) {
  // about 256 CTAs in all: the column sums run on a side stream beside the
  // step's critical path, and a wider grid would take SMs from it
  if (rows <= 512 || tiles <= 0) return 0;
  int nch = 256 / tiles;
  if (nch > kColsumMaxChunks) nch = kColsumMaxChunks;
  if (nch > rows / 256) nch = rows / 256;
  if (nch < 2) return 0;
  int cr = (rows + nch - 1) / nch;
  return (cr + 15) / 16 * 16;
}

cudaError_t launch_colsum_multi(const ColsumJobs& jobs, cudaStream_t st) {
  const int tiles = colsum_tiles(jobs);
  if (tiles == 0) return cudaSuccess;
  int rows = 0;
  for (int j = 0; j < jobs.n; ++j) rows = max(rows, jobs.job[j].rows);
  int nch = 1;
  if (jobs.chunk_rows > 0 && jobs.part && jobs.cnt) {
    for (int j = 0; j < jobs.n; ++j)
      if (jobs.job[j].rows != rows) return cudaErrorInvalidValue;  // one chunking for every job
    nch = (rows + jobs.chunk_rows - 1) / jobs.chunk_rows;
    if (nch > kColsumMaxChunks) return cudaErrorInvalidValue;
  }
  if (colsum_vec(jobs)) return launch_k(colsum_multi_kernel<true>, dim3(tiles, nch), dim3(512), 0, st, jobs);
  return launch_k(colsum_multi_kernel<false>, dim3(tiles, nch), dim3(512), 0, st, jobs);
}

// ============================================================================================
// Grouped column sums (bias and LN-affine gradients of independent per-file
// models): CTA = 32 columns of one job and one group, 16 warps; warp w sums
// the group's stream rows w, w + 16, ... for its lane's column, and the 16
// warp sums are added in warp order.
// ============================================================================================
__global__ void __launch_bounds__(512) colsum_groups_kernel(ColsumJobs jobs, const GroupInfo* __restrict__ gi,
                                                            size_t gs) {
  pdl_wait();
  pdl_launch();
  __shared__ float part[16][33];
  const ColsumJob j = jobs.job[blockIdx.z];
  const GroupInfo g = gi[blockIdx.y];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  float a = 0.f;
  if (c < j.cols) {
    const size_t ld = (size_t)j.ld;
    for (int r = g.r0 + w; r < g.r0 + g.s; r += 16)
      a += j.Y ? j.X[r * ld + c] * j.Y[r * ld + c] : j.X[r * ld + c];
  }
  part[w][lane] = a;
  __syncthreads();
  if (w == 0 && c < j.cols) {
    float t = part[0][lane];
#pragma unroll
    for (int q = 1; q < 16; ++q) t += part[q][lane];
    j.out[(size_t)blockIdx.y * gs + c] = t;
  }
}

cudaError_t launch_colsum_groups(const ColsumJobs& jobs, const GroupInfo* gi, int ngroups, size_t gs,
                                 cudaStream_t st) {
  if (jobs.n < 1 || jobs.n > kMaxColsumJobs || ngroups < 1 || ngroups > 65535 || !gi) return cudaErrorInvalidValue;
  int maxc = 0;
  for (int k = 0; k < jobs.n; ++k) maxc = max(maxc, jobs.job[k].cols);
  return launch_k(colsum_groups_kernel, dim3(div_up(maxc, 32), ngroups, jobs.n), dim3(512), 0, st, jobs, gi, gs);
}

// ============================================================================================
// Adam with the BF16 weight copy refreshed in the same pass; transposed copies
// of every weight matrix in one launch (32 x 32 tiles through shared memory).
// ============================================================================================
__global__ void adam_bf16_kernel(float* P, const float* Pin, const float* __restrict__ G, float* __restrict__ M,
                                 float* __restrict__ V, __nv_bfloat16* __restrict__ Pb, size_t n,
                                 const StepCtl* __restrict__ ctl) {
  pdl_wait();
  pdl_launch();
  const StepCtl c = *ctl;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float p = Pin[e], m = M[e], v = V[e];
    const float gr = G[e];
    adam1(p, m, v, gr, c.lr, c.bc1, c.bc2);
    P[e] = p;
    M[e] = m;
    V[e] = v;
    Pb[e] = __float2bfloat16_rn(p);
  }
}
cudaError_t launch_adam_bf16(float* P, const float* G, float* M, float* V, __nv_bfloat16* Pb, size_t n,
                             const StepCtl* ctl, cudaStream_t st, const float* Pin) {
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  return launch_k(adam_bf16_kernel, dim3(grid), dim3(256), 0, st, P, Pin ? Pin : P, G, M, V, Pb, n, ctl);
}

__global__ void transpose_tiles_kernel(const __nv_bfloat16* __restrict__ Pb, __nv_bfloat16* __restrict__ PbT,
                                       const TransposeTile* __restrict__ tiles, int ntiles) {
  pdl_wait();
  pdl_launch();
  __shared__ __nv_bfloat16 t[32][34];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = blockIdx.x; i < ntiles; i += gridDim.x) {  // several tiles per CTA when there are many
    const TransposeTile tl = tiles[i];
    if (i != (int)blockIdx.x) __syncthreads();  // the previous tile's reads of t are done
    for (int k = ty; k < 32; k += 8) {
      int r = tl.r0 + k, cc = tl.c0 + tx;
      t[k][tx] = (r < tl.rows && cc < tl.cols) ? Pb[tl.off + (size_t)r * tl.cols + cc] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
      int cc = tl.c0 + k, r = tl.r0 + tx;
      if (cc < tl.cols && r < tl.rows) PbT[tl.off + (size_t)cc * tl.rows + r] = t[tx][k];
    }
  }
}
cudaError_t launch_transpose_tiles(const __nv_bfloat16* Pb, __nv_bfloat16* PbT, const TransposeTile* tiles,
                                   int ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const int grid = ntiles < 152 * 16 ? ntiles : 152 * 16;
  return launch_k(transpose_tiles_kernel, dim3(grid), dim3(256), 0, st, Pb, PbT, tiles, ntiles);
}

// ============================================================================================
// FP32 -> BF16 operand copies (row-major and transposed), via a 32x32 tile.
// ============================================================================================
__global__ void to_bf16_kernel(const float* __restrict__ X, int rows, int cols, int ldx, __nv_bfloat16* Y, int ldy,
                               __nv_bfloat16* YT, int ldt) {
  pdl_wait();
  pdl_launch();
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, cc = c0 + tx;
    float v = (r < rows && cc < cols) ? X[(size_t)r * ldx + cc] : 0.f;
    tile[k][tx] = v;
    if (Y && r < rows && cc < cols) Y[(size_t)r * ldy + cc] = __float2bfloat16_rn(v);
  }
  if (!YT) return;
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int cc = c0 + k, r = r0 + tx;
    if (cc < cols && r < rows) YT[(size_t)cc * ldt + r] = __float2bfloat16_rn(tile[tx][k]);
  }
}

cudaError_t launch_to_bf16(const float* X, int rows, int cols, int ldx, __nv_bfloat16* Y, int ldy,
                           __nv_bfloat16* YT, int ldt, cudaStream_t st) {
  dim3 grid(div_up(cols, 32), div_up(rows, 32));
  return launch_k(to_bf16_kernel, dim3(grid), dim3(256), 0, st, X, rows, cols, ldx, Y, ldy, YT, ldt);
}

// ============================================================================================
// FP8 e4m3 operand quantization: amax pass (integer atomicMax on the float bits
// of |x|, order-independent), then the convert pass with s = 2^k.
// ============================================================================================
__device__ __forceinline__ int fp8_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  frexpf(amax, &e);  // amax = m 2^e, m in [0.5, 1)
  int k = 9 - e;     // amax 2^k in [256, 512)
  if (ldexpf(amax, k) > 448.f) k -= 1;
  return k < -120 ? -120 : (k > 120 ? 120 : k);
}

__global__ void fp8_amax_kernel(Fp8Jobs J) {
  pdl_wait();
  pdl_launch();
  const Fp8Job& jb = J.job[blockIdx.y];
  const long long n8 = (long long)jb.rows * (jb.cols / 8);  // 8 BF16 per 16-byte load
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / (jb.cols / 8), c = (i % (jb.cols / 8)) * 8;
    const uint4 v = *reinterpret_cast<const uint4*>(jb.src + r * jb.ld + c);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 f = __bfloat1622float2(h[q]);
      m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
    atomicMax(J.amax + jb.slot, __float_as_uint(m));
  }
}

__global__ void fp8_convert_kernel(Fp8Jobs J) {
  pdl_wait();
  pdl_launch();
  const Fp8Job& jb = J.job[blockIdx.y];
  const int k = fp8_exp(__uint_as_float(J.amax[jb.slot]));
  const float sc = ldexpf(1.f, k);
  if (blockIdx.x == 0 && threadIdx.x == 0) J.inv[jb.slot] = ldexpf(1.f, -k);
  const long long n8 = (long long)jb.rows * (jb.cols / 8);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n8; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / (jb.cols / 8), c = (i % (jb.cols / 8)) * 8;
    const uint4 v = *reinterpret_cast<const uint4*>(jb.src + r * jb.ld + c);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
    uint8_t o[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 f = __bfloat1622float2(h[q]);
      o[2 * q] = (uint8_t)__nv_cvt_float_to_fp8(f.x * sc, __NV_SATFINITE, __NV_E4M3);
      o[2 * q + 1] = (uint8_t)__nv_cvt_float_to_fp8(f.y * sc, __NV_SATFINITE, __NV_E4M3);
    }
    *reinterpret_cast<uint2*>(jb.dst + r * jb.ld8 + c) = *reinterpret_cast<const uint2*>(o);
  }
}

cudaError_t launch_fp8_quantize(const Fp8Jobs& J, cudaStream_t st) {
  if (J.n <= 0) return cudaSuccess;
  if (J.n > kMaxFp8Jobs) return cudaErrorInvalidValue;
  long long most = 0;
  for (int j = 0; j < J.n; ++j) {
    const Fp8Job& jb = J.job[j];
    // 16-byte loads and 8-byte stores: cols and both strides in whole vectors
    if (jb.cols % 8 || jb.ld % 8 || jb.ld8 % 8) return cudaErrorInvalidValue;
    most = std::max(most, (long long)jb.rows * (jb.cols / 8));
  }
  const int per_job = (int)std::min<long long>(std::max<long long>(1, (most + 255) / 256), 2 * 152);
  cudaError_t e = launch_k(fp8_amax_kernel, dim3(per_job, J.n), dim3(256), 0, st, J);
  if (e != cudaSuccess) return e;
  return launch_k(fp8_convert_kernel, dim3(per_job, J.n), dim3(256), 0, st, J);
}

__global__ void zero_u32_kernel(unsigned* p, int n) {
  pdl_wait();
  pdl_launch();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0u;
}

cudaError_t launch_zero_u32(unsigned* p, int n, cudaStream_t st) {
  return launch_k(zero_u32_kernel, dim3(1), dim3(256), 0, st, p, n);
}

}  // namespace edpc
