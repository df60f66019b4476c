// Row-wise, element-wise and coder kernels of the EDPC step.
//
// Every reduction runs in a fixed order (warp xor-butterflies, then shared
// memory in warp order), and nothing is accumulated with floating-point
// atomics. So the encoder and the decoder, which launch the same kernels on
// the same values, compute bit-identical probabilities and CDFs.
#include "kernels.cuh"

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
  init_values_kernel<<<grid, 256, 0, st>>>(dst, n, seed, tid, bound, start, fill);
  return cudaGetLastError();
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
                             uint8_t* __restrict__ ctx) {
  const int s = blockIdx.x;
  const int F = K * D;
  if (data) {
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
                         int D, float* X, uint8_t* ctx, cudaStream_t st) {
  embed_kernel<<<b, 128, 0, st>>>(data, sp, ctl, E, K, D, X, ctx);
  return cudaGetLastError();
}

// ============================================================================================
// LayerNorm forward (Eq. 9), one warp per row, two-pass statistics.
// ============================================================================================
__global__ void ln_fwd_kernel(const float* __restrict__ X, const float* __restrict__ g,
                              const float* __restrict__ be, float* __restrict__ xhat,
                              float* __restrict__ rstd, float* __restrict__ X0, int b, int F) {
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
  ln_fwd_kernel<<<div_up(b, 8), 256, 0, st>>>(X, g, be, xhat, rstd, X0, b, F);
  return cudaGetLastError();
}

// ============================================================================================
// MBRB branch fusion (Eqs. 11-12): G = GELU(X_1 * ... * X_k), exact erf GELU.
// ============================================================================================
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void branch_gelu_kernel(const float* __restrict__ A, int b, int H, int k, float* __restrict__ G) {
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
  branch_gelu_kernel<<<grid, 256, 0, st>>>(A, b, H, k, G);
  return cudaGetLastError();
}

__global__ void branch_gelu_bwd_kernel(const float* __restrict__ dG, const float* __restrict__ A, int b, int H,
                                       int k, float* __restrict__ dA) {
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
  branch_gelu_bwd_kernel<<<grid, 256, 0, st>>>(dG, A, b, H, k, dA);
  return cudaGetLastError();
}

// ============================================================================================
// Column sums over rows (bias and LN-affine gradients), fixed order:
// warp w sums rows w, w+8, ... for 32 columns; then warps are added in order.
// ============================================================================================
__global__ void colsum_kernel(const float* __restrict__ X, const float* __restrict__ Y, int rows, int cols,
                              int ld, float* __restrict__ out) {
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
  colsum_kernel<<<div_up(cols, 32), 256, 0, st>>>(X, Y, rows, cols, ld, out);
  return cudaGetLastError();
}

// ============================================================================================
// LayerNorm backward: dX = dRes + rstd * (dxh - mean(dxh) - xhat * mean(dxh * xhat)),
// dxh = dX0 * g; one warp per row.
// ============================================================================================
__global__ void ln_bwd_kernel(const float* __restrict__ dX0, const float* __restrict__ xhat,
                              const float* __restrict__ rstd, const float* __restrict__ g,
                              const float* __restrict__ dRes, float* __restrict__ dX, int b, int F) {
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
  ln_bwd_kernel<<<div_up(b, 8), 256, 0, st>>>(dX0, xhat, rstd, g, dRes, dX, b, F);
  return cudaGetLastError();
}

// ============================================================================================
// FDM forward (Eq. 15): y_s[j] = sum_i x'_s[i] U_s[i][j]. One CTA per stream;
// threads own 4 consecutive columns and a row group; row groups are added in order.
// ============================================================================================
__global__ void __launch_bounds__(256) fdm_fwd_kernel(const float* __restrict__ Xp, const float* __restrict__ U,
                                                      float* __restrict__ Y, int Fp) {
  extern __shared__ float sm[];
  float* xs = sm;              // Fp
  float* part = sm + Fp;       // groups x Fp
  const int s = blockIdx.x;
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
  }
}

cudaError_t launch_fdm_fwd(const float* Xp, const float* U, float* Y, int b, int Fp, cudaStream_t st) {
  const int cols4 = Fp / 4;
  const int threads = cols4 >= 256 ? cols4 : (256 / cols4) * cols4;
  const int groups = threads / cols4;
  size_t smem = (size_t)(Fp + groups * Fp) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fdm_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fdm_fwd_kernel<<<b, threads, smem, st>>>(Xp, U, Y, Fp);
  return cudaGetLastError();
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

template <int NCH>  // float4 chunks per lane per row: Fp = 128 * NCH
__global__ void __launch_bounds__(256) fdm_bwd_kernel(FdmBwdArgs a) {
  const int s = blockIdx.y;
  const int Fp = a.Fp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const StepCtl c = *a.ctl;
  bool act = a.active ? (a.active[s] != 0) : ((long long)c.i < a.sp.len(s));
  const int row0 = blockIdx.x * kFdmRowsPerCta;
  if (!act) {
    // dy is zero for an inactive stream, so dx' = 0 and its FDM state is left as is.
    for (int r = warp; r < kFdmRowsPerCta; r += 8)
      if (lane == 0 && row0 + r < Fp) a.dXp[(size_t)s * Fp + row0 + r] = 0.f;
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
    if (lane == 0) a.dXp[(size_t)s * Fp + i] = dot;
  }
}

// Generic fallback for F' not a multiple of 128: one element per lane step.
__global__ void __launch_bounds__(256) fdm_bwd_generic_kernel(FdmBwdArgs a) {
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
      if (lane == 0) a.dXp[(size_t)s * Fp + i] = 0.f;
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
    if (lane == 0) a.dXp[(size_t)s * Fp + i] = dot;
  }
}

cudaError_t launch_fdm_bwd(const FdmBwdArgs& a, cudaStream_t st) {
  dim3 grid(div_up(a.Fp, kFdmRowsPerCta), a.b);
  switch (a.Fp) {
    case 128: fdm_bwd_kernel<1><<<grid, 256, 0, st>>>(a); break;
    case 256: fdm_bwd_kernel<2><<<grid, 256, 0, st>>>(a); break;
    case 384: fdm_bwd_kernel<3><<<grid, 256, 0, st>>>(a); break;
    case 512: fdm_bwd_kernel<4><<<grid, 256, 0, st>>>(a); break;
    case 1024: fdm_bwd_kernel<8><<<grid, 256, 0, st>>>(a); break;
    default: fdm_bwd_generic_kernel<<<grid, 256, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

// ============================================================================================
// Embedding backward: scatter-add of dh0 into E's rows, owner-computes per symbol.
// CTA c scans all b*K positions in order (8 warps over contiguous slices,
// ballot per 32 positions); partial sums are added in warp order.
// ============================================================================================
__global__ void embed_bwd_kernel(const uint8_t* __restrict__ ctx, const float* __restrict__ dX, int b, int K,
                                 int D, float* __restrict__ dE) {
  __shared__ float part[8][64];
  const int c = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = b * K;
  const int per = (P + 7) / 8;
  const int p0 = w * per, p1 = min(P, p0 + per);
  float acc0 = 0.f, acc1 = 0.f;  // d = lane, d = lane + 32
  for (int base = p0; base < p1; base += 32) {
    int p = base + lane;
    bool hit = p < p1 && ctx[p] == c;
    unsigned m = __ballot_sync(0xffffffffu, hit);
    while (m) {
      int l = __ffs(m) - 1;
      m &= m - 1;
      int q = base + l;
      int s = q / K, k = q - s * K;
      const float* src = dX + (size_t)s * K * D + (size_t)k * D;
      if (lane < D) acc0 += src[lane];
      if (lane + 32 < D) acc1 += src[lane + 32];
    }
  }
  part[w][lane] = acc0;
  part[w][lane + 32] = acc1;
  __syncthreads();
  if (w == 0) {
    for (int d = lane; d < D; d += 32) {
      float t = part[0][d];
      for (int i = 1; i < 8; ++i) t += part[i][d];
      dE[(size_t)c * D + d] = t;
    }
  }
}

cudaError_t launch_embed_bwd(const uint8_t* ctx, const float* dX, int b, int K, int D, float* dE,
                             cudaStream_t st) {
  if (D > 64) return cudaErrorInvalidValue;
  embed_bwd_kernel<<<256, 256, 0, st>>>(ctx, dX, b, K, D, dE);
  return cudaGetLastError();
}

// ============================================================================================
// Adam on the shared parameters (Sec. 4.1: lr 1e-3; beta, eps as documented).
// ============================================================================================
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, size_t n, const StepCtl* __restrict__ ctl) {
  const StepCtl c = *ctl;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float p = P[e], m = M[e], v = V[e];
    adam1(p, m, v, G[e], c.lr, c.bc1, c.bc2);
    P[e] = p;
    M[e] = m;
    V[e] = v;
  }
}

cudaError_t launch_adam(float* P, const float* G, float* M, float* V, size_t n, const StepCtl* ctl,
                        cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  adam_kernel<<<grid, 256, 0, st>>>(P, G, M, V, n, ctl);
  return cudaGetLastError();
}

// ============================================================================================
// Step control: advance to the next time index and derive its scalars.
// ============================================================================================
__global__ void step_advance_kernel(StepCtl* ctl, Split sp, int K, int ring_slots, int b) {
  StepCtl c = *ctl;
  c.i += 1;
  c.t += 1;
  long long i = c.i;
  int bact = (i < sp.q) ? b : (i == sp.q ? sp.rem : 0);
  c.bact = bact;
  c.inv_bact = bact > 0 ? 1.0f / (float)bact : 0.f;
  c.bc1 = 1.0f - powf(kB1, (float)c.t);
  c.bc2 = 1.0f - powf(kB2, (float)c.t);
  c.slot = (int)((i - K) % ring_slots);
  *ctl = c;
}

cudaError_t launch_step_advance(StepCtl* ctl, Split sp, int K, int ring_slots, int b, cudaStream_t st) {
  step_advance_kernel<<<1, 1, 0, st>>>(ctl, sp, K, ring_slots, b);
  return cudaGetLastError();
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
  prefix_encode_kernel<<<div_up(b, 128), 128, 0, st>>>(es, data, sp, K, b, out, out_off, out_cap);
  return cudaGetLastError();
}

// One thread per stream codes `nsteps` consecutive ring slots. Reads of a slot
// are coalesced across the streams of a warp.
__global__ void range_encode_kernel(EncState* es, const uint32_t* __restrict__ ring, int ring_slots, int slot0,
                                    int nsteps, int b, uint8_t* out, const unsigned long long* out_off,
                                    const uint32_t* out_cap) {
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
  range_encode_kernel<<<div_up(b, 128), 128, 0, st>>>(es, ring, ring_slots, slot0, nsteps, b, out, out_off,
                                                       out_cap);
  return cudaGetLastError();
}

__global__ void encode_flush_kernel(EncState* es, int b, uint8_t* out, const unsigned long long* out_off,
                                    const uint32_t* out_cap, uint32_t* out_len) {
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
  encode_flush_kernel<<<div_up(b, 128), 128, 0, st>>>(es, b, out, out_off, out_cap, out_len);
  return cudaGetLastError();
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
  dec_init_kernel<<<div_up(b, 128), 128, 0, st>>>(ds, bits, off, len, b);
  return cudaGetLastError();
}

__global__ void prefix_decode_kernel(DecState* ds, const uint8_t* bits, const unsigned long long* off,
                                     const uint32_t* len, Split sp, int K, int b, uint8_t* data) {
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
  prefix_decode_kernel<<<div_up(b, 128), 128, 0, st>>>(ds, bits, off, len, sp, K, b, data);
  return cudaGetLastError();
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

__global__ void head_kernel(HeadArgs a) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= a.b) return;
  const StepCtl c = *a.ctl;
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
      x = a.data[a.sp.off(s) + c.i];
      uint32_t cx = __shfl_sync(0xffffffffu, cdf.cum[x & 7], x >> 3);
      uint32_t fx = __shfl_sync(0xffffffffu, cdf.f[x & 7], x >> 3);
      // (all lanes must take the shuffles with the same source index: x is warp-uniform)
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
  const float inv = (a.mode == 2) ? c.inv_bact : c.inv_bact;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int j = lane * 8 + q;
    dz[q] = active ? (p[q] - (j == x ? 1.0f : 0.0f)) * inv : 0.f;
    if (po) po[q] = p[q];
  }
}

cudaError_t launch_head(const HeadArgs& a, cudaStream_t st) {
  head_kernel<<<div_up(a.b, 8), 256, 0, st>>>(a);
  return cudaGetLastError();
}

__global__ void cdf_quantize_kernel(const float* __restrict__ P, int rows, uint32_t* freq, uint32_t* cum) {
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
  cdf_quantize_kernel<<<div_up(rows, 8), 256, 0, st>>>(p, rows, freq, cum);
  return cudaGetLastError();
}

// ============================================================================================
// FP32 -> BF16 operand copies (row-major and transposed), via a 32x32 tile.
// ============================================================================================
__global__ void to_bf16_kernel(const float* __restrict__ X, int rows, int cols, int ldx, __nv_bfloat16* Y, int ldy,
                               __nv_bfloat16* YT, int ldt) {
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
  to_bf16_kernel<<<grid, 256, 0, st>>>(X, rows, cols, ldx, Y, ldy, YT, ldt);
  return cudaGetLastError();
}

}  // namespace edpc
