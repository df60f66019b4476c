// Plain FP32 SIMT GEMM with a fused bias / residual epilogue.
//
// This is the "plain FP32" arithmetic of the model's Linear layers
// (Eqs. 10, 13, 14, 16, the head, and their adjoints). Each output element
// sums its K products in increasing k order, so results are deterministic.
// Tile 64 x 64 x 16, 256 threads, 4 x 4 outputs per thread (rows ty + 16i,
// columns tx + 16j), operands staged through shared memory in [k][m] / [k][n]
// order with coalesced global loads for either operand layout.
#include "kernels.cuh"
#include "launch.cuh"

namespace edpc {

template <bool AK, bool BK, int EPI>
__global__ void __launch_bounds__(256) gemm_f32_kernel(GemmF32 g) {
  constexpr int BM = 64, BN = 64, BKT = 16;
  pdl_wait();
  pdl_launch();
  __shared__ float As[BKT][BM + 4];
  __shared__ float Bs[BKT][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += BKT) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      int m, k;
      if (AK) {
        m = e >> 4;
        k = e & 15;
      } else {
        k = e >> 6;
        m = e & 63;
      }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.f;
      if (gm < g.M && gk < g.K) v = AK ? g.A[(size_t)gm * g.lda + gk] : g.A[(size_t)gk * g.lda + gm];
      As[k][m] = v;
      int n;
      if (BK) {
        n = e >> 4;
        k = e & 15;
      } else {
        k = e >> 6;
        n = e & 63;
      }
      const int gn = n0 + n, gk2 = k0 + k;
      float w = 0.f;
      if (gn < g.N && gk2 < g.K) w = BK ? g.B[(size_t)gn * g.ldb + gk2] : g.B[(size_t)gk2 * g.ldb + gn];
      Bs[k][n] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKT; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      if (EPI >= EPI_BIAS) v += g.bias[n];
      if (EPI == EPI_BIAS_RESID) v += g.R[(size_t)m * g.ldr + n];
      g.C[(size_t)m * g.ldc + n] = v;
    }
  }
}

template <bool AK, bool BK>
static cudaError_t dispatch_epi(const GemmF32& g, dim3 grid, cudaStream_t st) {
  switch (g.epi) {
    case EPI_STORE: return launch_k(gemm_f32_kernel<AK, BK, EPI_STORE>, grid, dim3(256), 0, st, g);
    case EPI_BIAS: return launch_k(gemm_f32_kernel<AK, BK, EPI_BIAS>, grid, dim3(256), 0, st, g);
    default: return launch_k(gemm_f32_kernel<AK, BK, EPI_BIAS_RESID>, grid, dim3(256), 0, st, g);
  }
}

cudaError_t launch_gemm_f32(const GemmF32& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid(div_up(g.N, 64), div_up(g.M, 64));
  if (g.a_kcont && g.b_kcont) return dispatch_epi<true, true>(g, grid, st);
  if (g.a_kcont && !g.b_kcont) return dispatch_epi<true, false>(g, grid, st);
  if (!g.a_kcont && g.b_kcont) return dispatch_epi<false, true>(g, grid, st);
  return dispatch_epi<false, false>(g, grid, st);
}

}  // namespace edpc
