// Mutual information of Sec. 3.1.1 (Information Flow Refinement): Kraskov's
// k-nearest-neighbour estimate of I(Z; Y) between an MBRB's skip input and
// its fused output.
//
// CTA i (one per sample, 256 threads) computes the FP32 max-norm distances
// dz(i, j) and dy(i, j) to every sample j (a warp per j, lanes over the
// coordinates, a butterfly max), takes eps(i) = the k-th smallest joint
// distance max(dz, dy) over j != i by an exact radix select on the bits of
// the non-negative floats (31 passes of CTA-wide integer counts), and counts
// c_z(i) = #{j != i: dz(i, j) < eps(i)} and c_y(i) likewise. |a - b| and max
// are exact in FP32, so the counts are fixed by the FP32 samples. The host
// then forms psi(k) + psi(N) - mean(psi(c_z + 1) + psi(c_y + 1)) in FP64.
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "launch.cuh"

namespace edpc {

namespace {

constexpr int kMiThreads = 256;

__device__ __forceinline__ int block_sum(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int s = 0;
#pragma unroll
  for (int q = 0; q < kMiThreads / 32; ++q) s += red[q];
  return s;
}

__global__ void __launch_bounds__(kMiThreads) ksg_kernel(const float* __restrict__ Z, const float* __restrict__ Y,
                                                         int N, int dz, int dy, int k, unsigned* __restrict__ cz,
                                                         unsigned* __restrict__ cy) {
  extern __shared__ float sm[];
  float* zi = sm;             // dz
  float* yi = zi + dz;        // dy
  float* sdz = yi + dy;       // N
  float* sdy = sdz + N;       // N
  __shared__ int red[kMiThreads / 32];
  const int i = blockIdx.x, t = threadIdx.x;
  const int w = t >> 5, lane = t & 31;
  for (int q = t; q < dz; q += kMiThreads) zi[q] = Z[(size_t)i * dz + q];
  for (int q = t; q < dy; q += kMiThreads) yi[q] = Y[(size_t)i * dy + q];
  __syncthreads();
  for (int j = w; j < N; j += kMiThreads / 32) {
    float a = 0.f, b = 0.f;
    for (int q = lane; q < dz; q += 32) a = fmaxf(a, fabsf(Z[(size_t)j * dz + q] - zi[q]));
    for (int q = lane; q < dy; q += 32) b = fmaxf(b, fabsf(Y[(size_t)j * dy + q] - yi[q]));
    for (int o = 16; o > 0; o >>= 1) {
      a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane == 0) {
      sdz[j] = a;
      sdy[j] = b;
    }
  }
  __syncthreads();
  // k-th smallest joint distance over j != i (non-negative floats order like their bits)
  unsigned prefix = 0, mask = 0;
  int kk = k;
  for (int bit = 30; bit >= 0; --bit) {
    int c = 0;
    for (int j = t; j < N; j += kMiThreads) {
      if (j == i) continue;
      const unsigned u = __float_as_uint(fmaxf(sdz[j], sdy[j]));
      c += ((u & mask) == prefix && ((u >> bit) & 1u) == 0u) ? 1 : 0;
    }
    c = block_sum(c, red);
    if (c < kk) {
      kk -= c;
      prefix |= 1u << bit;
    }
    mask |= 1u << bit;
  }
  const float eps = __uint_as_float(prefix);
  int nz = 0, ny = 0;
  for (int j = t; j < N; j += kMiThreads) {
    if (j == i) continue;
    nz += sdz[j] < eps ? 1 : 0;
    ny += sdy[j] < eps ? 1 : 0;
  }
  nz = block_sum(nz, red);
  ny = block_sum(ny, red);
  if (t == 0) {
    cz[i] = (unsigned)nz;
    cy[i] = (unsigned)ny;
  }
}

// psi(x) for x >= 1: recurrence up to x >= 10, then the asymptotic series
// ln x - 1/(2x) - sum_n B_2n / (2n x^2n) (Abramowitz & Stegun 6.3.6, 6.3.18).
double digamma_ge1(double x) {
  double r = 0;
  while (x < 10.0) {
    r -= 1.0 / x;
    x += 1.0;
  }
  const double x2 = 1.0 / (x * x);
  const double series =
      x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132 - x2 * 691.0 / 32760)))));
  return r + std::log(x) - 0.5 / x - series;
}

}  // namespace

}  // namespace edpc

using namespace edpc;

extern "C" int edpc_ksg_mi(const float* Z, const float* Y, uint32_t N, uint32_t dz, uint32_t dy, uint32_t k,
                           uint32_t* cz, uint32_t* cy, double* mi, void* cuda_stream) {
  if (!Z || !Y || !cz || !cy || !mi) return fail(EDPC_EINVAL, "NULL argument");
  if (N < 2 || N > 8192) return fail(EDPC_EINVAL, "N must be in [2, 8192]");
  if (k < 1 || k >= N || k > 64) return fail(EDPC_EINVAL, "k must be in [1, min(64, N - 1)]");
  if (dz < 1 || dy < 1 || dz + dy > 8192) return fail(EDPC_EINVAL, "dz, dy >= 1 and dz + dy <= 8192");
  const size_t smem = sizeof(float) * ((size_t)dz + dy + 2 * (size_t)N);
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(ksg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * (8192 + 2 * 8192)));
  });
  if (attr != cudaSuccess) return fail(EDPC_ECUDA, std::string("ksg attribute: ") + cudaGetErrorString(attr));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NoPdl scope;
  cudaError_t e = launch_k(ksg_kernel, dim3(N), dim3(kMiThreads), smem, st, Z, Y, (int)N, (int)dz, (int)dy, (int)k,
                           (unsigned*)cz, (unsigned*)cy);
  std::vector<uint32_t> hz(N), hy(N);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hz.data(), cz, 4 * (size_t)N, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hy.data(), cy, 4 * (size_t)N, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(EDPC_ECUDA, std::string("ksg: ") + cudaGetErrorString(e));
  double s = 0;
  for (uint32_t q = 0; q < N; ++q) s += digamma_ge1(hz[q] + 1.0) + digamma_ge1(hy[q] + 1.0);
  *mi = digamma_ge1((double)k) + digamma_ge1((double)N) - s / N;
  return EDPC_OK;
}
