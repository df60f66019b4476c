// Self-test of the bounded-wait error path. Every device-side wait of the
// library (the GEMMs' mbarrier waits, the FDM forward's bulk-copy waits) has
// a limit after which the kernel records an error bit and returns, so that a
// lost arrival ends in a status, not a hung GPU. This kernel makes such a wait
// run out on purpose: one thread waits on a shared-memory mbarrier that
// nothing arrives on, gives up after a clock budget (and, as a second bound,
// an iteration count), sets the error word and returns. The host maps the
// word to EDPC_ETIMEOUT and then checks that the context still runs work.
#include <cstdint>

#include "common.cuh"

namespace edpc {

namespace {

constexpr int kErrSelftestTimeout = 8;
constexpr uint32_t kSelftestIters = 1u << 20;

__global__ void wait_timeout_kernel(int* err, long long budget_cycles) {
  __shared__ uint64_t bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    uint32_t done = 0;
    for (uint32_t it = 0; it < kSelftestIters && !done; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(b), "r"(0u)
          : "memory");
      if (clock64() - t0 > budget_cycles) break;
    }
    if (!done) atomicOr(err, kErrSelftestTimeout);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
  }
  __syncthreads();
}

}  // namespace

}  // namespace edpc

extern "C" int edpc_selftest_wait_timeout(void* cuda_stream) {
  using namespace edpc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, khz = 0;
  EDPC_CUDA(cudaGetDevice(&dev));
  EDPC_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const long long budget = (long long)(khz > 0 ? khz : 2000000) * 50;  // about 50 ms of SM clock
  int* err = nullptr;
  EDPC_CUDA(cudaMalloc(&err, sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32, 0, st>>>(err, budget);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // the context still runs work after the expired wait
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) return fail(EDPC_ECUDA, std::string("self-test: ") + cudaGetErrorString(e));
  if (h & kErrSelftestTimeout) return fail(EDPC_ETIMEOUT, "self-test: the bounded wait expired as designed");
  return fail(EDPC_ECUDA, "self-test: the wait on an mbarrier with no arrivals completed");
}
