// Persistent tcgen05 GEMM (gemm_tcp_kernel.cuh): BF16 and FP8, every
// epilogue mode.
#include "gemm_tcp_kernel.cuh"

namespace edpc {
namespace tcp {

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  });
  return n;
}

}  // namespace tcp

cudaError_t launch_gemm_tcp(const TcGemm& g, cudaStream_t st) {
  return g.fp8 ? tcp::launch_tcp_t<true>(g, st) : tcp::launch_tcp_t<false>(g, st);
}

}  // namespace edpc
