// Persistent tcgen05 GEMM (gemm_tcp_kernel.cuh): launches without clusters,
// BF16 and FP8, every epilogue mode; the multicast variants are built in
// gemm_tcp_mc.cu.
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
  if (g.mcast > 1) return g.fp8 ? cudaErrorInvalidValue : launch_gemm_tcp_mc(g, st);
  return g.fp8 ? tcp::launch_tcp_t<true, 1>(g, st) : tcp::launch_tcp_t<false, 1>(g, st);
}

}  // namespace edpc
