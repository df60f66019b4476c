// Persistent tcgen05 GEMM (gemm_tcp_kernel.cuh) in clusters of 2 or 4 CTAs
// that share each B tile through TMA multicast; BF16.
#include "gemm_tcp_kernel.cuh"

namespace edpc {

cudaError_t launch_gemm_tcp_mc(const TcGemm& g, cudaStream_t st) {
  switch (g.mcast) {
    case 2: return tcp::launch_tcp_t<false, 2>(g, st);
    case 4: return tcp::launch_tcp_t<false, 4>(g, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace edpc
