// Range encoding without any device allocation.
//
// edpc_range_encode obtains its per-call scratch (one coder state, output
// offset and capacity per stream) from cudaMalloc and releases it with
// cudaFree. Some callers cannot allow that: services that reserve their whole
// device-memory budget at start-up and refuse later allocations, and
// latency-sensitive loops that cannot absorb the device-wide synchronisation
// cudaFree may perform. For them, edpc_range_encode_noalloc keeps the scratch
// in a fixed array that is part of the library image itself: it exists on
// every GPU that loads the library, from load until process exit.
#include <mutex>

#include "kernels.cuh"

namespace edpc {
namespace {

constexpr uint32_t kNoAllocMaxStreams = EDPC_NOALLOC_MAX_STREAMS;

// Layout of the scratch: coder states, then output offsets, capacities and
// one overflow flag.
constexpr size_t kEsBytes = sizeof(EncState) * kNoAllocMaxStreams;
constexpr size_t kOffBytes = sizeof(unsigned long long) * kNoAllocMaxStreams;
constexpr size_t kCapBytes = sizeof(uint32_t) * kNoAllocMaxStreams;
constexpr size_t kScratchBytes = kEsBytes + kOffBytes + kCapBytes + 256;

static __device__ __align__(256) unsigned char g_coder_scratch[kScratchBytes];

// Device address of g_coder_scratch per device. In host code the symbol is
// only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current. The address is looked up
// once per device and kept for the life of the process: it stays valid as
// long as the device's primary context does. A cudaDeviceReset destroys that
// context (and the module image with the array), so a process that resets a
// device must not call this entry point on it again.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  EDPC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(EDPC_EINVAL, "device ordinal out of range for the static scratch");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_coder_scratch);
    if (e != cudaSuccess || !p)
      return fail(EDPC_ECUDA, std::string("cudaGetSymbolAddress(g_coder_scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return EDPC_OK;
}

// Per-call set-up: every stream's output window and capacity; the overflow
// flag starts at zero. (The coder states are initialised by the prefix kernel.)
__global__ void noalloc_setup_kernel(unsigned long long* off, uint32_t* cap, uint32_t* flag, uint32_t streams,
                                     uint32_t c) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *flag = 0;
  if (s < streams) {
    off[s] = (unsigned long long)s * c;
    cap[s] = c;
  }
}

// A stream that ran out of room reports 0xFFFFFFFF from the flush kernel:
// clamp it to the capacity and raise the flag.
__global__ void noalloc_overflow_kernel(uint32_t* out_len, uint32_t* flag, uint32_t streams, uint32_t c) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < streams && out_len[s] == 0xFFFFFFFFu) {
    out_len[s] = c;
    atomicOr(flag, 1u);
  }
}

}  // namespace
}  // namespace edpc

using namespace edpc;

extern "C" int edpc_range_encode_noalloc(const uint32_t* sym, uint32_t nsym, uint32_t streams, uint8_t* out,
                                         uint32_t cap, uint32_t* out_len, void* stream) {
  if (!sym || !out || !out_len || streams == 0) return fail(EDPC_EINVAL, "NULL argument or no streams");
  if (streams > kNoAllocMaxStreams)
    return fail(EDPC_EINVAL, "edpc_range_encode_noalloc: streams exceeds EDPC_NOALLOC_MAX_STREAMS (" +
                                 std::to_string(kNoAllocMaxStreams) + ")");
  unsigned char* base = nullptr;
  EDPC_TRY(scratch_for_current_device(&base));
  EncState* es = reinterpret_cast<EncState*>(base);
  unsigned long long* off = reinterpret_cast<unsigned long long*>(base + kEsBytes);
  uint32_t* caps = reinterpret_cast<uint32_t*>(base + kEsBytes + kOffBytes);
  uint32_t* flag = reinterpret_cast<uint32_t*>(base + kEsBytes + kOffBytes + kCapBytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = div_up(streams, 128);
  noalloc_setup_kernel<<<grid, 128, 0, st>>>(off, caps, flag, streams, cap);
  EDPC_CUDA(cudaGetLastError());
  Split none{0, 0, 0};
  EDPC_CUDA(launch_prefix_encode(es, nullptr, none, 0, (int)streams, out, off, caps, st));
  EDPC_CUDA(launch_range_encode(es, sym, (int)nsym, 0, (int)nsym, (int)streams, out, off, caps, st));
  EDPC_CUDA(launch_encode_flush(es, (int)streams, out, off, caps, out_len, st));
  noalloc_overflow_kernel<<<grid, 128, 0, st>>>(out_len, flag, streams, cap);
  EDPC_CUDA(cudaGetLastError());
  uint32_t over = 0;
  EDPC_CUDA(cudaMemcpyAsync(&over, flag, sizeof(over), cudaMemcpyDeviceToHost, st));
  EDPC_CUDA(cudaStreamSynchronize(st));
  if (over) return fail(EDPC_EINVAL, "a stream needs more than cap bytes");
  return EDPC_OK;
}
