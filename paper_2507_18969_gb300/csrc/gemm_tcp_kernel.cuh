// Persistent BF16 / FP8 GEMM on the 5th-generation tensor cores (sm_103a).
//
// One CTA per SM walks output tiles of C = A B^T with 192 threads:
//   warp 0 (one lane)  TMA producer: 128-byte-wide A (128 rows) and B (BN rows)
//                      K blocks into a STAGES-deep ring that runs across tiles;
//   warp 1 (one lane)  MMA issuer: tcgen05.mma (M=128, N=BN) into one of two
//                      TMEM accumulators, alternating per tile; commits each
//                      stage to its "empty" barrier and each finished
//                      accumulator to its "full" barrier; warp 1 also
//                      allocates and frees the 2 x BN TMEM columns;
//   warps 2-5          epilogue: warp w drains TMEM lanes 32(w%4)..+31 (tile
//                      rows) with tcgen05.ld, runs the fused epilogue and
//                      releases the accumulator (one arrival per warp), so
//                      tile i's epilogue overlaps tile i+1's main loop.
// Work unit u = blockIdx.x, blockIdx.x + gridDim.x, ... (N tile fastest, then
// the M tile, then the split-K index).
// Each tile's MMAs run over K in the same order as in the one-tile kernel and
// the epilogue is the same code, so every variant gives identical results for
// the same N tile. Every wait is bounded; on expiry the kernel records
// kErrTcTimeout, lets its TMA copies land, frees its TMEM and returns.
#pragma once

#include <cudaTypedefs.h>

#include <climits>
#include <mutex>

#include "gemm_tc.cuh"
#include "gemm_tc_dev.cuh"
#include "launch.cuh"

namespace edpc {
namespace tcp {

using namespace tc;

// Ring depth: about 160-192 KB of stages (one CTA per SM).
template <int BN>
constexpr int pstages_for() { return BN <= 64 ? 8 : (BN <= 128 ? 6 : 4); }

constexpr size_t kStageT = 32 * 128 * sizeof(__nv_bfloat16);  // transposed-store staging

template <int BN>
constexpr size_t psmem_bytes() {
  return 1024 /*alignment slack*/ + (size_t)pstages_for<BN>() * (BM * BKB + BN * BKB) + kStageT + kStageOut + 256;
}
static_assert(psmem_bytes<256>() <= 232448 && psmem_bytes<128>() <= 232448, "shared memory per CTA");

template <int BN, int MODE, int KB, bool F8>
__global__ void __launch_bounds__(192, 1)
    gemm_tcp_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                    const __grid_constant__ CUtensorMap tmc, const __grid_constant__ CUtensorMap tmcb, const TcEpi e,
                    int nsplit) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int STAGES = pstages_for<BN>();
  constexpr uint32_t A_BYTES = BM * BKB, B_BYTES = BN * BKB;
  constexpr int BK = bk_elems<F8>();
  constexpr int SECTIONS = (MODE == TC_BRANCH) ? KB : 1;
  constexpr int SW = BN / SECTIONS;   // rows of B per section (TC_BRANCH)
  constexpr uint32_t ACC = (uint32_t)tmem_cols<BN>();  // columns of one accumulator
  static_assert(SW % 32 == 0, "sections are whole 32-column TMEM chunks");
  static_assert(2 * ACC <= 512, "two accumulators must fit TMEM");
  uint8_t* sA = smem;
  uint8_t* sB = sA + STAGES * A_BYTES;
  __nv_bfloat16* sT = reinterpret_cast<__nv_bfloat16*>(sB + STAGES * B_BYTES);
  uint8_t* sO = reinterpret_cast<uint8_t*>(sT) + kStageT;  // TMA-store staging, kStageOutWarp per warp
  uint64_t* full = reinterpret_cast<uint64_t*>(sO + kStageOut);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;  // [2] accumulator written
  uint64_t* tempty = tfull + 2;      // [2] accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* sk_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cid = blockIdx.x, ncl = gridDim.x;
  const int nunits = e.ntn * e.ntm * nsplit;
  const int nk_all = (e.K + BK - 1) / BK;
  struct Tile {
    int m0, n0, z, lo, nk, ci;
  };
  auto decode = [&](int u) {
    Tile q;
    const int tn = u % e.ntn, rest = u / e.ntn;
    const int tm = rest % e.ntm;
    q.z = rest / e.ntm;
    q.m0 = tm * BM;
    q.n0 = (MODE == TC_BRANCH) ? tn * SW : tn * BN;
    q.lo = (int)(((long long)nk_all * q.z) / nsplit);
    q.nk = (int)(((long long)nk_all * (q.z + 1)) / nsplit) - q.lo;
    q.ci = tm * e.ntn + tn;
    return q;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * ACC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_launch();

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      uint32_t it = 0;
      bool go = true;
      for (int u = cid; u < nunits && go; u += ncl) {
        const Tile q = decode(u);
        for (int kb = 0; kb < q.nk; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t ph = (it / STAGES) & 1u;
          if (it >= (uint32_t)STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            go = false;
            break;
          }
          mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
          const int kc = (q.lo + kb) * BK;
#pragma unroll
          for (int i = 0; i < SECTIONS; ++i) {
            const int brow = (MODE == TC_BRANCH ? i * e.H : 0) + q.n0;
            tma_load_2d(sB + s * B_BYTES + i * SW * BKB, &tb, kc, brow, &full[s]);
          }
          tma_load_2d(sA + s * A_BYTES, &ta, kc, q.m0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = F8 ? idesc_e4m3(BN) : idesc_bf16(BN);
      uint32_t it = 0;
      int tcount = 0;
      bool go = true;
      for (int u = cid; u < nunits && go; u += ncl, ++tcount) {
        const Tile q = decode(u);
        const int a = tcount & 1;
        // accumulator a was last used by tile tcount - 2: wait until it is drained
        if (tcount >= 2 && !mbar_wait(&tempty[a], (uint32_t)((tcount >> 1) - 1) & 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)a * ACC;
        for (int kb = 0; kb < q.nk; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            go = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int k = 0; k < BKB / 32; ++k) {  // one MMA per 32 bytes of K
            const uint64_t ad = sdesc(sA + s * A_BYTES + k * 32);
            const uint64_t bd = sdesc(sB + s * B_BYTES + k * 32);
            if (F8)
              mma_e4m3(dt, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            else
              mma_bf16(dt, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        if (go) mma_commit(&tfull[a]);
      }
    }
  } else {
    // epilogue warps 2-5; tcgen05.ld lets warp w reach TMEM lanes 32(w%4)..+31
    const int lg = warp & 3;
    const int r = lg * 32 + lane, et = threadIdx.x - 64;
    int tcount = 0;
    for (int u = cid; u < nunits; u += ncl, ++tcount) {
      const Tile q = decode(u);
      const int a = tcount & 1;
      if (!epi_and(mbar_wait(&tfull[a], (uint32_t)(tcount >> 1) & 1u, abort_flag))) break;
      tc_fence_after();
      if (q.m0 < e.M) {
        const EpiOut o{&tmc, &tmcb, sO + lg * kStageOutWarp, q.m0 + lg * 32, lane};
        tc_epilogue<BN, MODE, KB, F8>(e, tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)a * ACC, q.m0, q.n0, q.z,
                                      nsplit, q.ci, sT, sk_flag, r, et, o);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
    }
    tma_st_drain(lane);
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) {
    if (e.err) atomicOr(e.err, kErrTcTimeout);
    // Let any TMA copies still in flight land before the CTA exits.
    for (int s = 0; s < STAGES; ++s) {
      for (uint32_t it = 0; it < (1u << 20); ++it)
        if (mbar_try_wait(&full[s], 0) || mbar_try_wait(&full[s], 1)) break;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC));
  }
}

int sm_count();

template <int BN, int MODE, int KB, bool F8>
cudaError_t launch_p(const TcGemm& g, cudaStream_t st) {
  auto k = gemm_tcp_kernel<BN, MODE, KB, F8>;
  constexpr int SW = (MODE == TC_BRANCH) ? BN / KB : BN;
  // the tensor map's box must be one section of B
  if (g.box_b != SW) return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int max_ctas = 0;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem_bytes<BN>());
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    max_ctas = sm_count();
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int ntn = (MODE == TC_BRANCH) ? (g.H + SW - 1) / SW : (g.N + BN - 1) / BN;
  const int ntm = (g.M + BM - 1) / BM;
  const int S = g.splitk > 1 ? g.splitk : 1;
  TcEpi e{g.M, g.N, g.K, g.H, g.k, g.C, g.ldc, g.Cb, g.ldcb, g.CbT, g.ldct, g.bias, g.R, g.ldr, g.Aux, g.ldaux, g.err,
          g.inv_a, g.inv_b, 0, g.ws, g.cnt, ntn, ntm, g.has_tmc ? 1 : 0, g.has_tmcb ? 1 : 0,
          nullptr, nullptr, 0, INT_MAX};
  const long long units = (long long)ntn * ntm * S;
  if (units <= 0 || units > (1ll << 30)) return cudaErrorInvalidValue;
  const int nct = (int)(units < max_ctas ? units : max_ctas);
  return launch_k(k, dim3(nct), dim3(192), psmem_bytes<BN>(), st, g.ta, g.tb, g.tmc, g.tmcb, e, S);
}

// Dispatch on (mode, k, tile).
template <bool F8>
cudaError_t launch_tcp_t(const TcGemm& g, cudaStream_t st) {
  if (g.mode == TC_BRANCH) {
    if (g.bn != g.k * g.box_b) return cudaErrorInvalidValue;
    switch (g.k * 1000 + g.box_b) {
      case 1032: return launch_p<32, TC_BRANCH, 1, F8>(g, st);
      case 1064: return launch_p<64, TC_BRANCH, 1, F8>(g, st);
      case 1128: return launch_p<128, TC_BRANCH, 1, F8>(g, st);
      case 2032: return launch_p<64, TC_BRANCH, 2, F8>(g, st);
      case 2064: return launch_p<128, TC_BRANCH, 2, F8>(g, st);
      case 2128: return launch_p<256, TC_BRANCH, 2, F8>(g, st);
      case 3032: return launch_p<96, TC_BRANCH, 3, F8>(g, st);
      case 3064: return launch_p<192, TC_BRANCH, 3, F8>(g, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (g.box_b != g.bn) return cudaErrorInvalidValue;
  if (g.mode == TC_BRANCH_BWD) {
    switch (g.k * 1000 + g.bn) {
      case 1032: return launch_p<32, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2032: return launch_p<32, TC_BRANCH_BWD, 2, F8>(g, st);
      case 3032: return launch_p<32, TC_BRANCH_BWD, 3, F8>(g, st);
      case 1064: return launch_p<64, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2064: return launch_p<64, TC_BRANCH_BWD, 2, F8>(g, st);
      case 3064: return launch_p<64, TC_BRANCH_BWD, 3, F8>(g, st);
      case 1128: return launch_p<128, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2128: return launch_p<128, TC_BRANCH_BWD, 2, F8>(g, st);
      case 3128: return launch_p<128, TC_BRANCH_BWD, 3, F8>(g, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.bn) {
    case 32: return launch_p<32, TC_PLAIN, 1, F8>(g, st);
    case 64: return launch_p<64, TC_PLAIN, 1, F8>(g, st);
    case 128: return launch_p<128, TC_PLAIN, 1, F8>(g, st);
    case 256: return launch_p<256, TC_PLAIN, 1, F8>(g, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tcp
}  // namespace edpc
