// BF16 / FP8 GEMM on the 5th-generation tensor cores (sm_103a).
//
// One CTA computes a 128 x BN tile of C = A B^T:
//   warp 0 (one lane)  issues TMA loads of 128-byte-wide A (128 rows) and B
//                      (BN rows) tiles (64 BF16 or 128 FP8 elements of K,
//                      128-byte swizzle) into a STAGES-deep ring;
//   warp 1 (one lane)  issues tcgen05.mma (M=128, N=BN; kind::f16 with K=16
//                      for BF16, kind::f8f6f4 with K=32 for FP8 e4m3; FP32
//                      accumulation) into a TMEM accumulator and commits each
//                      stage back to its "empty" barrier;
//   warp 2             allocates / frees the TMEM columns;
//   warps 0-3          drain TMEM with tcgen05.ld (warp w owns lanes 32w..32w+31,
//                      i.e. tile rows) and run the fused epilogue.
// The MMA order over K is fixed, so results are deterministic.
// Barrier set-up, TMEM allocation and tensor-map prefetch run before the
// programmatic-dependent-launch wait, overlapping the previous kernel's tail.
// Every mbarrier wait is bounded; on expiry the kernel records kErrTcTimeout,
// stops waiting, frees its TMEM and returns.
#include <cudaTypedefs.h>

#include <climits>

#include <mutex>

#include "gemm_tc.cuh"
#include "gemm_tc_dev.cuh"
#include "kernels.cuh"
#include "launch.cuh"

namespace edpc {

namespace {

using namespace tc;

// Pipeline depth: enough stages to hold the whole K panel in flight for the
// small-N tiles (8 x 20-24 KB, one CTA per SM); 3 stages for N tiles of 96-128
// and 2 for 192-256 (about 97 KB), so that two CTAs share an SM and one's
// epilogue overlaps the other's main loop.
template <int BN>
constexpr int stages_for() { return BN <= 64 ? 8 : (BN <= 128 ? 3 : 2); }

template <int BN>
constexpr size_t smem_bytes() {
  return 1024 /*alignment slack*/ + (size_t)stages_for<BN>() * (BM * BKB + BN * BKB) + 256;
}

// KB: branch count k (TC_BRANCH, TC_BRANCH_BWD; 1 otherwise). In TC_BRANCH mode
// the N tile holds k sections of SW = BN / k hidden units each.
// GR: grouped mode (the tile list, or each group's K range; see TcGemm). The
// other instantiations carry none of its code.
template <int BN, int MODE, int KB, bool F8, bool GR>
__global__ void __launch_bounds__(128, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                   const __grid_constant__ CUtensorMap tmc, const __grid_constant__ CUtensorMap tmcb, const TcEpi e) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int STAGES = stages_for<BN>();
  constexpr uint32_t A_BYTES = BM * BKB, B_BYTES = BN * BKB;
  constexpr int BK = bk_elems<F8>();
  constexpr int SECTIONS = (MODE == TC_BRANCH) ? KB : 1;
  constexpr int SW = BN / SECTIONS;  // rows of B per section (TC_BRANCH)
  static_assert(SW % 32 == 0, "sections are whole 32-column TMEM chunks");
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);  // tmem_slot + 2: split-K flag

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Rows [m0, mend) of the tile are stored; grouped mode reads the tile (and
  // its group) from the tile list, or the group's K range (weight gradients).
  int m0 = blockIdx.y * BM, mend = e.M, grp = 0;
  if (GR && e.mt) {
    const int4 t = e.mt[blockIdx.y];
    m0 = t.x;
    mend = t.y;
    grp = t.z;
  }
  // N offset of the tile: in TC_BRANCH mode a tile covers hidden units
  // [SW*bx, SW*bx + SW) of every branch.
  const int n0 = (MODE == TC_BRANCH) ? blockIdx.x * SW : blockIdx.x * BN;
  // K blocks of this CTA: all of them, split z of gridDim.z (split-K), or the
  // group's own range (grouped weight gradients; k0 is a multiple of 64)
  int kel0 = 0, kb_lo = 0, nk = 0;
  if (GR && e.gk) {
    grp = blockIdx.z;
    const int4 t = e.gk[grp];
    kel0 = t.x;
    nk = t.y;
  } else {
    const int nk_all = (e.K + BK - 1) / BK;
    kb_lo = (int)(((long long)nk_all * blockIdx.z) / gridDim.z);
    nk = (int)(((long long)nk_all * (blockIdx.z + 1)) / gridDim.z) - kb_lo;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)tmem_cols<BN>()));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // When B (weights, or activations of the forward pass) was written at least
  // two kernels earlier (b_early), its first tiles are fetched before the
  // programmatic-dependent-launch wait; A comes from the previous kernel.
  auto load_b = [&](int kb, int s) {
    const int kc = kel0 + (kb_lo + kb) * BK;
#pragma unroll
    for (int i = 0; i < SECTIONS; ++i) {
      const int brow = (MODE == TC_BRANCH ? i * e.H : 0) + n0;
      if (GR && e.mt)
        tma_load_3d(sB + s * B_BYTES + i * (SW * BKB), &tb, kc, brow, grp, &full[s]);
      else
        tma_load_2d(sB + s * B_BYTES + i * (SW * BKB), &tb, kc, brow, &full[s]);
    }
  };
  const int npre = e.b_early ? (nk < STAGES ? nk : STAGES) : 0;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < npre; ++kb) {
      mbar_expect_tx(&full[kb], A_BYTES + B_BYTES);
      load_b(kb, kb);
    }
  }
  pdl_wait();
  pdl_launch();

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
      if (kb >= npre) {
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        load_b(kb, s);
      }
      tma_load_2d(sA + s * A_BYTES, &ta, kel0 + (kb_lo + kb) * BK, m0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = F8 ? idesc_e4m3(BN) : idesc_bf16(BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, abort_flag)) break;
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < BKB / 32; ++k) {  // one MMA per 32 bytes of K
        const uint64_t ad = sdesc(sA + s * A_BYTES + k * 32);
        const uint64_t bd = sdesc(sB + s * B_BYTES + k * 32);
        if (F8)
          mma_e4m3(tmem, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
        else
          mma_bf16(tmem, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  // Epilogue: thread (warp w, lane l) owns tile row 32w + l. The TMEM loads are
  // warp-collective, so the wait result is made CTA-uniform first.
  const bool ok = __syncthreads_and(mbar_wait(done, 0, abort_flag) ? 1 : 0) != 0;
  tc_fence_after();
  // The pipeline's A stages are idle now: reuse them to stage the transposed
  // stores (8 KB) and the TMA stores (6 KB per warp).
  static_assert(STAGES * A_BYTES >= 8192 + kStageOut, "A stages hold the epilogue staging");
  if (ok) {
    const EpiOut o{&tmc, &tmcb, sA + 8192 + warp * kStageOutWarp, m0 + warp * 32, lane};
    if constexpr (GR) {
      // grouped mode: the tile's row bound, its group's bias or gradient output
      TcEpi eg = e;
      eg.M = mend;
      eg.rlim = mend;
      if (e.mt && e.bias) eg.bias = e.bias + (long long)grp * e.gs;
      if (e.gk) eg.C = e.C + (long long)grp * e.gs;
      tc_epilogue<BN, MODE, KB, F8>(eg, tmem + ((uint32_t)(warp * 32) << 16), m0, n0, 0, 1, 0,
                                    reinterpret_cast<__nv_bfloat16*>(sA),
                                    reinterpret_cast<volatile int*>(tmem_slot + 2), threadIdx.x, threadIdx.x, o);
    } else {
      tc_epilogue<BN, MODE, KB, F8>(e, tmem + ((uint32_t)(warp * 32) << 16), m0, n0, blockIdx.z, gridDim.z,
                                    blockIdx.y * gridDim.x + blockIdx.x, reinterpret_cast<__nv_bfloat16*>(sA),
                                    reinterpret_cast<volatile int*>(tmem_slot + 2), threadIdx.x, threadIdx.x, o);
    }
    tma_st_drain(lane);
  }
  if (!ok && threadIdx.x == 0 && e.err) atomicOr(e.err, kErrTcTimeout);
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) {
    // Let any TMA copies still in flight land before the CTA exits.
    for (int s = 0; s < STAGES; ++s) {
      for (uint32_t it = 0; it < (1u << 20); ++it)
        if (mbar_try_wait(&full[s], 0) || mbar_try_wait(&full[s], 1)) break;
    }
  }
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)tmem_cols<BN>()));
  }
}

template <int BN, int MODE, int KB, bool F8, bool GR>
cudaError_t launch_bn_mode_g(const TcGemm& g, cudaStream_t st) {
  auto k = gemm_tc_kernel<BN, MODE, KB, F8, GR>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<BN>());
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  });
  if (attr_err != cudaSuccess) return attr_err;
  TcEpi e{g.M, g.N, g.K, g.H, g.k, g.C, g.ldc, g.Cb, g.ldcb, g.CbT, g.ldct, g.bias, g.R, g.ldr, g.Aux, g.ldaux, g.err,
          g.inv_a, g.inv_b, g.b_early ? 1 : 0, g.ws, g.cnt, 0, 0, g.has_tmc ? 1 : 0, g.has_tmcb ? 1 : 0,
          g.mt, g.gk, (long long)g.gs, INT_MAX};
  constexpr int SW = (MODE == TC_BRANCH) ? BN / KB : BN;
  const int ntile = (MODE == TC_BRANCH) ? (g.H + SW - 1) / SW : (g.N + BN - 1) / BN;
  dim3 grid(ntile, g.mt ? g.nmt : (g.M + BM - 1) / BM, g.gk ? g.ngk : (g.splitk > 1 ? g.splitk : 1));
  return launch_k(k, grid, dim3(128), smem_bytes<BN>(), st, g.ta, g.tb, g.tmc, g.tmcb, e);
}

// Grouped launches (BF16 only) use the GR instantiation.
template <int BN, int MODE, int KB = 1, bool F8 = false>
cudaError_t launch_bn_mode(const TcGemm& g, cudaStream_t st) {
  if (g.mt || g.gk) return F8 ? cudaErrorInvalidValue : launch_bn_mode_g<BN, MODE, KB, false, true>(g, st);
  return launch_bn_mode_g<BN, MODE, KB, F8, false>(g, st);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

int make_tmap_bf16(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
  auto enc = get_encode();
  if (!enc) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled is not available");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15))
    return fail(EDPC_EINVAL, "tensor map base or row stride is not 16-byte aligned");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return EDPC_OK;
}

int make_tmap_bf16_groups(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                          uint64_t groups, uint64_t gstride, uint32_t box_rows) {
  auto enc = get_encode();
  if (!enc) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled is not available");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15) || ((gstride * 2) & 15) || groups < 1)
    return fail(EDPC_EINVAL, "grouped tensor map base or strides are not 16-byte aligned");
  cuuint64_t dims[3] = {cols, rows, groups};
  cuuint64_t strides[2] = {ld * 2, gstride * 2};
  cuuint32_t box[3] = {64, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled (3-D) failed: " + std::to_string((int)r));
  return EDPC_OK;
}

int make_tmap_u8(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
  auto enc = get_encode();
  if (!enc) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled is not available");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld & 15))
    return fail(EDPC_EINVAL, "FP8 tensor map base or row stride is not 16-byte aligned");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld};
  cuuint32_t box[2] = {128, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled (u8) failed: " + std::to_string((int)r));
  return EDPC_OK;
}

int tc_build_out_maps(TcGemm* g) {
  g->has_tmc = g->has_tmcb = false;
  auto enc = get_encode();
  if (!enc) return fail(EDPC_ECUDA, "cuTensorMapEncodeTiled is not available");
  const int wc = (g->mode == TC_PLAIN) ? g->N : g->k * g->H;                          // columns of C
  const int wcb = (g->mode == TC_PLAIN) ? g->N : (g->mode == TC_BRANCH ? g->H : g->k * g->H);  // of Cb
  auto build = [&](CUtensorMap* tm, void* base, int cols, int ld, int esize, CUtensorMapDataType dt,
                   CUtensorMapSwizzle sw) -> bool {
    if (!base || cols < 32 || g->M < 32) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (((size_t)ld * esize) & 15)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)g->M};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  // A TMA store must start on a 16-byte boundary: the branch modes start
  // branch i's chunks at column i * H, so H must be a multiple of 8 (BF16).
  const bool cols_ok = g->mode == TC_PLAIN || g->H % 8 == 0;
  // split-K partials and their sums, and grouped weight gradients (one output
  // base per group), keep direct stores
  if (g->splitk <= 1 && cols_ok && !g->gk) {
    g->has_tmc = build(&g->tmc, g->C, wc, g->ldc, 4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_128B);
    g->has_tmcb = build(&g->tmcb, g->Cb, wcb, g->ldcb, 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, CU_TENSOR_MAP_SWIZZLE_64B);
  }
  return EDPC_OK;
}

namespace {
template <bool F8>
cudaError_t launch_gemm_tc_t(const TcGemm& g, cudaStream_t st);
}

int tc_splitk(int M, int N, int K, int bn) {
  const int tiles = tc_tiles(M, N, bn);
  const int nk = (K + 63) / 64;
  int s = 64 / (tiles > 0 ? tiles : 1);
  if (s > nk / 8) s = nk / 8;
  if (s > 32) s = 32;
  return s < 2 ? 1 : s;
}

cudaError_t launch_gemm_tc(const TcGemm& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (g.fp8) {
    if (!g.inv_a || !g.inv_b) return cudaErrorInvalidValue;
    return launch_gemm_tc_t<true>(g, st);
  }
  return launch_gemm_tc_t<false>(g, st);
}

namespace {
template <bool F8>
cudaError_t launch_gemm_tc_t(const TcGemm& g, cudaStream_t st) {
  // The kernel's B tile (and the expected TMA byte count) must match the box
  // the tensor map was encoded with; refuse any mismatch before launching.
  if (g.k < 1 || g.k > 3) return cudaErrorInvalidValue;
  if (g.splitk > 1) {
    // split-K: plain FP32 output only, at least one K block per split, scratch present
    const int nk = (g.K + bk_elems<F8>() - 1) / bk_elems<F8>();
    if (g.mode != TC_PLAIN || g.bias || g.R || g.Cb || g.CbT || !g.ws || !g.cnt || g.splitk > nk ||
        g.splitk > 65535)
      return cudaErrorInvalidValue;
  }
  if (g.mt || g.gk) {
    // grouped mode: one-tile kernel, no split-K, a non-empty tile or group list
    if (g.persistent || g.splitk > 1 || (g.mt && g.gk) || (g.mt && (g.nmt < 1 || g.nmt > 65535)) ||
        (g.gk && (g.ngk < 1 || g.ngk > 65535)) || (g.gk && (g.has_tmc || g.has_tmcb)))
      return cudaErrorInvalidValue;
  }
  if (g.persistent) return launch_gemm_tcp(g, st);  // checks the tile against the box itself
  if (g.mode == TC_BRANCH) {
    // box_b = section width; bn = k sections
    if (g.bn != g.k * g.box_b) return cudaErrorInvalidValue;
    switch (g.k * 1000 + g.box_b) {
      case 1032: return launch_bn_mode<32, TC_BRANCH, 1, F8>(g, st);
      case 1064: return launch_bn_mode<64, TC_BRANCH, 1, F8>(g, st);
      case 1128: return launch_bn_mode<128, TC_BRANCH, 1, F8>(g, st);
      case 2032: return launch_bn_mode<64, TC_BRANCH, 2, F8>(g, st);
      case 2064: return launch_bn_mode<128, TC_BRANCH, 2, F8>(g, st);
      case 2128: return launch_bn_mode<256, TC_BRANCH, 2, F8>(g, st);
      case 3032: return launch_bn_mode<96, TC_BRANCH, 3, F8>(g, st);
      case 3064: return launch_bn_mode<192, TC_BRANCH, 3, F8>(g, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (g.box_b != g.bn) return cudaErrorInvalidValue;
  if (g.mode == TC_BRANCH_BWD) {
    switch (g.k * 1000 + g.bn) {
      case 1032: return launch_bn_mode<32, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2032: return launch_bn_mode<32, TC_BRANCH_BWD, 2, F8>(g, st);
      case 3032: return launch_bn_mode<32, TC_BRANCH_BWD, 3, F8>(g, st);
      case 1064: return launch_bn_mode<64, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2064: return launch_bn_mode<64, TC_BRANCH_BWD, 2, F8>(g, st);
      case 3064: return launch_bn_mode<64, TC_BRANCH_BWD, 3, F8>(g, st);
      case 1128: return launch_bn_mode<128, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2128: return launch_bn_mode<128, TC_BRANCH_BWD, 2, F8>(g, st);
      case 3128: return launch_bn_mode<128, TC_BRANCH_BWD, 3, F8>(g, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.bn) {
    case 32: return launch_bn_mode<32, TC_PLAIN, 1, F8>(g, st);
    case 64: return launch_bn_mode<64, TC_PLAIN, 1, F8>(g, st);
    case 128: return launch_bn_mode<128, TC_PLAIN, 1, F8>(g, st);
    case 256: return launch_bn_mode<256, TC_PLAIN, 1, F8>(g, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

}  // namespace edpc
