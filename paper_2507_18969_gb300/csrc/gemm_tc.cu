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

#include <mutex>

#include "gemm_tc.cuh"
#include "kernels.cuh"
#include "launch.cuh"

namespace edpc {

namespace {

constexpr int BM = 128;
constexpr int BKB = 128;  // bytes of K per stage row (one 128-byte swizzle span)
template <bool F8>
constexpr int bk_elems() { return F8 ? 128 : 64; }
// Pipeline depth: enough stages to hold the whole K panel in flight for the
// small-N tiles (8 x 20-24 KB), 4 for wider tiles.
template <int BN>
constexpr int stages_for() { return BN <= 64 ? 8 : 4; }
constexpr uint32_t kSpinLimit = 1u << 26;

struct TcEpi {
  int M, N, K, H, k;
  float* C;
  int ldc;
  __nv_bfloat16* Cb;
  int ldcb;
  __nv_bfloat16* CbT;
  int ldct;
  const float* bias;
  const float* R;
  int ldr;
  const float* Aux;
  int ldaux;
  int* err;
  const float* inv_a;  // FP8: 1 / scale of A and of B (powers of two)
  const float* inv_b;
  int b_early;         // B may be fetched before the dependent-launch wait
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and raises the CTA's abort flag) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 128-byte swizzle: rows of 128 bytes, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1, layout 2.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  uint64_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (a & 0x3FFFFull) >> 4;
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
// kind::f8f6f4 with A = B = E4M3 (type code 0), D = F32, K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_e4m3(int bn) {
  return (1u << 4) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_e4m3(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Loads 32 consecutive FP32 values of one row (vectorised when in range and aligned).
__device__ __forceinline__ void load_row32(const float* src, int n0, int N, float (&v)[32]) {
  if (n0 + 32 <= N && ((reinterpret_cast<uintptr_t>(src + n0) & 15) == 0)) {
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      float4 q = *reinterpret_cast<const float4*>(src + n0 + j);
      v[j] = q.x;
      v[j + 1] = q.y;
      v[j + 2] = q.z;
      v[j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = (n0 + j < N) ? src[n0 + j] : 0.f;
  }
}

// Stores 32 consecutive values of one row as FP32 and/or BF16 (vectorised when
// the whole chunk is in range and aligned).
__device__ __forceinline__ void store_row32(const float (&v)[32], bool rok, int n0, int N, float* crow,
                                            __nv_bfloat16* cbrow) {
  if (!rok) return;
  const bool full = n0 + 32 <= N;
  if (crow) {
    float* p = crow + n0;
    if (full && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
#pragma unroll
      for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (n0 + j < N) p[j] = v[j];
    }
  }
  if (cbrow) {
    __nv_bfloat16* p = cbrow + n0;
    if (full && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
#pragma unroll
      for (int j = 0; j < 32; j += 8) {
        __align__(16) __nv_bfloat162 h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[j + 2 * q], v[j + 2 * q + 1]);
        *reinterpret_cast<uint4*>(p + j) = *reinterpret_cast<const uint4*>(h);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (n0 + j < N) p[j] = __float2bfloat16_rn(v[j]);
    }
  }
}

// Transposed BF16 store of a 128-row x 32-column chunk: every thread puts its
// row into shared memory (column-major), then the CTA writes each column's 128
// rows as 16-byte runs to CT[(n0 + c) * ldct + m0 + r]. Columns at or beyond N
// and 8-row runs at or beyond ldct are skipped. CTA-collective.
__device__ __forceinline__ void store_T32(const float (&v)[32], __nv_bfloat16* sT, int m0, int n0, int N,
                                          __nv_bfloat16* CT, int ldct) {
  const int r = threadIdx.x;  // tile row
#pragma unroll
  for (int c = 0; c < 32; ++c) sT[c * 128 + r] = __float2bfloat16_rn(v[c]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * 16; idx += 128) {
    const int c = idx >> 4, seg = idx & 15;
    const int row0 = m0 + seg * 8;
    if (n0 + c < N && row0 + 8 <= ldct)
      *reinterpret_cast<uint4*>(CT + (size_t)(n0 + c) * ldct + row0) =
          *reinterpret_cast<const uint4*>(sT + c * 128 + seg * 8);
  }
  __syncthreads();
}

template <int BN>
constexpr int tmem_cols() {
  return BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
}

template <int BN>
constexpr size_t smem_bytes() {
  return 1024 /*alignment slack*/ + (size_t)stages_for<BN>() * (BM * BKB + BN * BKB) + 256;
}

template <int BN, int MODE, int KB, bool F8>
__global__ void __launch_bounds__(128, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const TcEpi e) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int STAGES = stages_for<BN>();
  constexpr uint32_t A_BYTES = BM * BKB, B_BYTES = BN * BKB;
  constexpr int BK = bk_elems<F8>();
  constexpr int SECTIONS = (MODE == TC_BRANCH) ? BN / 32 : 1;
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM;
  // N offset of the tile: in TC_BRANCH mode a tile covers hidden units
  // [32*bx, 32*bx + 32) of every branch.
  const int n0 = (MODE == TC_BRANCH) ? blockIdx.x * 32 : blockIdx.x * BN;
  const int nk = (e.K + BK - 1) / BK;

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
    if (MODE == TC_BRANCH) {
#pragma unroll
      for (int i = 0; i < SECTIONS; ++i)
        tma_load_2d(sB + s * B_BYTES + i * (32 * BKB), &tb, kb * BK, i * e.H + n0, &full[s]);
    } else {
      tma_load_2d(sB + s * B_BYTES, &tb, kb * BK, n0, &full[s]);
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
      tma_load_2d(sA + s * A_BYTES, &ta, kb * BK, m0, &full[s]);
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
  const int row = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  // The pipeline's A stages are idle now: reuse them to stage transposed stores.
  __nv_bfloat16* sT = reinterpret_cast<__nv_bfloat16*>(sA);
  const bool rok = row < e.M;
  // FP8: undo the operands' power-of-two scales (exact)
  const float sc = F8 ? e.inv_a[0] * e.inv_b[0] : 1.f;
  if (ok) {
    if (MODE == TC_PLAIN) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(trow + (uint32_t)c0, v);
        if (F8) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] *= sc;
        }
        const int nb = n0 + c0;
        if (e.bias) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += (nb + j < e.N) ? e.bias[nb + j] : 0.f;
        }
        if (e.R && rok) {
          float r[32];
          load_row32(e.R + (size_t)row * e.ldr, nb, e.N, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += r[j];
        }
        store_row32(v, rok, nb, e.N, e.C ? e.C + (size_t)row * e.ldc : nullptr,
                    e.Cb ? e.Cb + (size_t)row * e.ldcb : nullptr);
        if (e.CbT) store_T32(v, sT, m0, nb, e.N, e.CbT, e.ldct);
      }
    } else if (MODE == TC_BRANCH) {
      // X_i for the tile's 32 hidden units h = n0 + j, then G = GELU(prod X_i).
      float g[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) g[j] = 1.f;
#pragma unroll 1
      for (int i = 0; i < SECTIONS; ++i) {
        float v[32];
        tmem_ld32(trow + (uint32_t)(i * 32), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (F8) v[j] *= sc;
          const int h = n0 + j;
          if (h < e.H) v[j] += e.bias[i * e.H + h];
          g[j] *= v[j];
        }
        // X_i -> C[row][i*H + h] (FP32, kept for the adjoint)
        store_row32(v, rok, n0, e.H, e.C + (size_t)row * e.ldc + i * e.H, nullptr);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) g[j] = gelu_f(g[j]);
      store_row32(g, rok, n0, e.H, nullptr, e.Cb + (size_t)row * e.ldcb);
      store_T32(g, sT, m0, n0, e.H, e.CbT, e.ldct);
    } else {
      // TC_BRANCH_BWD: dG tile of hidden units [n0, n0 + BN).
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float dg[32];
        tmem_ld32(trow + (uint32_t)c0, dg);
        if (F8) {
#pragma unroll
          for (int j = 0; j < 32; ++j) dg[j] *= sc;
        }
        const int hb = n0 + c0;
        float xs[KB][32];
        float xf[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) xf[j] = 1.f;
#pragma unroll
        for (int i = 0; i < KB; ++i) {
          if (rok) {
            load_row32(e.Aux + (size_t)row * e.ldaux + i * e.H, hb, e.H, xs[i]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) xs[i][j] = 0.f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) xf[j] *= xs[i][j];
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) dg[j] *= gelu_grad_f(xf[j]);
#pragma unroll
        for (int i = 0; i < KB; ++i) {
          float dd[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float o = 1.f;
#pragma unroll
            for (int l = 0; l < KB; ++l)
              if (l != i) o *= xs[l][j];
            dd[j] = dg[j] * o;
          }
          const int colb = i * e.H;
          store_row32(dd, rok, hb, e.H, e.C + (size_t)row * e.ldc + colb, e.Cb + (size_t)row * e.ldcb + colb);
          store_T32(dd, sT, m0, colb + hb, colb + e.H, e.CbT, e.ldct);
        }
      }
    }
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

template <int BN, int MODE, int KB = 1, bool F8 = false>
cudaError_t launch_bn_mode(const TcGemm& g, cudaStream_t st) {
  auto k = gemm_tc_kernel<BN, MODE, KB, F8>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<BN>());
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  });
  if (attr_err != cudaSuccess) return attr_err;
  TcEpi e{g.M, g.N, g.K, g.H, g.k, g.C, g.ldc, g.Cb, g.ldcb, g.CbT, g.ldct, g.bias, g.R, g.ldr, g.Aux, g.ldaux, g.err,
          g.inv_a, g.inv_b, g.b_early ? 1 : 0};
  const int ntile = (MODE == TC_BRANCH) ? (g.H + 31) / 32 : (g.N + BN - 1) / BN;
  dim3 grid(ntile, (g.M + BM - 1) / BM);
  return launch_k(k, grid, dim3(128), smem_bytes<BN>(), st, g.ta, g.tb, e);
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

namespace {
template <bool F8>
cudaError_t launch_gemm_tc_t(const TcGemm& g, cudaStream_t st);
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
  if (g.mode == TC_BRANCH) {
    if (g.box_b != 32 || g.k < 1 || g.k > 3) return cudaErrorInvalidValue;
    switch (g.k) {
      case 1: return launch_bn_mode<32, TC_BRANCH, 1, F8>(g, st);
      case 2: return launch_bn_mode<64, TC_BRANCH, 1, F8>(g, st);
      default: return launch_bn_mode<96, TC_BRANCH, 1, F8>(g, st);
    }
  }
  if (g.box_b != g.bn) return cudaErrorInvalidValue;
  if (g.mode == TC_BRANCH_BWD) {
    if (g.bn != 32 || g.k < 1 || g.k > 3) return cudaErrorInvalidValue;
    switch (g.k) {
      case 1: return launch_bn_mode<32, TC_BRANCH_BWD, 1, F8>(g, st);
      case 2: return launch_bn_mode<32, TC_BRANCH_BWD, 2, F8>(g, st);
      default: return launch_bn_mode<32, TC_BRANCH_BWD, 3, F8>(g, st);
    }
  }
  switch (g.bn) {
    case 32: return launch_bn_mode<32, TC_PLAIN, 1, F8>(g, st);
    case 64: return launch_bn_mode<64, TC_PLAIN, 1, F8>(g, st);
    case 128: return launch_bn_mode<128, TC_PLAIN, 1, F8>(g, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

}  // namespace edpc
