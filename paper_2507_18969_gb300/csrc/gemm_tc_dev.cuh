// Device-side pieces shared by the tcgen05 GEMM kernels (one-tile and
// persistent): PTX wrappers for mbarriers, TMA, tcgen05 MMA / TMEM loads, the
// shared-memory operand descriptors, and the fused epilogue of one 128 x BN
// accumulator tile (plain, MBRB branch Eqs. 10-12, branch adjoint, split-K).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "gemm_tc.cuh"

namespace edpc {
namespace tc {

constexpr int BM = 128;
constexpr int BKB = 128;  // bytes of K per stage row (one 128-byte swizzle span)
template <bool F8>
constexpr int bk_elems() { return F8 ? 128 : 64; }
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
  float* ws;           // split-K partial tiles [splits][M][N]
  unsigned* cnt;       // split-K arrival counter per output tile
  int ntn, ntm;        // persistent kernel: N tiles and M tiles of the problem
  int tma_c, tma_cb;   // C / Cb have output tensor maps: whole 32 x 32 chunks go out by TMA store
  const int4* mt;      // grouped mode (see TcGemm): M tiles of the forward / dX GEMMs
  const int4* gk;      // grouped mode: K ranges of the weight-gradient GEMMs
  long long gs;        // grouped mode: parameter stride between groups (floats)
  int rlim;            // rows at or beyond rlim are not written by the transposed stores
};

// Per-warp output staging for TMA stores: 4 KB FP32 rows (128-byte swizzle)
// then 2 KB BF16 rows (64-byte swizzle); the 4 epilogue warps' areas are 6 KB
// apart (1024-aligned).
constexpr int kStageOutWarp = 6144;
constexpr int kStageOut = 4 * kStageOutWarp;

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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// 3-D tiled load (grouped mode: coordinate c2 selects the group's matrix).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
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

// Barrier of the 128 epilogue threads (named barrier 1; the whole CTA in the
// one-tile kernel, warps 2-5 in the persistent one).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// CTA-uniform AND of a predicate over the 128 epilogue threads.
__device__ __forceinline__ bool epi_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred o, 1, 128, q;\n selp.u32 %0, 1, 0, o;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

// Transposed BF16 store of a 128-row x 32-column chunk: every epilogue thread
// (tile row r, epilogue thread index et) puts its row into shared memory
// (column-major), then the 128 threads write each column's 128 rows as 16-byte
// runs to CT[(n0 + c) * ldct + m0 + row]. Columns at or beyond N and 8-row runs
// at or beyond ldct are skipped. Collective over the epilogue threads.
__device__ __forceinline__ void store_T32(const float (&v)[32], __nv_bfloat16* sT, int m0, int n0, int N,
                                          __nv_bfloat16* CT, int ldct, int r, int et, int rlim) {
#pragma unroll
  for (int c = 0; c < 32; ++c) sT[c * 128 + r] = __float2bfloat16_rn(v[c]);
  epi_sync();
  for (int idx = et; idx < 32 * 16; idx += 128) {
    const int c = idx >> 4, seg = idx & 15;
    const int row0 = m0 + seg * 8;
    if (n0 + c < N && row0 + 8 <= ldct && row0 + 8 <= rlim)
      *reinterpret_cast<uint4*>(CT + (size_t)(n0 + c) * ldct + row0) =
          *reinterpret_cast<const uint4*>(sT + c * 128 + seg * 8);
  }
  epi_sync();
}

// A warp's 32 x 32 FP32 chunk (lane = row; rows r0..r0+31, columns
// [col, col+32) of the tensor behind tm) through shared memory and one TMA
// tensor store. The staging rows follow the 128-byte swizzle of the map.
__device__ __forceinline__ void tma_st_f32(const float (&v)[32], uint8_t* stg, const CUtensorMap* tm, int col, int r0,
                                           int lane) {
  if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // staging free again
  __syncwarp();
  uint8_t* rowp = stg + lane * 128;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    *reinterpret_cast<float4*>(rowp + ((j ^ (lane & 7)) << 4)) =
        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(col), "r"(r0), "r"(smem_u32(stg))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
}

// The same for a BF16 chunk (64-byte rows, 64-byte swizzle), staged 4 KB in.
__device__ __forceinline__ void tma_st_bf16(const float (&v)[32], uint8_t* stg, const CUtensorMap* tm, int col,
                                            int r0, int lane) {
  uint8_t* sb = stg + 4096;
  if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncwarp();
  uint8_t* rowp = sb + lane * 64;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __align__(16) __nv_bfloat162 h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[8 * j + 2 * q], v[8 * j + 2 * q + 1]);
    *reinterpret_cast<uint4*>(rowp + ((j ^ ((lane >> 1) & 3)) << 4)) = *reinterpret_cast<const uint4*>(h);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(col), "r"(r0), "r"(smem_u32(sb))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
}

// Waits until this warp's TMA stores have completed (before the CTA exits).
__device__ __forceinline__ void tma_st_drain(int lane) {
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncwarp();
}

// Output of one 32-column chunk of the warp's 32 rows: whole chunks (columns
// [col, col+32) inside the logical width `w` starting at `base`, all 32 rows
// below M) go out by TMA store when the map exists; others by direct stores.
struct EpiOut {
  const CUtensorMap* tmc;   // C (FP32)
  const CUtensorMap* tmcb;  // Cb (BF16)
  uint8_t* stg;             // this warp's staging area
  int r0, lane;             // first row of the warp's 32 rows; lane
};

__device__ __forceinline__ void out_chunk(const TcEpi& e, const EpiOut& o, const float (&v)[32], bool rok, int row,
                                          int base, int cb, int w, float* C, int ldc, __nv_bfloat16* Cb, int ldcb) {
  // base: first column of the logical region in C / Cb; cb: chunk start within it; w: its width
  const bool whole = cb + 32 <= w && o.r0 + 32 <= e.M;
  if (C) {
    if (whole && e.tma_c)
      tma_st_f32(v, o.stg, o.tmc, base + cb, o.r0, o.lane);
    else
      store_row32(v, rok, cb, w, C + (size_t)row * ldc + base, nullptr);
  }
  if (Cb) {
    if (whole && e.tma_cb)
      tma_st_bf16(v, o.stg, o.tmcb, base + cb, o.r0, o.lane);
    else
      store_row32(v, rok, cb, w, nullptr, Cb + (size_t)row * ldcb + base);
  }
}

template <int BN>
constexpr int tmem_cols() {
  return BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
}
static_assert(tmem_cols<256>() == 256, "N tiles above 256 do not fit one MMA");

// Split-K: every CTA of the tile arrives on the tile's counter after writing
// (and fencing) its FP32 partial; the last to arrive adds the partials of splits
// 0, 1, ..., S - 1 in that order and writes C, then zeroes the counter.
// Collective over the epilogue threads; `flag` is a shared-memory word; S is
// the split count and tile the output tile's counter index.
template <int BN>
__device__ __forceinline__ void splitk_finish(const TcEpi& e, int m0, int n0, int S, int tile, volatile int* flag,
                                              int et) {
  epi_sync();
  if (et == 0) *flag = (atomicAdd(&e.cnt[tile], 1u) == (unsigned)(S - 1)) ? 1 : 0;
  epi_sync();
  if (!*flag) return;
  __threadfence();
  const size_t plane = (size_t)e.M * e.N;
  const bool vec = (e.N % 4 == 0) && (e.ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(e.C) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(e.ws) & 15) == 0);
  constexpr int C4 = BN / 4;
  for (int idx = et; idx < BM * C4; idx += 128) {
    const int r = idx / C4, c = (idx % C4) * 4;
    const int gm = m0 + r, gn = n0 + c;
    if (gm >= e.M || gn >= e.N) continue;
    const float* src = e.ws + (size_t)gm * e.N + gn;
    float* dst = e.C + (size_t)gm * e.ldc + gn;
    if (vec) {
      float4 a = __ldcg(reinterpret_cast<const float4*>(src));
      for (int z = 1; z < S; ++z) {
        const float4 b = __ldcg(reinterpret_cast<const float4*>(src + (size_t)z * plane));
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
      }
      *reinterpret_cast<float4*>(dst) = a;
    } else {
      for (int q = 0; q < 4 && gn + q < e.N; ++q) {
        float a = __ldcg(src + q);
        for (int z = 1; z < S; ++z) a += __ldcg(src + (size_t)z * plane + q);
        dst[q] = a;
      }
    }
  }
  if (et == 0) e.cnt[tile] = 0u;
}

// The fused epilogue of one 128 x BN accumulator tile, run by the 128
// epilogue threads: thread (tile row r, index et) reads TMEM lane r at `trow`
// (its lane group's base plus the accumulator's first column). z, S, tile:
// split-K index, split count and the output tile's counter index. sT: 8 KB of
// shared memory for the transposed stores; flag: a shared word.
// o: the warp's TMA-store state (maps, staging, first row).
template <int BN, int MODE, int KB, bool F8>
__device__ __forceinline__ void tc_epilogue(const TcEpi& e, uint32_t trow, int m0, int n0, int z, int S, int tile,
                                            __nv_bfloat16* sT, volatile int* flag, int r, int et, const EpiOut& o) {
  constexpr int SECTIONS = (MODE == TC_BRANCH) ? KB : 1;
  constexpr int SW = BN / SECTIONS;  // hidden units per branch section (TC_BRANCH)
  const int row = m0 + r;
  const bool rok = row < e.M;
  // FP8: undo the operands' power-of-two scales (exact)
  const float sc = F8 ? e.inv_a[0] * e.inv_b[0] : 1.f;
  if (MODE == TC_PLAIN && S > 1) {
    // split-K: FP32 partial tile -> ws[z], then the tile's last CTA sums in split order
    float* wrow = e.ws + ((size_t)z * e.M + row) * e.N;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(trow + (uint32_t)c0, v);
      if (F8) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= sc;
      }
      store_row32(v, rok, n0 + c0, e.N, wrow, nullptr);
    }
    __threadfence();
    splitk_finish<BN>(e, m0, n0, S, tile, flag, et);
  } else if (MODE == TC_PLAIN) {
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
        float rr[32];
        load_row32(e.R + (size_t)row * e.ldr, nb, e.N, rr);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += rr[j];
      }
      out_chunk(e, o, v, rok, row, 0, nb, e.N, e.C, e.ldc, e.Cb, e.ldcb);
      if (e.CbT) store_T32(v, sT, m0, nb, e.N, e.CbT, e.ldct, r, et, e.rlim);
    }
  } else if (MODE == TC_BRANCH) {
    // X_i for the tile's hidden units h = n0 + c0 + j (32 at a time), then
    // G = GELU(prod X_i); section i of the accumulator is TMEM columns [i*SW, i*SW + SW).
#pragma unroll 1
    for (int c0 = 0; c0 < SW; c0 += 32) {
      const int hb = n0 + c0;
      float g[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) g[j] = 1.f;
#pragma unroll 1
      for (int i = 0; i < SECTIONS; ++i) {
        float v[32];
        tmem_ld32(trow + (uint32_t)(i * SW + c0), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (F8) v[j] *= sc;
          const int h = hb + j;
          if (h < e.H) v[j] += e.bias[i * e.H + h];
          g[j] *= v[j];
        }
        // X_i -> C[row][i*H + h] (FP32, kept for the adjoint)
        out_chunk(e, o, v, rok, row, i * e.H, hb, e.H, e.C, e.ldc, nullptr, 0);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) g[j] = gelu_f(g[j]);
      out_chunk(e, o, g, rok, row, 0, hb, e.H, nullptr, 0, e.Cb, e.ldcb);
      store_T32(g, sT, m0, hb, e.H, e.CbT, e.ldct, r, et, e.rlim);
    }
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
          float prod = 1.f;
#pragma unroll
          for (int l = 0; l < KB; ++l)
            if (l != i) prod *= xs[l][j];
          dd[j] = dg[j] * prod;
        }
        const int colb = i * e.H;
        out_chunk(e, o, dd, rok, row, colb, hb, e.H, e.C, e.ldc, e.Cb, e.ldcb);
        store_T32(dd, sT, m0, colb + hb, colb + e.H, e.CbT, e.ldct, r, et, e.rlim);
      }
    }
  }
}

}  // namespace tc
}  // namespace edpc
