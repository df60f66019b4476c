// The model of Sec. 3 on the GPU and the launch sequence of one step of
// Algorithm 1 for b streams at once.
//
// Forward (Model(x_{i-t..i-1})):
//   embed -> Local MBRBs (LN, branch GEMM, GELU of the product, out GEMM +
//   residual; Eqs. 9-13) -> LTE down (Eq. 14) -> per-stream FDM (Eq. 15) ->
//   LTE up (Eq. 16) -> Global MBRBs -> head GEMM.
// Head: softmax, CDF quantization, coding (encode: ring slot for the coder
//   stage; decode: symbol search inline), CE gradient (Eq. 2).
// Backward: the hand-written adjoint of every forward op in reverse; the FDM
//   adjoint is fused with the FDM's Adam update. Adam on the shared params.
//
// Two arithmetic paths share this sequence:
//   FP32  SIMT GEMMs and separate element-wise kernels.
//   BF16  tcgen05 GEMMs whose epilogues fuse the MBRB element-wise ops and
//         write the BF16 (and transposed BF16) operands of the next GEMMs; the
//         weight-gradient GEMMs and column sums, which nothing on the step's
//         critical path waits for, run on a side stream forked per layer and
//         joined before Adam.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "engine.cuh"
#include "launch.cuh"

namespace edpc {

Dims make_dims(const edpc_cfg& c, int b) {
  Dims d;
  d.b = b;
  d.K = (int)c.context;
  d.D = (int)c.embed_dim;
  d.F = d.K * d.D;
  d.lte = c.latent != 0;
  d.Fp = d.lte ? (int)c.latent : d.F;
  d.H = (int)c.hidden;
  d.n = (int)c.blocks;
  d.nloc = d.n / 2;
  d.k = (int)c.branches;
  d.ldT = (int)round_up(b, kRowsT);
  return d;
}

ParamOff make_offsets(const Dims& d) {
  ParamOff o;
  size_t off = 0;
  auto take = [&](size_t n) {
    size_t r = off;
    off += n;
    return r;
  };
  o.E = take((size_t)256 * d.D);
  for (int j = 0; j < d.n; ++j) {
    o.blk[j].ln_g = take(d.F);
    o.blk[j].ln_b = take(d.F);
    o.blk[j].W = take((size_t)d.k * d.H * d.F);
    o.blk[j].c = take((size_t)d.k * d.H);
    o.blk[j].Wo = take((size_t)d.F * d.H);
    o.blk[j].co = take(d.F);
  }
  if (d.lte) {
    o.W1 = take((size_t)d.Fp * d.F);
    o.b1 = take(d.Fp);
    o.W2 = take((size_t)d.F * d.Fp);
    o.b2 = take(d.F);
  } else {
    o.W1 = o.b1 = o.W2 = o.b2 = off;  // none
  }
  o.Wh = take((size_t)256 * d.F);
  o.bh = take(256);
  o.total = off;
  return o;
}

namespace {

// Timing event: an external event-record node when the stream is being captured.
cudaError_t record_timing(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(st, &cs);
  if (r != cudaSuccess) return r;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                             : cudaEventRecord(e, st);
}

struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += n * sizeof(T);
    return p;
  }
};

// Call-site ids of the BF16 GEMM plan.
enum SiteKind { BR_FWD = 0, OUT_FWD, OUT_DW, OUT_DX, BR_DW, BR_DX, kPerBlockKinds };
constexpr int kSiteLteDownFwd = kPerBlockKinds * kMaxBlocks;
constexpr int kSiteLteUpFwd = kSiteLteDownFwd + 1;
constexpr int kSiteHeadFwd = kSiteLteDownFwd + 2;
constexpr int kSiteHeadDx = kSiteLteDownFwd + 3;
constexpr int kSiteHeadDw = kSiteLteDownFwd + 4;
constexpr int kSiteLteUpDw = kSiteLteDownFwd + 5;
constexpr int kSiteLteUpDx = kSiteLteDownFwd + 6;
constexpr int kSiteLteDownDw = kSiteLteDownFwd + 7;
constexpr int kSiteLteDownDx = kSiteLteDownFwd + 8;
inline int blk_site(int kind, int j) { return kind * kMaxBlocks + j; }

__global__ void set_ctl_kernel(StepCtl* ctl, int i, int t, int bact, int slot, float lr) {
  StepCtl c;
  memset(&c, 0, sizeof(c));
  c.i = i;
  c.t = t;
  c.bact = bact;
  c.inv_bact = bact > 0 ? 1.0f / (float)bact : 0.f;
  c.bc1 = 1.0f - powf(kB1, (float)t);
  c.bc2 = 1.0f - powf(kB2, (float)t);
  c.slot = slot;
  c.lr = lr;
  c.err = 0;
  *ctl = c;
}

}  // namespace

Model::~Model() {
  for (auto& e : ev_fdm)
    if (e) cudaEventDestroy(e);
  for (auto& e : fork)
    if (e) cudaEventDestroy(e);
  if (join_ev) cudaEventDestroy(join_ev);
  if (tr_ev) cudaEventDestroy(tr_ev);
  if (fdm_join_ev) cudaEventDestroy(fdm_join_ev);
  if (dx_ev) cudaEventDestroy(dx_ev);
  if (adam_ev) cudaEventDestroy(adam_ev);
  if (tick_ev) cudaEventDestroy(tick_ev);
  if (bwd_ev) cudaEventDestroy(bwd_ev);
  if (side) cudaStreamDestroy(side);
  if (side_fdm) cudaStreamDestroy(side_fdm);
  if (bwd_st) cudaStreamDestroy(bwd_st);
  if (gU) cudaFree(gU);
  if (f8_arena) cudaFree(f8_arena);
  if (arena_) cudaFree(arena_);
}

int Model::init(const edpc_cfg& cfg, int streams, const std::vector<GroupInfo>* groups) {
  d = make_dims(cfg, streams);
  po = make_offsets(d);
  precision = cfg.precision;
  seed = cfg.seed;
  lr = cfg.lr;
  nparam = po.total;
  np_all = nparam;
  if (groups) {
    // grouped mode: BF16, Algorithm 1's schedule, groups tiling the rows in
    // order with boundaries on multiples of kGroupAlign
    if (precision != EDPC_BF16 || (cfg.flags & (EDPC_FLAG_DELAYED_UPDATE | EDPC_FLAG_OVERLAP_FDM)))
      return fail(EDPC_EINVAL, "independent per-file models in one batch need BF16 and Algorithm 1's schedule");
    if (groups->empty() || groups->size() > 65535) return fail(EDPC_EINVAL, "group count out of range");
    int r = 0;
    for (const GroupInfo& g : *groups) {
      if (g.r0 != r || g.r1 <= g.r0 || g.r0 % kGroupAlign || g.r1 % kGroupAlign || g.s < 1 || g.s > g.r1 - g.r0 ||
          g.rem < 0 || g.rem >= g.s || g.q < 0 || (long long)(g.r1 - g.r0) * d.K > (1ll << 30))
        return fail(EDPC_EINVAL, "malformed group table");
      r = g.r1;
    }
    if (r != streams) return fail(EDPC_EINVAL, "groups do not cover the rows");
    groups_h = *groups;
    ngroups = (int)groups->size();
    gstride = (size_t)round_up((long long)nparam, 64);
    np_all = gstride * (size_t)ngroups;
  }
  const size_t bF = (size_t)d.b * d.F, bFp = (size_t)d.b * d.Fp, bH = (size_t)d.b * d.H;
  const int kH = d.k * d.H;
  const size_t bkH = (size_t)d.b * kH, fdm = (size_t)d.b * d.Fp * d.Fp;
  const bool bf16 = precision != EDPC_FP32;  // BF16 operand copies (also the FP8 mode's sources)
  const bool overlap = bf16 && (cfg.flags & EDPC_FLAG_OVERLAP_FDM);
  const size_t T = d.ldT;

  // weight matrices that need transposed BF16 copies (32 x 32 tiles)
  std::vector<TransposeTile> th;
  if (bf16) {
    auto mat = [&](size_t off, int rows, int cols) {
      for (int r0 = 0; r0 < rows; r0 += 32)
        for (int c0 = 0; c0 < cols; c0 += 32) th.push_back({off, rows, cols, r0, c0});
    };
    for (int j = 0; j < d.n; ++j) {
      mat(po.blk[j].W, kH, d.F);
      mat(po.blk[j].Wo, d.F, d.H);
    }
    if (d.lte) {
      mat(po.W1, d.Fp, d.F);
      mat(po.W2, d.F, d.Fp);
    }
    mat(po.Wh, 256, d.F);
    if (ngroups > 1) {  // every group's matrices
      const size_t n1 = th.size();
      for (int g = 1; g < ngroups; ++g)
        for (size_t t = 0; t < n1; ++t) {
          TransposeTile x = th[t];
          x.off += (unsigned long long)g * gstride;
          th.push_back(x);
        }
    }
  }
  ntiles = (int)th.size();
  // grouped mode: tile list of the forward / dX GEMMs and K ranges of the weight gradients
  std::vector<int4> mt_h, gk_h;
  for (int g = 0; g < ngroups; ++g) {
    const GroupInfo& gi = groups_h[g];
    for (int m0 = gi.r0; m0 < gi.r1; m0 += 128) mt_h.push_back(make_int4(m0, std::min(m0 + 128, gi.r1), g, 0));
    gk_h.push_back(make_int4(gi.r0, (gi.r1 - gi.r0) / 64, 0, 0));
  }
  ngtiles = (int)mt_h.size();
  if (ngtiles > 65535) return fail(EDPC_EINVAL, "too many row tiles for independent models in one batch");

  delayed = (cfg.flags & EDPC_FLAG_DELAYED_UPDATE) != 0;
  const int npar = delayed ? 2 : 1;
  // The FDM update on its own stream (fdm_dx now, fdm_adam beside the next
  // layers, from copies of x' and dy): optional for Algorithm 1's schedule,
  // always for the delayed update, where it leaves the adjoint's critical path.
  const bool split = overlap || delayed;
  // what the forward pass and the head write, the parameters, the FDMs and the
  // step control: one copy, or one per parity for the delayed update
  auto take_parity = [&](Arena& a) {
    P = a.take<float>(np_all);
    U = a.take<float>(fdm);
    ctl = a.take<StepCtl>(1);
    ctx = a.take<uint8_t>((size_t)d.b * d.K);
    for (int s = 0; s < d.n + 2; ++s) S[s] = a.take<float>(bF);
    for (int j = 0; j < d.n; ++j) {
      ba[j].xhat = a.take<float>(bF);
      ba[j].rstd = a.take<float>(d.b);
      ba[j].A = a.take<float>(bkH);
      if (!bf16) {
        ba[j].X0 = a.take<float>(bF);
        ba[j].G = a.take<float>(bH);
      }
    }
    Xp = a.take<float>(bFp);
    Y = a.take<float>(bFp);
    z = a.take<float>((size_t)d.b * 256);
    p = a.take<float>((size_t)d.b * 256);
    dz = a.take<float>((size_t)d.b * 256);
    if (split) {
      xp_pend = a.take<float>(bFp);
      dy_pend = a.take<float>(bFp);
      pend = a.take<FdmPend>(1);
    }
    if (bf16) {
      Pb = a.take<__nv_bfloat16>(np_all);
      PbT = a.take<__nv_bfloat16>(np_all);
      for (int j = 0; j < d.n; ++j) {
        bb[j].X0b = a.take<__nv_bfloat16>(bF);
        bb[j].X0bT = a.take<__nv_bfloat16>((size_t)d.F * T);
        bb[j].Gb = a.take<__nv_bfloat16>(bH);
        bb[j].GbT = a.take<__nv_bfloat16>((size_t)d.H * T);
      }
      Slte_b = a.take<__nv_bfloat16>(bF);
      Slte_bT = a.take<__nv_bfloat16>((size_t)d.F * T);
      Shead_b = a.take<__nv_bfloat16>(bF);
      Shead_bT = a.take<__nv_bfloat16>((size_t)d.F * T);
      Yb = a.take<__nv_bfloat16>(bFp);
      YbT = a.take<__nv_bfloat16>((size_t)d.Fp * T);
      dzb = a.take<__nv_bfloat16>((size_t)d.b * 256);
      dzbT = a.take<__nv_bfloat16>((size_t)256 * T);
    }
  };

  for (int pass = 0; pass < 2; ++pass) {
    Arena a;
    a.base = static_cast<char*>(arena_);
    for (int q = 0; q < npar; ++q) {
      take_parity(a);
      save_parity(q);
    }
    G = a.take<float>(np_all);
    M = a.take<float>(np_all);
    V = a.take<float>(np_all);
    if (ngroups) {
      row_grp = a.take<int>(d.b);
      ginfo = a.take<GroupInfo>(ngroups);
      gtiles = a.take<int4>(ngtiles);
      gkr = a.take<int4>(ngroups);
    }
    Um = a.take<float>(fdm);
    Uv = a.take<float>(fdm);
    dY = a.take<float>(bFp);
    dXp = a.take<float>(bFp);
    if (embed_bwd_chunks(d.b, d.K) > 1) {
      emb_part = a.take<float>((size_t)256 * embed_bwd_chunks(d.b, d.K) * d.D);
      emb_cnt = a.take<unsigned>(256);
    }
    if (bf16) {
      // column sums of one launch: at most 4 jobs of at most max(F, kH, 256) columns
      // (32-column tiles, or 128-column tiles each rounded up: 4 * ceil(max / 128) * 128 columns)
      const int maxc = std::max(std::max(d.F, kH), 256);
      cs_tiles = 4 * ((maxc + 31) / 32);
      cs_cols = 4 * ((maxc + 127) / 128) * 128;
      cs_part = a.take<float>((size_t)cs_cols * kColsumMaxChunks);
      cs_cnt = a.take<unsigned>((size_t)cs_tiles);
      // split-K scratch: the largest splitk * M * N of any dW GEMM at any N tile
      sk_ws_floats = 0;
      const int dw[5][2] = {{d.F, d.H}, {kH, d.F}, {256, d.F}, {d.F, d.Fp}, {d.Fp, d.F}};
      for (const auto& mn : dw)
        for (int bn : {32, 64, 128, 256}) {
          const int sk = tc_splitk(mn[0], mn[1], d.b, bn);
          if (sk > 1) sk_ws_floats = std::max(sk_ws_floats, (size_t)sk * mn[0] * mn[1]);
        }
      if (sk_ws_floats) {
        sk_ws = a.take<float>(sk_ws_floats);
        sk_cnt = a.take<unsigned>(kSplitCounters);
      }
    }
    if (!bf16) {
      dXa = a.take<float>(bF);
      dXb = a.take<float>(bF);
      dX0 = a.take<float>(bF);
      dA = a.take<float>(bkH);
      dG = a.take<float>(bH);
    } else {
      tiles = a.take<TransposeTile>(std::max(1, ntiles));
      for (int j = 0; j < d.n; ++j) {
        BlockBf16& q = bb[j];
        q.dOut = a.take<float>(bF);
        q.dOutb = a.take<__nv_bfloat16>(bF);
        q.dOutbT = a.take<__nv_bfloat16>((size_t)d.F * T);
        q.dA = a.take<float>(bkH);
        q.dAb = a.take<__nv_bfloat16>(bkH);
        q.dAbT = a.take<__nv_bfloat16>((size_t)kH * T);
        q.dX0 = a.take<float>(bF);
      }
      dLte = a.take<float>(bF);
      dLteb = a.take<__nv_bfloat16>(bF);
      dLtebT = a.take<__nv_bfloat16>((size_t)d.F * T);
      dXpb = a.take<__nv_bfloat16>(bFp);
      dXpbT = a.take<__nv_bfloat16>((size_t)d.Fp * T);
      dh0 = a.take<float>(bF);
    }
    if (pass == 0) {
      arena_bytes_ = a.off + 256;
      cudaError_t e = cudaMalloc(&arena_, arena_bytes_);
      if (e != cudaSuccess) {
        arena_ = nullptr;
        return fail(EDPC_ENOMEM, "device allocation of " + std::to_string(arena_bytes_) + " bytes failed");
      }
    }
  }
  if (!d.lte) {
    // "w/o LTE": the FDM reads the last Local block's output and writes the
    // first Global block's input; in BF16 mode its adjoint reads that input's
    // gradient and writes the last Local block's output gradient and its BF16
    // copies (the FP32 adjoint sets dY and dXp per step).
    for (int q = 0; q < npar; ++q) {
      par[q].Xp = par[q].S[d.nloc];
      par[q].Y = par[q].S[d.nloc + 1];
      par[q].Yb = par[q].YbT = nullptr;
    }
  }
  select(0);
  if (!d.lte) {
    if (bf16) {
      dY = dLte;
      if (d.nloc > 0) {
        dXp = bb[d.nloc - 1].dOut;
        dXpb = bb[d.nloc - 1].dOutb;
        dXpbT = bb[d.nloc - 1].dOutbT;
      } else {
        dXp = dh0;
        dXpb = dXpbT = nullptr;
      }
    }
  }
  cudaStream_t st = 0;
  // zero everything once (transposed copies keep zero padding columns)
  EDPC_CUDA(cudaMemsetAsync(arena_, 0, arena_bytes_, st));
  // Initial values (counter-based SplitMix64 rule, tensor id = canonical order).
  const double F = d.F, H = d.H, Fp = d.Fp;
  struct Tn {
    size_t off, n;
    float bound;
    float fill;
  };
  std::vector<Tn> ts;
  ts.push_back({po.E, (size_t)256 * d.D, (float)std::sqrt(3.0), 0.f});
  for (int j = 0; j < d.n; ++j) {
    const BlockOff& b = po.blk[j];
    ts.push_back({b.ln_g, (size_t)d.F, -1.f, 1.f});
    ts.push_back({b.ln_b, (size_t)d.F, -1.f, 0.f});
    ts.push_back({b.W, (size_t)kH * d.F, (float)(1.0 / std::sqrt(F)), 0.f});
    ts.push_back({b.c, (size_t)kH, (float)(1.0 / std::sqrt(F)), 0.f});
    ts.push_back({b.Wo, (size_t)d.F * d.H, (float)(1.0 / std::sqrt(H)), 0.f});
    ts.push_back({b.co, (size_t)d.F, (float)(1.0 / std::sqrt(H)), 0.f});
  }
  if (d.lte) {  // tensor ids follow the canonical order, which has no LTE tensors without it
    ts.push_back({po.W1, (size_t)d.Fp * d.F, (float)(1.0 / std::sqrt(F)), 0.f});
    ts.push_back({po.b1, (size_t)d.Fp, (float)(1.0 / std::sqrt(F)), 0.f});
    ts.push_back({po.W2, (size_t)d.F * d.Fp, (float)(1.0 / std::sqrt(Fp)), 0.f});
    ts.push_back({po.b2, (size_t)d.F, (float)(1.0 / std::sqrt(Fp)), 0.f});
  }
  ts.push_back({po.Wh, (size_t)256 * d.F, (float)(1.0 / std::sqrt(F)), 0.f});
  ts.push_back({po.bh, (size_t)256, (float)(1.0 / std::sqrt(F)), 0.f});
  for (size_t tid = 0; tid < ts.size(); ++tid)
    EDPC_CUDA(launch_init_values(P + ts[tid].off, ts[tid].n, seed, (int)tid, ts[tid].bound, 0, ts[tid].fill, st));
  if (ngroups) {
    // every group starts from the same initial values (those of a single-file model)
    for (int g = 1; g < ngroups; ++g)
      EDPC_CUDA(cudaMemcpyAsync(P + (size_t)g * gstride, P, nparam * sizeof(float), cudaMemcpyDeviceToDevice, st));
    std::vector<int> rg(d.b);
    for (int g = 0; g < ngroups; ++g)
      for (int r = groups_h[g].r0; r < groups_h[g].r1; ++r) rg[r] = g;
    EDPC_CUDA(cudaMemcpyAsync(row_grp, rg.data(), sizeof(int) * d.b, cudaMemcpyHostToDevice, st));
    EDPC_CUDA(cudaMemcpyAsync(ginfo, groups_h.data(), sizeof(GroupInfo) * ngroups, cudaMemcpyHostToDevice, st));
    EDPC_CUDA(cudaMemcpyAsync(gtiles, mt_h.data(), sizeof(int4) * ngtiles, cudaMemcpyHostToDevice, st));
    EDPC_CUDA(cudaMemcpyAsync(gkr, gk_h.data(), sizeof(int4) * ngroups, cudaMemcpyHostToDevice, st));
    EDPC_CUDA(cudaStreamSynchronize(st));  // the host tables above are locals
  }
  if (ngroups) {
    // each group's FDMs start as its file's would alone: row j of the group
    // takes the values of stream j (the counter restarts at the group's first row)
    const size_t per = (size_t)d.Fp * d.Fp;
    for (const GroupInfo& g : groups_h)
      EDPC_CUDA(launch_init_values(U + (size_t)g.r0 * per, (size_t)(g.r1 - g.r0) * per, seed, kFdmTid,
                                   (float)std::sqrt(3.0 / Fp), 0, 0.f, st));
  } else {
    EDPC_CUDA(launch_init_values(U, fdm, seed, kFdmTid, (float)std::sqrt(3.0 / Fp), 0, 0.f, st));
  }
  // Stream priorities (the default is the least): with the delayed update the
  // adjoint's streams go first and the FDM update last.
  int prio_least = 0, prio_greatest = 0;
  EDPC_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
  if (bf16) {
    if (ntiles) EDPC_CUDA(cudaMemcpyAsync(tiles, th.data(), th.size() * sizeof(TransposeTile), cudaMemcpyHostToDevice, st));
    EDPC_TRY(refresh_bf16_weights(st));
    EDPC_TRY(build_tc_plan());
    EDPC_CUDA(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, delayed ? prio_greatest : prio_least));
    for (auto& e : fork) EDPC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    EDPC_CUDA(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
    EDPC_CUDA(cudaEventCreateWithFlags(&tr_ev, cudaEventDisableTiming));
    EDPC_CUDA(cudaEventCreateWithFlags(&fdm_join_ev, cudaEventDisableTiming));
  }
  if (split) {
    EDPC_CUDA(cudaStreamCreateWithPriority(&side_fdm, cudaStreamNonBlocking, prio_least));
    EDPC_CUDA(cudaEventCreateWithFlags(&dx_ev, cudaEventDisableTiming));
    EDPC_CUDA(cudaEventCreateWithFlags(&adam_ev, cudaEventDisableTiming));
  }
  if (delayed) {
    // the adjoint (the longer of the two chains of a step) and its side stream first
    EDPC_CUDA(cudaStreamCreateWithPriority(&bwd_st, cudaStreamNonBlocking, prio_greatest));
    EDPC_CUDA(cudaEventCreateWithFlags(&tick_ev, cudaEventDisableTiming));
    EDPC_CUDA(cudaEventCreateWithFlags(&bwd_ev, cudaEventDisableTiming));
  }
  EDPC_CUDA(cudaStreamSynchronize(st));
  return EDPC_OK;
}

void Model::save_parity(int q) {
  Parity& r = par[q];
  r.P = P;
  r.U = U;
  r.Pb = Pb;
  r.PbT = PbT;
  r.ctl = ctl;
  r.ctx = ctx;
  for (int s = 0; s < kMaxBlocks + 2; ++s) r.S[s] = S[s];
  for (int j = 0; j < kMaxBlocks; ++j) {
    r.ba[j] = ba[j];
    r.X0b[j] = bb[j].X0b;
    r.X0bT[j] = bb[j].X0bT;
    r.Gb[j] = bb[j].Gb;
    r.GbT[j] = bb[j].GbT;
  }
  r.Slte_b = Slte_b;
  r.Slte_bT = Slte_bT;
  r.Shead_b = Shead_b;
  r.Shead_bT = Shead_bT;
  r.Yb = Yb;
  r.YbT = YbT;
  r.dzb = dzb;
  r.dzbT = dzbT;
  r.Xp = Xp;
  r.Y = Y;
  r.z = z;
  r.p = p;
  r.dz = dz;
  r.xp_pend = xp_pend;
  r.dy_pend = dy_pend;
  r.pend = pend;
}

void Model::select(int q) {
  const Parity& r = par[q];
  P = r.P;
  U = r.U;
  Pb = r.Pb;
  PbT = r.PbT;
  ctl = r.ctl;
  ctx = r.ctx;
  for (int s = 0; s < kMaxBlocks + 2; ++s) S[s] = r.S[s];
  for (int j = 0; j < kMaxBlocks; ++j) {
    ba[j] = r.ba[j];
    bb[j].X0b = r.X0b[j];
    bb[j].X0bT = r.X0bT[j];
    bb[j].Gb = r.Gb[j];
    bb[j].GbT = r.GbT[j];
  }
  Slte_b = r.Slte_b;
  Slte_bT = r.Slte_bT;
  Shead_b = r.Shead_b;
  Shead_bT = r.Shead_bT;
  Yb = r.Yb;
  YbT = r.YbT;
  dzb = r.dzb;
  dzbT = r.dzbT;
  Xp = r.Xp;
  Y = r.Y;
  z = r.z;
  p = r.p;
  dz = r.dz;
  xp_pend = r.xp_pend;
  dy_pend = r.dy_pend;
  pend = r.pend;
  U_base = delayed ? par[q ^ 1].U : nullptr;
  cur = q;
}

int Model::set_ctl_for_step(int i, int t, int bact, int ring_slots, cudaStream_t st) {
  int slot = ring_slots > 0 ? (int)(((long long)i - d.K) % ring_slots) : 0;
  if (slot < 0) slot = 0;
  if (!delayed) {
    set_ctl_kernel<<<1, 1, 0, st>>>(ctl, i, t, bact, slot, lr);
    EDPC_CUDA(cudaGetLastError());
    return EDPC_OK;
  }
  // Delayed update: both parities start at the first step. The first step's
  // adjoint runs on parity 1 with a zero head gradient (every gradient is then
  // zero), so its updates copy parity 0's parameters and FDMs exactly.
  for (int q = 0; q < 2; ++q) {
    set_ctl_kernel<<<1, 1, 0, st>>>(par[q].ctl, i, t, bact, slot, lr);
    EDPC_CUDA(cudaGetLastError());
  }
  EDPC_CUDA(cudaMemsetAsync(par[1].dz, 0, sizeof(float) * d.b * 256, st));
  if (par[1].dzb) EDPC_CUDA(cudaMemsetAsync(par[1].dzb, 0, sizeof(__nv_bfloat16) * d.b * 256, st));
  if (par[1].dzbT) EDPC_CUDA(cudaMemsetAsync(par[1].dzbT, 0, sizeof(__nv_bfloat16) * 256 * d.ldT, st));
  return EDPC_OK;
}

int Model::refresh_bf16_weights(cudaStream_t st) {
  if (np_all > (size_t)INT32_MAX) return fail(EDPC_EINVAL, "parameter count exceeds 2^31 - 1");
  EDPC_CUDA(launch_to_bf16(P, 1, (int)np_all, (int)np_all, Pb, (int)np_all, nullptr, 0, st));
  EDPC_CUDA(launch_transpose_tiles(Pb, PbT, tiles, ntiles, st));
  return EDPC_OK;
}

// ==========================================================================================
// FP32 path
// ==========================================================================================
int Model::linear_fwd(const float* X, int rows, int in, size_t w_off, size_t b_off, int out, const float* resid,
                      float* Yo, cudaStream_t st) {
  const int epi = resid ? EPI_BIAS_RESID : EPI_BIAS;
  GemmF32 g{rows, out, in, X, in, true, P + w_off, in, true, Yo, out, epi, P + b_off, resid, out};
  EDPC_CUDA(launch_gemm_f32(g, st));
  return EDPC_OK;
}

int Model::linear_dx(const float* dOut, int rows, int out, size_t w_off, int in, float* dX, cudaStream_t st) {
  GemmF32 g{rows, in, out, dOut, out, true, P + w_off, in, false, dX, in, EPI_STORE, nullptr, nullptr, 0};
  EDPC_CUDA(launch_gemm_f32(g, st));
  return EDPC_OK;
}

int Model::linear_dw(const float* dOut, int rows, int out, const float* X, int in, size_t w_off, cudaStream_t st) {
  GemmF32 g{out, in, rows, dOut, out, false, X, in, false, G + w_off, in, EPI_STORE, nullptr, nullptr, 0};
  EDPC_CUDA(launch_gemm_f32(g, st));
  return EDPC_OK;
}

int Model::block_fwd(int j, const float* Xin, float* Xout, cudaStream_t st) {
  const BlockOff& o = po.blk[j];
  BlockAct& a = ba[j];
  const int kH = d.k * d.H;
  EDPC_CUDA(launch_ln_fwd(Xin, P + o.ln_g, P + o.ln_b, a.xhat, a.rstd, a.X0, d.b, d.F, st));  // Eq. 9
  EDPC_TRY(linear_fwd(a.X0, d.b, d.F, o.W, o.c, kH, nullptr, a.A, st));                       // Eq. 10
  EDPC_CUDA(launch_branch_gelu(a.A, d.b, d.H, d.k, a.G, st));                                 // Eqs. 11-12
  EDPC_TRY(linear_fwd(a.G, d.b, d.H, o.Wo, o.co, d.F, Xin, Xout, st));                        // Eq. 13
  return EDPC_OK;
}

int Model::fdm_fwd_call(const StepIO& io, cudaStream_t st) {
  const bool waited = fdm_pending;
  EDPC_TRY(flush(st));  // the previous step's FDM update must have landed
  if (timing && ev_fdm[0]) EDPC_CUDA(record_timing(ev_fdm[0], st));
  FdmAct act;
  act.ctl = ctl;
  act.sp = io.sp;
  act.active = io.mode == 2 ? io.active : nullptr;
  if (waited) {
    NoPdl scope;  // first launch after a cross-stream wait
    EDPC_CUDA(launch_fdm_fwd(Xp, U, Y, d.b, d.Fp, st, Yb, YbT, d.ldT, &ctl->err, act));  // Eq. 15
  } else {
    EDPC_CUDA(launch_fdm_fwd(Xp, U, Y, d.b, d.Fp, st, Yb, YbT, d.ldT, &ctl->err, act));  // Eq. 15
  }
  if (timing && ev_fdm[1]) EDPC_CUDA(record_timing(ev_fdm[1], st));
  return EDPC_OK;
}

int Model::forward_f32(const StepIO& io, cudaStream_t st) {
  EDPC_CUDA(launch_embed(io.mode == 2 ? nullptr : io.data, io.sp, ctl, P + po.E, d.b, d.K, d.D, S[0], ctx, st));
  for (int j = 0; j < d.nloc; ++j) EDPC_TRY(block_fwd(j, S[j], S[j + 1], st));
  if (d.lte) EDPC_TRY(linear_fwd(S[d.nloc], d.b, d.F, po.W1, po.b1, d.Fp, nullptr, Xp, st));  // Eq. 14
  EDPC_TRY(fdm_fwd_call(io, st));  // Eq. 15 (w/o LTE: on S[nloc] into S[nloc + 1])
  if (d.lte) EDPC_TRY(linear_fwd(Y, d.b, d.Fp, po.W2, po.b2, d.F, nullptr, S[d.nloc + 1], st));  // Eq. 16
  for (int j = d.nloc; j < d.n; ++j) EDPC_TRY(block_fwd(j, S[j + 1], S[j + 2], st));
  EDPC_TRY(linear_fwd(S[d.n + 1], d.b, d.F, po.Wh, po.bh, 256, nullptr, z, st));
  return EDPC_OK;
}

int Model::block_bwd(int j, const float* dOut, float* dXnew, cudaStream_t st) {
  const BlockOff& o = po.blk[j];
  BlockAct& a = ba[j];
  const int kH = d.k * d.H;
  // Eq. 13: out = G Wo^T + co + X
  EDPC_TRY(linear_dw(dOut, d.b, d.F, a.G, d.H, o.Wo, st));
  EDPC_CUDA(launch_colsum(dOut, nullptr, d.b, d.F, d.F, G + o.co, st));
  EDPC_TRY(linear_dx(dOut, d.b, d.F, o.Wo, d.H, dG, st));
  // Eqs. 11-12: G = GELU(prod X_i)
  EDPC_CUDA(launch_branch_gelu_bwd(dG, a.A, d.b, d.H, d.k, dA, st));
  // Eq. 10: X_i = X0 W_i^T + c_i
  EDPC_TRY(linear_dw(dA, d.b, kH, a.X0, d.F, o.W, st));
  EDPC_CUDA(launch_colsum(dA, nullptr, d.b, kH, kH, G + o.c, st));
  EDPC_TRY(linear_dx(dA, d.b, kH, o.W, d.F, dX0, st));
  // Eq. 9: X0 = g * xhat + beta, plus the residual path of Eq. 13
  EDPC_CUDA(launch_colsum(dX0, a.xhat, d.b, d.F, d.F, G + o.ln_g, st));
  EDPC_CUDA(launch_colsum(dX0, nullptr, d.b, d.F, d.F, G + o.ln_b, st));
  EDPC_CUDA(launch_ln_bwd(dX0, a.xhat, a.rstd, P + o.ln_g, dOut, dXnew, d.b, d.F, st));
  return EDPC_OK;
}

int Model::flush(cudaStream_t st) {
  if (!fdm_pending) return EDPC_OK;
  EDPC_CUDA(cudaStreamWaitEvent(st, adam_ev, 0));
  fdm_pending = false;
  return EDPC_OK;
}

int Model::fdm_bwd_call(const StepIO& io, cudaStream_t st) {
  if (side_fdm && io.update) {
    // dx' now (the rest of the adjoint needs it); U's Adam update on its own
    // stream, overlapping the rest of this step and the next step's layers up
    // to the FDM forward, which waits for it (flush).
    FdmSplitArgs sa{};
    sa.Xp = Xp;
    sa.dY = dY;
    sa.U = U;
    sa.Um = Um;
    sa.Uv = Uv;
    sa.dXp = dXp;
    sa.dXpb = dXpb;
    sa.dXpbT = dXpbT;
    sa.ldT = d.ldT;
    sa.xp_pend = xp_pend;
    sa.dy_pend = dy_pend;
    sa.pend = pend;
    sa.ctl = ctl;
    sa.sp = io.sp;
    sa.active = io.mode == 2 ? io.active : nullptr;
    sa.b = d.b;
    sa.Fp = d.Fp;
    sa.Ub = U_base;  // delayed update: Adam from the next step's FDMs into this parity's
    if (timing && ev_fdm[2]) EDPC_CUDA(record_timing(ev_fdm[2], st));
    EDPC_CUDA(launch_fdm_dx(sa, st));
    if (timing && ev_fdm[3]) EDPC_CUDA(record_timing(ev_fdm[3], st));
    EDPC_CUDA(cudaEventRecord(dx_ev, st));
    EDPC_CUDA(cudaStreamWaitEvent(side_fdm, dx_ev, 0));
    {
      NoPdl scope;
      if (timing && ev_fdm[4]) EDPC_CUDA(record_timing(ev_fdm[4], side_fdm));
      // delayed update: a CTA per 32 rows on a low-priority stream, so that
      // the adjoint's and the forward pass's GEMM CTAs (up to 255 registers a
      // thread, which leave no room beside a resident update CTA) go first
      EDPC_CUDA(launch_fdm_adam(sa, side_fdm, !delayed));
      if (timing && ev_fdm[5]) EDPC_CUDA(record_timing(ev_fdm[5], side_fdm));
    }
    EDPC_CUDA(cudaEventRecord(adam_ev, side_fdm));
    fdm_pending = true;
    return EDPC_OK;
  }
  FdmBwdArgs fa{};
  fa.Xp = Xp;
  fa.dY = dY;
  fa.U = U;
  fa.Um = Um;
  fa.Uv = Uv;
  fa.dXp = dXp;
  fa.gU = gU;
  fa.ctl = ctl;
  fa.sp = io.sp;
  fa.active = io.mode == 2 ? io.active : nullptr;
  fa.b = d.b;
  fa.Fp = d.Fp;
  fa.update = io.update;
  fa.dXpb = dXpb;
  fa.dXpbT = dXpbT;
  fa.ldT = d.ldT;
  if (timing && ev_fdm[2]) EDPC_CUDA(record_timing(ev_fdm[2], st));
  EDPC_CUDA(launch_fdm_bwd(fa, st));
  if (timing && ev_fdm[3]) EDPC_CUDA(record_timing(ev_fdm[3], st));
  return EDPC_OK;
}

int Model::backward_f32(const StepIO& io, cudaStream_t st) {
  const float* head_in = S[d.n + 1];
  EDPC_TRY(linear_dw(dz, d.b, 256, head_in, d.F, po.Wh, st));
  EDPC_CUDA(launch_colsum(dz, nullptr, d.b, 256, 256, G + po.bh, st));
  EDPC_TRY(linear_dx(dz, d.b, 256, po.Wh, d.F, dXa, st));
  float* cur = dXa;
  float* nxt = dXb;
  for (int j = d.n - 1; j >= d.nloc; --j) {
    EDPC_TRY(block_bwd(j, cur, nxt, st));
    std::swap(cur, nxt);
  }
  if (d.lte) {
    // LTE up (Eq. 16)
    EDPC_TRY(linear_dw(cur, d.b, d.F, Y, d.Fp, po.W2, st));
    EDPC_CUDA(launch_colsum(cur, nullptr, d.b, d.F, d.F, G + po.b2, st));
    EDPC_TRY(linear_dx(cur, d.b, d.F, po.W2, d.Fp, dY, st));
    // FDM (Eq. 15): adjoint fused with the FDM's Adam update
    EDPC_TRY(fdm_bwd_call(io, st));
    // LTE down (Eq. 14)
    EDPC_TRY(linear_dw(dXp, d.b, d.Fp, S[d.nloc], d.F, po.W1, st));
    EDPC_CUDA(launch_colsum(dXp, nullptr, d.b, d.Fp, d.Fp, G + po.b1, st));
    EDPC_TRY(linear_dx(dXp, d.b, d.Fp, po.W1, d.F, cur, st));
  } else {
    // w/o LTE: the FDM's adjoint maps the gradient of S[nloc + 1] to that of S[nloc]
    dY = cur;
    dXp = nxt;
    EDPC_TRY(fdm_bwd_call(io, st));
    std::swap(cur, nxt);
  }
  for (int j = d.nloc - 1; j >= 0; --j) {
    EDPC_TRY(block_bwd(j, cur, nxt, st));
    std::swap(cur, nxt);
  }
  EDPC_CUDA(launch_embed_bwd(ctx, cur, d.b, d.K, d.D, G + po.E, emb_part, emb_cnt, st));
  return EDPC_OK;
}

// ==========================================================================================
// BF16 path
// ==========================================================================================
// FP8 e4m3 shadow of a BF16 operand matrix (one per distinct source).
int Model::fp8_shadow(const void* src, int rows, int cols, int ld) {
  const auto* p = static_cast<const __nv_bfloat16*>(src);
  for (size_t i = 0; i < f8.size(); ++i)
    if (f8[i].src == p && f8[i].rows == rows && f8[i].cols == cols && f8[i].ld == ld) return (int)i;
  Fp8Shadow sh;
  sh.src = p;
  sh.rows = rows;
  sh.cols = cols;
  sh.ld = ld;
  sh.ld8 = (int)round_up(cols, 16);
  // quantized columns: whole 8-element vectors; a transposed operand's extra
  // columns up to ld are its zero padding (b rounded up to 16)
  sh.qcols = (int)std::min<long long>(ld, round_up(cols, 8));
  sh.weight = (p >= Pb && p < Pb + nparam) || (p >= PbT && p < PbT + nparam);
  sh.transposed = p >= PbT && p < PbT + nparam;
  f8.push_back(sh);
  return (int)f8.size() - 1;
}

int Model::build_tc_plan() {
  if (!delayed) return build_tc_plan_one();
  const int keep = cur;
  int r = EDPC_OK;
  for (int q = 0; q < 2 && r == EDPC_OK; ++q) {
    select(q);
    r = build_tc_plan_one();
    if (r == EDPC_OK) par[q].tcp = tcp;
  }
  select(keep);
  return r;
}

int Model::build_tc_plan_one() {
  if (precision == EDPC_FP8E4M3 && !f8_arena) {
    // first pass: collect the operand shadows; then allocate them
    f8.clear();
    f8_collect = true;
    int r = build_tc_sites();
    f8_collect = false;
    if (r != EDPC_OK) return r;
    size_t tot = 256 + 8 * f8.size();  // amax words and inverse scales first
    for (auto& sh : f8) tot += round_up((long long)sh.rows * sh.ld8, 256);
    EDPC_CUDA(cudaMalloc(&f8_arena, tot));
    EDPC_CUDA(cudaMemset(f8_arena, 0, tot));
    f8_amax = reinterpret_cast<unsigned*>(f8_arena);
    f8_inv = reinterpret_cast<float*>(f8_arena + 4 * f8.size());
    size_t off = round_up(8 * (long long)f8.size(), 256);
    for (auto& sh : f8) {
      sh.dst = f8_arena + off;
      off += round_up((long long)sh.rows * sh.ld8, 256);
    }
    f8_done.assign(f8.size(), 0);
  }
  return build_tc_sites();
}

// FP8: quantizes the step's weight shadows (transposed ones or not) in one
// amax + convert launch pair per group of kMaxFp8Jobs.
int Model::quantize_weights(bool transposed, cudaStream_t st) {
  Fp8Jobs J{};
  J.amax = f8_amax;
  J.inv = f8_inv;
  for (size_t i = 0; i <= f8.size(); ++i) {
    if (i < f8.size() && f8[i].weight && f8[i].transposed == transposed) {
      const Fp8Shadow& sh = f8[i];
      J.job[J.n++] = {sh.src, sh.rows, sh.qcols, sh.ld, sh.dst, sh.ld8, (int)i};
    }
    if (J.n == kMaxFp8Jobs || (i == f8.size() && J.n)) {
      EDPC_CUDA(launch_fp8_quantize(J, st));
      J.n = 0;
    }
  }
  return EDPC_OK;
}

// FP8: quantizes the activation shadows a GEMM site reads, once per step.
int Model::quantize_site(int site, cudaStream_t st) {
  Fp8Jobs J{};
  J.amax = f8_amax;
  J.inv = f8_inv;
  for (int id : {site_fa[site], site_fb[site]}) {
    if (f8[id].weight || f8_done[id]) continue;
    const Fp8Shadow& sh = f8[id];
    J.job[J.n++] = {sh.src, sh.rows, sh.qcols, sh.ld, sh.dst, sh.ld8, id};
    f8_done[id] = 1;
  }
  if (J.n) EDPC_CUDA(launch_fp8_quantize(J, st));
  return EDPC_OK;
}

int Model::build_tc_sites() {
  const int kH = d.k * d.H;
  const int T = d.ldT;
  // N tile: the site's tile code when one is set (tuned or read from a
  // bitstream); else 32 while 64-wide tiles would leave the GPU mostly idle
  // (small b), else 64; the GEMMs over the streams (M = b) take 128-wide
  // tiles from 2048 streams on, where they were measured fastest.
  // Grouped mode: tile shapes that do not depend on the batch (a member's
  // arithmetic must be the same alone and in any batch).
  const bool big = !ngroups && d.b >= 2048;
  auto bn_heur = [&](int N) { return ngroups ? 64 : (((d.b + 127) / 128) * ((N + 63) / 64) < 2 * 152 ? 32 : 64); };
  auto bn_site = [&](int id, int N) { return (tile_code[id] & 15) ? 32 * (tile_code[id] & 15) : bn_heur(N); };
  auto bn_rows = [&](int id, int N) { return (tile_code[id] & 15) || !big ? bn_site(id, N) : 128; };
  // Weight gradients: in grouped mode every group contracts only its own rows
  // (a few K blocks), so wide N tiles keep the CTA count (groups x tiles) and
  // the per-CTA fixed cost down.
  auto bn_dw = [&](int id, int N) { return ngroups ? (N >= 256 ? 256 : (N >= 128 ? 128 : (N >= 64 ? 64 : 32)))
                                                   : bn_site(id, N); };
  // dW GEMMs (K = streams): split K when the output has too few tiles for the GPU
  auto split_site = [&](int id) -> int {
    TcGemm& g = tcp.site[id];
    g.splitk = ngroups ? 1 : tc_splitk(g.M, g.N, g.K, g.bn);  // grouped: each group's own K range
    if (g.splitk > 1) {
      if (!sk_ws || (size_t)g.splitk * g.M * g.N > sk_ws_floats || tc_tiles(g.M, g.N, g.bn) > kSplitCounters)
        return fail(EDPC_EINVAL, "split-K GEMM exceeds its scratch");
      g.ws = sk_ws;
      g.cnt = sk_cnt;
    } else {
      g.ws = nullptr;
      g.cnt = nullptr;
    }
    return EDPC_OK;
  };
  auto site = [&](int id, int M, int N, int K, const void* a, int a_rows, int a_cols, int a_ld, const void* b,
                  int b_rows, int b_cols, int b_ld, int bn, int box_b) -> int {
    TcGemm& g = tcp.site[id];
    g.M = M;
    g.N = N;
    g.K = K;
    g.bn = bn;
    g.persistent = (tile_code[id] & 16) != 0;
    g.box_b = box_b;
    g.err = &ctl->err;
    if (precision == EDPC_FP8E4M3) {
      // e4m3 shadows of both BF16 operands, quantized before the launch
      const int ia = fp8_shadow(a, a_rows, a_cols, a_ld), ib = fp8_shadow(b, b_rows, b_cols, b_ld);
      site_fa[id] = ia;
      site_fb[id] = ib;
      if (f8_collect) return EDPC_OK;
      EDPC_TRY(make_tmap_u8(&g.ta, f8[ia].dst, a_rows, a_cols, f8[ia].ld8, 128));
      EDPC_TRY(make_tmap_u8(&g.tb, f8[ib].dst, b_rows, b_cols, f8[ib].ld8, box_b));
      g.fp8 = true;
      g.inv_a = f8_inv + ia;
      g.inv_b = f8_inv + ib;
      g.b_early = f8[ib].weight;  // activation shadows are written by the launch just before
      return EDPC_OK;
    }
    EDPC_TRY(make_tmap_bf16(&g.ta, a, a_rows, a_cols, a_ld, 128));
    EDPC_TRY(make_tmap_bf16(&g.tb, b, b_rows, b_cols, b_ld, box_b));
    g.mt = nullptr;
    g.gk = nullptr;
    if (ngroups) {
      // grouped mode: a weight operand is one matrix per group (3-D map, tile
      // list over the groups' rows); otherwise B holds activations and the
      // GEMM is a weight gradient contracting each group's own rows
      const auto* pb = static_cast<const __nv_bfloat16*>(b);
      const bool weight = (pb >= Pb && pb < Pb + np_all) || (pb >= PbT && pb < PbT + np_all);
      g.gs = gstride;
      if (weight) {
        EDPC_TRY(make_tmap_bf16_groups(&g.tb, b, b_rows, b_cols, b_ld, ngroups, gstride, box_b));
        g.mt = gtiles;
        g.nmt = ngtiles;
      } else {
        g.gk = gkr;
        g.ngk = ngroups;
      }
    }
    return EDPC_OK;
  };
  const int b = d.b, F = d.F, H = d.H, Fp = d.Fp;
  for (int j = 0; j < d.n; ++j) {
    const BlockOff& o = po.blk[j];
    BlockBf16& q = bb[j];
    // Eqs. 10-12: branch GEMM, B loaded as k sections of 32 hidden units
    {
      int id = blk_site(BR_FWD, j);
      // hidden units per branch section: 32 * code, halved until the k sections fit one MMA
      int sw = (tile_code[id] & 15) ? 32 * (tile_code[id] & 15) : (big ? 64 : 32);
      while (sw > 32 && (sw > 128 || sw * d.k > 256)) sw /= 2;
      EDPC_TRY(site(id, b, kH, F, q.X0b, b, F, F, Pb + o.W, kH, F, F, sw * d.k, sw));
      TcGemm& g = tcp.site[id];
      g.mode = TC_BRANCH;
      g.H = H;
      g.k = d.k;
      g.C = ba[j].A;
      g.ldc = kH;
      g.Cb = q.Gb;
      g.ldcb = H;
      g.CbT = q.GbT;
      g.ldct = T;
      g.bias = P + o.c;
    }
    // Eq. 13: out GEMM + residual (the output's BF16 copies when a GEMM reads it next)
    {
      int id = blk_site(OUT_FWD, j);
      int bn = bn_rows(id, F);
      EDPC_TRY(site(id, b, F, H, q.Gb, b, H, H, Pb + o.Wo, F, H, H, bn, bn));
      TcGemm& g = tcp.site[id];
      int out = (j < d.nloc) ? j + 1 : j + 2;
      int in = (j < d.nloc) ? j : j + 1;
      g.C = S[out];
      g.ldc = F;
      g.bias = P + o.co;
      g.R = S[in];
      g.ldr = F;
      if (j == d.nloc - 1) {
        g.Cb = Slte_b;
        g.ldcb = F;
        g.CbT = Slte_bT;
        g.ldct = T;
      } else if (j == d.n - 1) {
        g.Cb = Shead_b;
        g.ldcb = F;
        g.CbT = Shead_bT;
        g.ldct = T;
      }
    }
    // adjoint of Eq. 13 w.r.t. G, fused with the adjoint of Eqs. 11-12
    {
      int id = blk_site(OUT_DX, j);
      const int bn = (tile_code[id] & 15) ? std::min(128, 32 * (tile_code[id] & 15)) : (big ? 128 : 32);
      EDPC_TRY(site(id, b, H, F, q.dOutb, b, F, F, PbT + o.Wo, H, F, F, bn, bn));
      TcGemm& g = tcp.site[id];
      g.mode = TC_BRANCH_BWD;
      g.H = H;
      g.k = d.k;
      g.C = q.dA;
      g.ldc = kH;
      g.Cb = q.dAb;
      g.ldcb = kH;
      g.CbT = q.dAbT;
      g.ldct = T;
      g.Aux = ba[j].A;
      g.ldaux = kH;
    }
    {  // dWo = dOut^T G
      int id = blk_site(OUT_DW, j);
      int bn = bn_dw(id, H);
      EDPC_TRY(site(id, F, H, b, q.dOutbT, F, b, T, q.GbT, H, b, T, bn, bn));
      TcGemm& g = tcp.site[id];
      g.C = G + o.Wo;
      g.ldc = H;
      EDPC_TRY(split_site(id));
    }
    {  // dX0 = dA W
      int id = blk_site(BR_DX, j);
      int bn = bn_rows(id, F);
      EDPC_TRY(site(id, b, F, kH, q.dAb, b, kH, kH, PbT + o.W, F, kH, kH, bn, bn));
      TcGemm& g = tcp.site[id];
      g.C = q.dX0;
      g.ldc = F;
    }
    {  // dW = dA^T X0
      int id = blk_site(BR_DW, j);
      int bn = bn_dw(id, F);
      EDPC_TRY(site(id, kH, F, b, q.dAbT, kH, b, T, q.X0bT, F, b, T, bn, bn));
      TcGemm& g = tcp.site[id];
      g.C = G + o.W;
      g.ldc = F;
      EDPC_TRY(split_site(id));
    }
  }
  if (d.lte) {  // Eq. 14
    int bn = bn_rows(kSiteLteDownFwd, Fp);
    EDPC_TRY(site(kSiteLteDownFwd, b, Fp, F, Slte_b, b, F, F, Pb + po.W1, Fp, F, F, bn, bn));
    TcGemm& g = tcp.site[kSiteLteDownFwd];
    g.C = Xp;
    g.ldc = Fp;
    g.bias = P + po.b1;
  }
  if (d.lte) {  // Eq. 16
    int bn = bn_rows(kSiteLteUpFwd, F);
    EDPC_TRY(site(kSiteLteUpFwd, b, F, Fp, Yb, b, Fp, Fp, Pb + po.W2, F, Fp, Fp, bn, bn));
    TcGemm& g = tcp.site[kSiteLteUpFwd];
    g.C = S[d.nloc + 1];
    g.ldc = F;
    g.bias = P + po.b2;
  }
  {  // head
    const int bh = (tile_code[kSiteHeadFwd] & 15) ? 32 * (tile_code[kSiteHeadFwd] & 15) : 64;
    EDPC_TRY(site(kSiteHeadFwd, b, 256, F, Shead_b, b, F, F, Pb + po.Wh, 256, F, F, bh, bh));
    TcGemm& g = tcp.site[kSiteHeadFwd];
    g.C = z;
    g.ldc = 256;
    g.bias = P + po.bh;
  }
  {  // head adjoint: dX = dz Wh -> gradient of the last block's output
    int bn = bn_rows(kSiteHeadDx, F);
    EDPC_TRY(site(kSiteHeadDx, b, F, 256, dzb, b, 256, 256, PbT + po.Wh, F, 256, 256, bn, bn));
    TcGemm& g = tcp.site[kSiteHeadDx];
    BlockBf16& q = bb[d.n - 1];
    g.C = q.dOut;
    g.ldc = F;
    g.Cb = q.dOutb;
    g.ldcb = F;
    g.CbT = q.dOutbT;
    g.ldct = T;
  }
  {  // dWh = dz^T X
    int bn = bn_dw(kSiteHeadDw, F);
    EDPC_TRY(site(kSiteHeadDw, 256, F, b, dzbT, 256, b, T, Shead_bT, F, b, T, bn, bn));
    TcGemm& g = tcp.site[kSiteHeadDw];
    g.C = G + po.Wh;
    g.ldc = F;
    EDPC_TRY(split_site(kSiteHeadDw));
  }
  if (d.lte) {  // LTE up adjoint: dY = dX W2
    int bn = bn_rows(kSiteLteUpDx, Fp);
    EDPC_TRY(site(kSiteLteUpDx, b, Fp, F, dLteb, b, F, F, PbT + po.W2, Fp, F, F, bn, bn));
    TcGemm& g = tcp.site[kSiteLteUpDx];
    g.C = dY;
    g.ldc = Fp;
  }
  if (d.lte) {  // dW2 = dX^T Y
    int bn = bn_dw(kSiteLteUpDw, Fp);
    EDPC_TRY(site(kSiteLteUpDw, F, Fp, b, dLtebT, F, b, T, YbT, Fp, b, T, bn, bn));
    TcGemm& g = tcp.site[kSiteLteUpDw];
    g.C = G + po.W2;
    g.ldc = Fp;
    EDPC_TRY(split_site(kSiteLteUpDw));
  }
  if (d.lte) {  // LTE down adjoint: dX = dX' W1 -> gradient of the last Local block's output
    int bn = bn_rows(kSiteLteDownDx, F);
    EDPC_TRY(site(kSiteLteDownDx, b, F, Fp, dXpb, b, Fp, Fp, PbT + po.W1, F, Fp, Fp, bn, bn));
    TcGemm& g = tcp.site[kSiteLteDownDx];
    g.ldc = F;
    if (d.nloc > 0) {
      BlockBf16& q = bb[d.nloc - 1];
      g.C = q.dOut;
      g.Cb = q.dOutb;
      g.ldcb = F;
      g.CbT = q.dOutbT;
      g.ldct = T;
    } else {
      g.C = dh0;
    }
  }
  if (d.lte) {  // dW1 = dX'^T X
    int bn = bn_dw(kSiteLteDownDw, F);
    EDPC_TRY(site(kSiteLteDownDw, Fp, F, b, dXpbT, Fp, b, T, Slte_bT, F, b, T, bn, bn));
    TcGemm& g = tcp.site[kSiteLteDownDw];
    g.C = G + po.W1;
    g.ldc = F;
    EDPC_TRY(split_site(kSiteLteDownDw));
  }
  // output tensor maps of every site (after its outputs and split-K factor are set)
  for (int id = 0; id < TcPlan::kMaxSites; ++id)
    if (tcp.site[id].M > 0) EDPC_TRY(tc_build_out_maps(&tcp.site[id]));
  tcp.ready = true;
  return EDPC_OK;
}

void Model::tunable_sites(std::vector<int>* ids) const {
  ids->clear();
  for (int kind : {BR_FWD, OUT_FWD, OUT_DX, OUT_DW, BR_DX, BR_DW})
    for (int j = 0; j < d.n; ++j) ids->push_back(blk_site(kind, j));
  for (int id = kSiteLteDownFwd; id <= kSiteLteDownDx; ++id)
    if (d.lte || id == kSiteHeadFwd || id == kSiteHeadDx || id == kSiteHeadDw) ids->push_back(id);
}

// Tile codes: 0 (size heuristic), or w + v with w in {1, 2, 4, 8} and v in
// {0, 16}. The N tile (for the fused branch GEMM: the section of hidden units
// per branch) is 32 * w, capped at the widest the site supports (128 for the
// branch adjoint; k sections of at most 128 within 256 columns for the branch
// GEMM). v selects the kernel: 0 one tile per CTA, 16 persistent. Both kernels
// give the same results for the same tile. (Codes with v = 48 or 80 named
// kernels that are no longer built; containers that carry them are refused.)
bool Model::tile_code_ok(int, uint8_t c) const {
  if (c == 0) return true;
  const int w = c & 15, v = c >> 4;
  if (w != 1 && w != 2 && w != 4 && w != 8) return false;
  return v == 0 || v == 1;
}

int Model::set_tiles(const uint8_t* code, int n) {
  if (precision == EDPC_FP32) return EDPC_OK;
  if (ngroups) return fail(EDPC_EINVAL, "independent models in one batch use the size-heuristic tiles");
  // validate every code before any is taken, so a refused set leaves the plan as it was
  for (int i = 0; i < TcPlan::kMaxSites; ++i) {
    const uint8_t c = (code && i < n) ? code[i] : 0;
    if (!tile_code_ok(i, c)) return fail(EDPC_EARCH, "unknown GEMM tile code " + std::to_string(c));
  }
  for (int i = 0; i < TcPlan::kMaxSites; ++i) tile_code[i] = (code && i < n) ? code[i] : 0;
  return build_tc_plan();
}

// Autotuner for the GEMM N tiles: every tcgen05 site of the step (but the head
// GEMM) is timed with each tile code it accepts (N tiles of 32 to 256; branch
// sections of 32 to 128) with CUDA events, after a warm-up launch, on the
// model's own buffers, and keeps the fastest. Runs before the first step: the
// GEMMs only overwrite per-step outputs (activations, BF16 copies, gradients).
int Model::tune_tiles(cudaStream_t st) {
  if (precision == EDPC_FP32 || ngroups) return EDPC_OK;
  std::vector<int> ids;
  tunable_sites(&ids);
  cudaEvent_t e0, e1;
  EDPC_CUDA(cudaEventCreate(&e0));
  EDPC_CUDA(cudaEventCreate(&e1));
  int r = EDPC_OK;
  const int reps = 4;
  for (int id : ids) {
    float best = 1e30f;
    uint8_t best_code = 1;
    int seen[16] = {}, nseen = 0;
    static const uint8_t kCodes[] = {1, 2, 4, 8, 17, 18, 20, 24};
    for (uint8_t code : kCodes) {
      if (!tile_code_ok(id, code)) continue;
      tile_code[id] = code;
      if ((r = build_tc_plan()) != EDPC_OK) break;
      // a capped code repeats a (tile, kernel) pair already timed
      const int key = tcp.site[id].bn * 16 + (tcp.site[id].persistent ? 8 : 0);
      bool dup = false;
      for (int q = 0; q < nseen; ++q) dup |= seen[q] == key;
      if (dup) continue;
      seen[nseen++] = key;
      NoPdl scope;
      cudaError_t e = launch_gemm_tc(tcp.site[id], st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int q = 0; q < reps && e == cudaSuccess; ++q) e = launch_gemm_tc(tcp.site[id], st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        r = fail(EDPC_ECUDA, std::string("GEMM tile tuning: ") + cudaGetErrorString(e));
        break;
      }
      if (ms < best) {
        best = ms;
        best_code = code;
      }
    }
    if (r != EDPC_OK) break;
    tile_code[id] = best_code;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != EDPC_OK) return r;
  return build_tc_plan();
}

int Model::time_sites(cudaStream_t st, int reps, double* ms, double* flop, double* bytes, int cap) {
  if (precision == EDPC_FP32 || !tcp.ready) return fail(EDPC_EINVAL, "no tcgen05 GEMM sites (FP32 model)");
  if (reps < 1) reps = 1;
  cudaEvent_t e0, e1;
  EDPC_CUDA(cudaEventCreate(&e0));
  EDPC_CUDA(cudaEventCreate(&e1));
  int r = EDPC_OK;
  for (int id = 0; id < TcPlan::kMaxSites && id < cap; ++id) {
    const TcGemm& g = tcp.site[id];
    ms[id] = 0;
    flop[id] = 0;
    if (bytes) bytes[id] = 0;
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) continue;
    NoPdl scope;
    // (FP8: the operands' e4m3 shadows are timed as they stand; values do not change the time)
    cudaError_t e = launch_gemm_tc(g, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int q = 0; q < reps && e == cudaSuccess; ++q) e = launch_gemm_tc(g, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) {
      r = fail(EDPC_ECUDA, std::string("GEMM site timing: ") + cudaGetErrorString(e));
      break;
    }
    ms[id] = t / reps;
    flop[id] = 2.0 * g.M * g.N * g.K;
    if (bytes) {
      // compulsory traffic: operands read once, epilogue inputs read once, outputs written once
      const double M = g.M, es = g.fp8 ? 1.0 : 2.0, kH = (double)g.k * g.H;
      const double wc = g.mode == TC_PLAIN ? g.N : kH, wcb = g.mode == TC_PLAIN ? g.N : (g.mode == TC_BRANCH ? g.H : kH);
      double by = (M + g.N) * g.K * es;
      if (g.C) by += M * wc * 4;
      if (g.Cb) by += M * wcb * 2;
      if (g.CbT) by += M * wcb * 2;
      if (g.R) by += M * g.N * 4;
      if (g.Aux) by += M * kH * 4;
      bytes[id] = by;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

int Model::run_tc(int site, cudaStream_t st) {
  if (st == side) {
    NoPdl scope;
    if (precision == EDPC_FP8E4M3) EDPC_TRY(quantize_site(site, st));
    EDPC_CUDA(launch_gemm_tc(plan().site[site], st));
  } else {
    if (precision == EDPC_FP8E4M3) EDPC_TRY(quantize_site(site, st));
    EDPC_CUDA(launch_gemm_tc(plan().site[site], st));
  }
  return EDPC_OK;
}

int Model::colsums(ColsumJobs cj, cudaStream_t st) {
  NoPdl scope;
  if (ngroups) {  // each group's own rows into its own gradient
    EDPC_CUDA(launch_colsum_groups(cj, ginfo, ngroups, gstride, st));
    return EDPC_OK;
  }
  cj.chunk_rows = colsum_chunk_rows(d.b, colsum_tiles(cj));
  if (cj.chunk_rows > 0) {
    const int tw = colsum_vec(cj) ? 128 : 32;
    if (colsum_tiles(cj) > cs_tiles || colsum_tiles(cj) * tw > cs_cols)
      return fail(EDPC_EINVAL, "column-sum launch exceeds its scratch");
    cj.part = cs_part;
    cj.cnt = cs_cnt;
  }
  EDPC_CUDA(launch_colsum_multi(cj, st));
  return EDPC_OK;
}

int Model::fork_side(cudaStream_t st) {
  if (nfork_ >= kForks) return fail(EDPC_EINVAL, "too many side-stream forks in one step");
  cudaEvent_t e = fork[nfork_++];
  EDPC_CUDA(cudaEventRecord(e, st));
  EDPC_CUDA(cudaStreamWaitEvent(side, e, 0));
  return EDPC_OK;
}

int Model::forward_bf16(const StepIO& io, cudaStream_t st) {
  nfork_ = 0;
  const bool f8m = precision == EDPC_FP8E4M3;
  if (f8m) {
    std::fill(f8_done.begin(), f8_done.end(), 0);
    EDPC_CUDA(launch_zero_u32(f8_amax, (int)f8.size(), st));  // this step's amax slots
  }
  // Transposed BF16 weight copies for this step's dX GEMMs, from the weights the
  // previous Adam wrote, on the side stream while the forward pass runs.
  EDPC_TRY(fork_side(st));
  {
    NoPdl scope;
    EDPC_CUDA(launch_transpose_tiles(Pb, PbT, tiles, ntiles, side));
    if (f8m) EDPC_TRY(quantize_weights(true, side));
  }
  EDPC_CUDA(cudaEventRecord(tr_ev, side));
  if (f8m) EDPC_TRY(quantize_weights(false, st));
  // the embedding, fused with the first block's LayerNorm when a Local block follows it
  const bool fuse0 = d.nloc > 0 && (d.F == 128 || d.F == 256 || d.F == 512 || d.F == 1024);
  if (fuse0) {
    const BlockOff& o = po.blk[0];
    EDPC_CUDA(launch_embed_ln_bf16(io.mode == 2 ? nullptr : io.data, io.sp, ctl, P + po.E, d.b, d.K, d.D, S[0], ctx,
                                   P + o.ln_g, P + o.ln_b, ba[0].xhat, ba[0].rstd, bb[0].X0b, bb[0].X0bT, d.ldT, st,
                                   row_grp, gstride));  // Eq. 9 of block 0
  } else {
    EDPC_CUDA(launch_embed(io.mode == 2 ? nullptr : io.data, io.sp, ctl, P + po.E, d.b, d.K, d.D, S[0], ctx, st,
                           row_grp, gstride));
  }
  if (d.nloc == 0) EDPC_CUDA(launch_to_bf16(S[0], d.b, d.F, d.F, Slte_b, d.F, Slte_bT, d.ldT, st));
  for (int jj = 0; jj < d.n; ++jj) {
    if (jj == d.nloc) {
      if (d.lte) EDPC_TRY(run_tc(kSiteLteDownFwd, st));  // Eq. 14
      EDPC_TRY(fdm_fwd_call(io, st));                      // Eq. 15 (w/o LTE: on S[nloc] into S[nloc + 1])
      if (d.lte) EDPC_TRY(run_tc(kSiteLteUpFwd, st));    // Eq. 16
    }
    const BlockOff& o = po.blk[jj];
    const float* Xin = S[jj < d.nloc ? jj : jj + 1];
    if (!(jj == 0 && fuse0))
      EDPC_CUDA(launch_ln_fwd_bf16(Xin, P + o.ln_g, P + o.ln_b, ba[jj].xhat, ba[jj].rstd, bb[jj].X0b, bb[jj].X0bT,
                                   d.b, d.F, d.ldT, st, row_grp, gstride));  // Eq. 9
    EDPC_TRY(run_tc(blk_site(BR_FWD, jj), st));         // Eqs. 10-12
    EDPC_TRY(run_tc(blk_site(OUT_FWD, jj), st));        // Eq. 13
  }
  EDPC_TRY(run_tc(kSiteHeadFwd, st));
  return EDPC_OK;
}

int Model::fdm_bwd_joined(const StepIO& io, cudaStream_t st) {
  if (d.b < 2048) return fdm_bwd_call(io, st);
  // From 2048 streams on the FDM adjoint (milliseconds of HBM-bound
  // streaming) runs faster alone than beside the side stream's pending
  // weight gradients, so it waits for them (measured: 6.63 -> 5.81 ms per
  // step at 4096 streams; at 512 streams the overlap wins).
  EDPC_CUDA(cudaEventRecord(fdm_join_ev, side));
  EDPC_CUDA(cudaStreamWaitEvent(st, fdm_join_ev, 0));
  NoPdl scope;  // two incoming dependencies
  return fdm_bwd_call(io, st);
}

int Model::backward_bf16(const StepIO& io, cudaStream_t st) {
  const int kH = d.k * d.H;
  // PbT is read by the dX GEMMs below (delayed update: this parity's copies
  // were made during the previous step)
  if (!delayed) EDPC_CUDA(cudaStreamWaitEvent(st, tr_ev, 0));
  // side: head weight gradients
  EDPC_TRY(fork_side(st));
  EDPC_TRY(run_tc(kSiteHeadDw, side));
  {
    ColsumJobs cj{};
    cj.job[0] = {dz, nullptr, d.b, 256, 256, G + po.bh};
    cj.n = 1;
    EDPC_TRY(colsums(cj, side));
  }
  {
    NoPdl scope;  // the stream also waits on the transposes' event
    EDPC_TRY(run_tc(kSiteHeadDx, st));  // dOut of the last block
  }
  for (int j = d.n - 1; j >= 0; --j) {
    const BlockOff& o = po.blk[j];
    BlockBf16& q = bb[j];
    if (j == d.nloc - 1 && !d.lte) EDPC_TRY(fdm_bwd_joined(io, st));  // w/o LTE: the FDM alone
    if (j == d.nloc - 1 && d.lte) {
      // LTE (Eqs. 14-16) between the Global and the Local blocks
      EDPC_TRY(fork_side(st));
      EDPC_TRY(run_tc(kSiteLteUpDw, side));
      ColsumJobs cj{};
      cj.job[0] = {dLte, nullptr, d.b, d.F, d.F, G + po.b2};
      cj.n = 1;
      EDPC_TRY(colsums(cj, side));
      EDPC_TRY(run_tc(kSiteLteUpDx, st));
      EDPC_TRY(fdm_bwd_joined(io, st));
      EDPC_TRY(fork_side(st));
      EDPC_TRY(run_tc(kSiteLteDownDw, side));
      ColsumJobs cj2{};
      cj2.job[0] = {dXp, nullptr, d.b, d.Fp, d.Fp, G + po.b1};
      cj2.n = 1;
      EDPC_TRY(colsums(cj2, side));
      EDPC_TRY(run_tc(kSiteLteDownDx, st));
    }
    EDPC_TRY(fork_side(st));  // dOut_j is ready
    EDPC_TRY(run_tc(blk_site(OUT_DW, j), side));
    EDPC_TRY(run_tc(blk_site(OUT_DX, j), st));  // dA (adjoint of Eqs. 11-13)
    EDPC_TRY(fork_side(st));
    EDPC_TRY(run_tc(blk_site(BR_DW, j), side));
    EDPC_TRY(run_tc(blk_site(BR_DX, j), st));  // dX0 (adjoint of Eq. 10)
    EDPC_TRY(fork_side(st));
    {
      ColsumJobs cj{};
      cj.job[0] = {q.dOut, nullptr, d.b, d.F, d.F, G + o.co};
      cj.job[1] = {q.dA, nullptr, d.b, kH, kH, G + o.c};
      cj.job[2] = {q.dX0, ba[j].xhat, d.b, d.F, d.F, G + o.ln_g};
      cj.job[3] = {q.dX0, nullptr, d.b, d.F, d.F, G + o.ln_b};
      cj.n = 4;
      EDPC_TRY(colsums(cj, side));
    }
    // LN adjoint (Eq. 9) + residual path: gradient of the block input
    float* out;
    __nv_bfloat16 *outb = nullptr, *outbT = nullptr;
    if (j == d.nloc) {
      out = dLte;
      outb = dLteb;
      outbT = dLtebT;
    } else if (j == 0) {
      out = dh0;
    } else {
      out = bb[j - 1].dOut;
      outb = bb[j - 1].dOutb;
      outbT = bb[j - 1].dOutbT;
    }
    EDPC_CUDA(launch_ln_bwd_bf16(q.dX0, ba[j].xhat, ba[j].rstd, P + o.ln_g, q.dOut, out, outb, outbT, d.b, d.F,
                                 d.ldT, st, row_grp, gstride));
  }
  if (d.nloc == 0 && !d.lte) EDPC_TRY(fdm_bwd_joined(io, st));  // w/o LTE: writes dh0
  if (d.nloc == 0 && d.lte) {
    // LTE before any Local block: its adjoint runs after the Global blocks.
    EDPC_TRY(fork_side(st));
    EDPC_TRY(run_tc(kSiteLteUpDw, side));
    ColsumJobs cj{};
    cj.job[0] = {dLte, nullptr, d.b, d.F, d.F, G + po.b2};
    cj.n = 1;
    EDPC_TRY(colsums(cj, side));
    EDPC_TRY(run_tc(kSiteLteUpDx, st));
    EDPC_TRY(fdm_bwd_call(io, st));
    EDPC_TRY(fork_side(st));
    EDPC_TRY(run_tc(kSiteLteDownDw, side));
    ColsumJobs cj2{};
    cj2.job[0] = {dXp, nullptr, d.b, d.Fp, d.Fp, G + po.b1};
    cj2.n = 1;
    EDPC_TRY(colsums(cj2, side));
    EDPC_TRY(run_tc(kSiteLteDownDx, st));  // writes dh0
  }
  if (ngroups)
    EDPC_CUDA(launch_embed_bwd_groups(ctx, dh0, d.K, d.D, G + po.E, ginfo, ngroups, gstride, st));
  else
    EDPC_CUDA(launch_embed_bwd(ctx, dh0, d.b, d.K, d.D, G + po.E, emb_part, emb_cnt, st));
  // join the side stream
  EDPC_CUDA(cudaEventRecord(join_ev, side));
  EDPC_CUDA(cudaStreamWaitEvent(st, join_ev, 0));
  return EDPC_OK;
}

// ==========================================================================================
// step
// ==========================================================================================
int Model::forward(const StepIO& io, cudaStream_t st) {
  return precision != EDPC_FP32 ? forward_bf16(io, st) : forward_f32(io, st);
}

int Model::head(const StepIO& io, cudaStream_t st) {
  HeadArgs h{};
  h.z = z;
  h.b = d.b;
  h.ctl = ctl;
  h.sp = io.sp;
  h.mode = io.mode;
  h.data = io.data;
  h.targets = io.targets;
  h.active = io.active;
  h.p = p;
  h.dz = dz;
  h.ring = io.ring;
  h.dec = io.dec;
  h.bits = io.bits;
  h.bits_off = io.bits_off;
  h.bits_len = io.bits_len;
  h.dzb = dzb;
  h.dzbT = dzbT;
  h.ldT = d.ldT;
  h.err = &ctl->err;
  h.rg = row_grp;
  h.gi = ginfo;
  EDPC_CUDA(launch_head(h, st));
  return EDPC_OK;
}

int Model::backward(const StepIO& io, cudaStream_t st) {
  return precision != EDPC_FP32 ? backward_bf16(io, st) : backward_f32(io, st);
}

int Model::adam(cudaStream_t st) {
  if (precision != EDPC_FP32) {
    NoPdl scope;  // follows the join of the side stream
    EDPC_CUDA(launch_adam_bf16(P, G, M, V, Pb, np_all, ctl, st));
  } else {
    EDPC_CUDA(launch_adam(P, G, M, V, nparam, ctl, st));
  }
  return EDPC_OK;
}

int Model::step(const StepIO& io, cudaStream_t st) {
  if (delayed) return step_delayed(io, st);
  EDPC_TRY(forward(io, st));
  EDPC_TRY(head(io, st));
  EDPC_TRY(backward(io, st));
  if (io.update) EDPC_TRY(adam(st));
  if (io.advance) EDPC_CUDA(launch_step_advance(ctl, io.sp, d.K, io.ring_slots, d.b, st));
  return EDPC_OK;
}

// Step s of the delayed-update schedule (parity q = s % 2): the forward pass
// and the head of step s on st with parity q; beside them, on bwd_st, the
// adjoint of step s - 1 with parity q ^ 1 (its FDM update, launched on
// side_fdm, writes the FDMs of step s + 1, from those of step s, over parity
// q ^ 1's; the FDM forward of step s + 1 waits for it); then, after both,
// Adam writes the parameters of step s + 1 into parity q ^ 1 from parity q's
// and the gradient of step s - 1, with step s - 1's Adam counter.
int Model::step_delayed(const StepIO& io, cudaStream_t st) {
  const int q = io.tick & 1;
  EDPC_CUDA(cudaEventRecord(tick_ev, st));  // after the previous step's Adam and step control
  EDPC_CUDA(cudaStreamWaitEvent(bwd_st, tick_ev, 0));
  select(q);
  EDPC_TRY(forward(io, st));
  EDPC_TRY(head(io, st));
  select(q ^ 1);
  if (precision == EDPC_FP32) {
    NoPdl scope;  // the first launch on bwd_st follows a cross-stream wait
    EDPC_TRY(backward(io, bwd_st));
  } else {
    EDPC_TRY(backward(io, bwd_st));  // its first launch on bwd_st is made without PDL
  }
  EDPC_CUDA(cudaEventRecord(bwd_ev, bwd_st));
  EDPC_CUDA(cudaStreamWaitEvent(st, bwd_ev, 0));
  const Parity& now = par[q];
  const Parity& nxt = par[q ^ 1];
  if (io.update) {
    NoPdl scope;  // follows the join of bwd_st
    if (precision != EDPC_FP32)
      EDPC_CUDA(launch_adam_bf16(nxt.P, G, M, V, nxt.Pb, nparam, nxt.ctl, st, now.P));
    else
      EDPC_CUDA(launch_adam(nxt.P, G, M, V, nparam, nxt.ctl, st, now.P));
  }
  if (io.advance) EDPC_CUDA(launch_step_advance(now.ctl, io.sp, d.K, io.ring_slots, d.b, st, nxt.ctl));
  select(q ^ 1);
  return EDPC_OK;
}

int Model::launches_per_step() const {
  if (precision != EDPC_FP32) {
    // forward: embed (with block 0's LN) + 3 per block (2 for block 0) + LTE (2 GEMMs + FDM) + head GEMM + head
    int n = 1 + 3 * d.n - (d.nloc > 0 ? 1 : 0) + 3 + 1 + 1;
    // backward: head dW/colsum/dX, per block 3 main + 3 side, LTE 3 + 2 side ... + embed
    n += 3 + 6 * d.n + 3 + 4 + 1;
    return n + 3;  // adam, transpose, advance
  }
  int n = 1 + 4 * d.n + 3 + 1 + 1;
  n += 3 + 10 * d.n + 3 + 1 + 3 + 1;
  return n + 2;
}

}  // namespace edpc
