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
#include <cmath>
#include <cstring>

#include "engine.cuh"

namespace edpc {

Dims make_dims(const edpc_cfg& c, int b) {
  Dims d;
  d.b = b;
  d.K = (int)c.context;
  d.D = (int)c.embed_dim;
  d.F = d.K * d.D;
  d.Fp = (int)c.latent;
  d.H = (int)c.hidden;
  d.n = (int)c.blocks;
  d.nloc = d.n / 2;
  d.k = (int)c.branches;
  d.ldT = (int)round_up(b, 8);
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
  o.W1 = take((size_t)d.Fp * d.F);
  o.b1 = take(d.Fp);
  o.W2 = take((size_t)d.F * d.Fp);
  o.b2 = take(d.F);
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
  if (gU) cudaFree(gU);
  if (arena_) cudaFree(arena_);
}

int Model::init(const edpc_cfg& cfg, int streams) {
  d = make_dims(cfg, streams);
  po = make_offsets(d);
  precision = cfg.precision;
  seed = cfg.seed;
  lr = cfg.lr;
  nparam = po.total;
  const size_t bF = (size_t)d.b * d.F, bFp = (size_t)d.b * d.Fp, bH = (size_t)d.b * d.H;
  const size_t bkH = (size_t)d.b * d.k * d.H, fdm = (size_t)d.b * d.Fp * d.Fp;
  const bool bf16 = precision == EDPC_BF16;
  // Largest activation operand copies (row-major b x max and transposed max x ldT).
  const int maxw = std::max(std::max(d.F, d.k * d.H), std::max(256, d.Fp));

  for (int pass = 0; pass < 2; ++pass) {
    Arena a;
    a.base = static_cast<char*>(arena_);
    P = a.take<float>(nparam);
    G = a.take<float>(nparam);
    M = a.take<float>(nparam);
    V = a.take<float>(nparam);
    U = a.take<float>(fdm);
    Um = a.take<float>(fdm);
    Uv = a.take<float>(fdm);
    ctl = a.take<StepCtl>(1);
    ctx = a.take<uint8_t>((size_t)d.b * d.K);
    for (int s = 0; s < d.n + 2; ++s) S[s] = a.take<float>(bF);
    for (int j = 0; j < d.n; ++j) {
      ba[j].xhat = a.take<float>(bF);
      ba[j].rstd = a.take<float>(d.b);
      ba[j].X0 = a.take<float>(bF);
      ba[j].A = a.take<float>(bkH);
      ba[j].G = a.take<float>(bH);
    }
    Xp = a.take<float>(bFp);
    Y = a.take<float>(bFp);
    z = a.take<float>((size_t)d.b * 256);
    p = a.take<float>((size_t)d.b * 256);
    dz = a.take<float>((size_t)d.b * 256);
    dXa = a.take<float>(bF);
    dXb = a.take<float>(bF);
    dX0 = a.take<float>(bF);
    dA = a.take<float>(bkH);
    dG = a.take<float>(bH);
    dY = a.take<float>(bFp);
    dXp = a.take<float>(bFp);
    if (bf16) {
      Pb = a.take<__nv_bfloat16>(nparam);
      PbT = a.take<__nv_bfloat16>(nparam);
      xa = a.take<__nv_bfloat16>((size_t)d.b * maxw);
      xb = a.take<__nv_bfloat16>((size_t)d.b * maxw);
      xaT = a.take<__nv_bfloat16>((size_t)d.ldT * maxw);
      xbT = a.take<__nv_bfloat16>((size_t)d.ldT * maxw);
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
  cudaStream_t st = 0;
  // Initial values (counter-based SplitMix64 rule, tensor id = canonical order).
  const double F = d.F, H = d.H, Fp = d.Fp;
  struct T {
    size_t off, n;
    float bound;
    float fill;
  };
  std::vector<T> ts;
  ts.push_back({po.E, (size_t)256 * d.D, (float)std::sqrt(3.0), 0.f});
  for (int j = 0; j < d.n; ++j) {
    const BlockOff& b = po.blk[j];
    ts.push_back({b.ln_g, (size_t)d.F, -1.f, 1.f});
    ts.push_back({b.ln_b, (size_t)d.F, -1.f, 0.f});
    ts.push_back({b.W, (size_t)d.k * d.H * d.F, (float)(1.0 / std::sqrt(F)), 0.f});
    ts.push_back({b.c, (size_t)d.k * d.H, (float)(1.0 / std::sqrt(F)), 0.f});
    ts.push_back({b.Wo, (size_t)d.F * d.H, (float)(1.0 / std::sqrt(H)), 0.f});
    ts.push_back({b.co, (size_t)d.F, (float)(1.0 / std::sqrt(H)), 0.f});
  }
  ts.push_back({po.W1, (size_t)d.Fp * d.F, (float)(1.0 / std::sqrt(F)), 0.f});
  ts.push_back({po.b1, (size_t)d.Fp, (float)(1.0 / std::sqrt(F)), 0.f});
  ts.push_back({po.W2, (size_t)d.F * d.Fp, (float)(1.0 / std::sqrt(Fp)), 0.f});
  ts.push_back({po.b2, (size_t)d.F, (float)(1.0 / std::sqrt(Fp)), 0.f});
  ts.push_back({po.Wh, (size_t)256 * d.F, (float)(1.0 / std::sqrt(F)), 0.f});
  ts.push_back({po.bh, (size_t)256, (float)(1.0 / std::sqrt(F)), 0.f});
  for (size_t tid = 0; tid < ts.size(); ++tid)
    EDPC_CUDA(launch_init_values(P + ts[tid].off, ts[tid].n, seed, (int)tid, ts[tid].bound, 0, ts[tid].fill, st));
  EDPC_CUDA(launch_init_values(U, fdm, seed, kFdmTid, (float)std::sqrt(3.0 / Fp), 0, 0.f, st));
  EDPC_CUDA(cudaMemsetAsync(M, 0, nparam * sizeof(float), st));
  EDPC_CUDA(cudaMemsetAsync(V, 0, nparam * sizeof(float), st));
  EDPC_CUDA(cudaMemsetAsync(G, 0, nparam * sizeof(float), st));
  EDPC_CUDA(cudaMemsetAsync(Um, 0, fdm * sizeof(float), st));
  EDPC_CUDA(cudaMemsetAsync(Uv, 0, fdm * sizeof(float), st));
  if (bf16) {
    EDPC_CUDA(cudaMemsetAsync(xaT, 0, (size_t)d.ldT * maxw * 2, st));
    EDPC_CUDA(cudaMemsetAsync(xbT, 0, (size_t)d.ldT * maxw * 2, st));
    EDPC_TRY(refresh_bf16_weights(st));
    EDPC_TRY(build_tc_plan());
  }
  EDPC_CUDA(cudaStreamSynchronize(st));
  return EDPC_OK;
}

int Model::set_ctl_for_step(int i, int t, int bact, int ring_slots, cudaStream_t st) {
  int slot = ring_slots > 0 ? (int)(((long long)i - d.K) % ring_slots) : 0;
  if (slot < 0) slot = 0;
  set_ctl_kernel<<<1, 1, 0, st>>>(ctl, i, t, bact, slot, lr);
  EDPC_CUDA(cudaGetLastError());
  return EDPC_OK;
}

// ------------------------------------------------------------------------------------------
// BF16: weight copies and the tensor-map plan
// ------------------------------------------------------------------------------------------
int Model::refresh_bf16_weights(cudaStream_t st) {
  auto mat = [&](size_t off, int rows, int cols) -> cudaError_t {
    return launch_to_bf16(P + off, rows, cols, cols, Pb + off, cols, PbT + off, rows, st);
  };
  for (int j = 0; j < d.n; ++j) {
    EDPC_CUDA(mat(po.blk[j].W, d.k * d.H, d.F));
    EDPC_CUDA(mat(po.blk[j].Wo, d.F, d.H));
  }
  EDPC_CUDA(mat(po.W1, d.Fp, d.F));
  EDPC_CUDA(mat(po.W2, d.F, d.Fp));
  EDPC_CUDA(mat(po.Wh, 256, d.F));
  return EDPC_OK;
}

static int pick_bn(int N) { return N <= 128 ? 64 : (N <= 512 ? 64 : 128); }

int Model::build_tc_plan() {
  auto fwd = [&](int site, int in, size_t w_off, int out) -> int {
    TcGemm& g = tc.site[site];
    g.M = d.b;
    g.N = out;
    g.K = in;
    g.bn = pick_bn(out);
    EDPC_TRY(make_tmap_bf16(&g.ta, xa, d.b, in, in, 128));
    EDPC_TRY(make_tmap_bf16(&g.tb, Pb + w_off, out, in, in, g.bn));
    return EDPC_OK;
  };
  auto dx = [&](int site, int out, size_t w_off, int in) -> int {
    TcGemm& g = tc.site[site];
    g.M = d.b;
    g.N = in;
    g.K = out;
    g.bn = pick_bn(in);
    EDPC_TRY(make_tmap_bf16(&g.ta, xa, d.b, out, out, 128));
    EDPC_TRY(make_tmap_bf16(&g.tb, PbT + w_off, in, out, out, g.bn));
    return EDPC_OK;
  };
  auto dw = [&](int site, int out, int in) -> int {
    TcGemm& g = tc.site[site];
    g.M = out;
    g.N = in;
    g.K = d.b;
    g.bn = pick_bn(in);
    EDPC_TRY(make_tmap_bf16(&g.ta, xaT, out, d.b, d.ldT, 128));
    EDPC_TRY(make_tmap_bf16(&g.tb, xbT, in, d.b, d.ldT, g.bn));
    return EDPC_OK;
  };
  const int kH = d.k * d.H;
  for (int j = 0; j < d.n; ++j) {
    EDPC_TRY(fwd(blk_site(BR_FWD, j), d.F, po.blk[j].W, kH));
    EDPC_TRY(fwd(blk_site(OUT_FWD, j), d.H, po.blk[j].Wo, d.F));
    EDPC_TRY(dw(blk_site(OUT_DW, j), d.F, d.H));
    EDPC_TRY(dx(blk_site(OUT_DX, j), d.F, po.blk[j].Wo, d.H));
    EDPC_TRY(dw(blk_site(BR_DW, j), kH, d.F));
    EDPC_TRY(dx(blk_site(BR_DX, j), kH, po.blk[j].W, d.F));
  }
  EDPC_TRY(fwd(kSiteLteDownFwd, d.F, po.W1, d.Fp));
  EDPC_TRY(fwd(kSiteLteUpFwd, d.Fp, po.W2, d.F));
  EDPC_TRY(fwd(kSiteHeadFwd, d.F, po.Wh, 256));
  EDPC_TRY(dx(kSiteHeadDx, 256, po.Wh, d.F));
  EDPC_TRY(dw(kSiteHeadDw, 256, d.F));
  EDPC_TRY(dw(kSiteLteUpDw, d.F, d.Fp));
  EDPC_TRY(dx(kSiteLteUpDx, d.F, po.W2, d.Fp));
  EDPC_TRY(dw(kSiteLteDownDw, d.Fp, d.F));
  EDPC_TRY(dx(kSiteLteDownDx, d.Fp, po.W1, d.F));
  tc.ready = true;
  return EDPC_OK;
}

// ------------------------------------------------------------------------------------------
// Linear layers (Y = X W^T + b) and their adjoints, in FP32 SIMT or BF16 tcgen05.
// ------------------------------------------------------------------------------------------
int Model::linear_fwd(int site, const float* X, int rows, int in, size_t w_off, size_t b_off, int out,
                      const float* resid, float* Yo, cudaStream_t st) {
  const int epi = resid ? EPI_BIAS_RESID : EPI_BIAS;
  if (precision == EDPC_BF16) {
    EDPC_CUDA(launch_to_bf16(X, rows, in, in, xa, in, nullptr, 0, st));
    TcGemm g = tc.site[site];
    g.C = Yo;
    g.ldc = out;
    g.epi = epi;
    g.bias = P + b_off;
    g.R = resid;
    g.ldr = out;
    g.err = &ctl->err;
    EDPC_CUDA(launch_gemm_tc(g, st));
    return EDPC_OK;
  }
  GemmF32 g{rows, out, in, X, in, true, P + w_off, in, true, Yo, out, epi, P + b_off, resid, out};
  EDPC_CUDA(launch_gemm_f32(g, st));
  return EDPC_OK;
}

int Model::linear_dx(int site, const float* dOut, int rows, int out, size_t w_off, int in, float* dX,
                     cudaStream_t st) {
  if (precision == EDPC_BF16) {
    EDPC_CUDA(launch_to_bf16(dOut, rows, out, out, xa, out, nullptr, 0, st));
    TcGemm g = tc.site[site];
    g.C = dX;
    g.ldc = in;
    g.epi = EPI_STORE;
    g.err = &ctl->err;
    EDPC_CUDA(launch_gemm_tc(g, st));
    return EDPC_OK;
  }
  GemmF32 g{rows, in, out, dOut, out, true, P + w_off, in, false, dX, in, EPI_STORE, nullptr, nullptr, 0};
  EDPC_CUDA(launch_gemm_f32(g, st));
  return EDPC_OK;
}

int Model::linear_dw(int site, const float* dOut, int rows, int out, const float* X, int in, size_t w_off,
                     cudaStream_t st) {
  if (precision == EDPC_BF16) {
    EDPC_CUDA(launch_to_bf16(dOut, rows, out, out, nullptr, 0, xaT, d.ldT, st));
    EDPC_CUDA(launch_to_bf16(X, rows, in, in, nullptr, 0, xbT, d.ldT, st));
    TcGemm g = tc.site[site];
    g.C = G + w_off;
    g.ldc = in;
    g.epi = EPI_STORE;
    g.err = &ctl->err;
    EDPC_CUDA(launch_gemm_tc(g, st));
    return EDPC_OK;
  }
  GemmF32 g{out, in, rows, dOut, out, false, X, in, false, G + w_off, in, EPI_STORE, nullptr, nullptr, 0};
  EDPC_CUDA(launch_gemm_f32(g, st));
  return EDPC_OK;
}

// ------------------------------------------------------------------------------------------
// Forward
// ------------------------------------------------------------------------------------------
int Model::block_fwd(int j, const float* Xin, float* Xout, cudaStream_t st) {
  const BlockOff& o = po.blk[j];
  BlockAct& a = ba[j];
  const int kH = d.k * d.H;
  EDPC_CUDA(launch_ln_fwd(Xin, P + o.ln_g, P + o.ln_b, a.xhat, a.rstd, a.X0, d.b, d.F, st));   // Eq. 9
  EDPC_TRY(linear_fwd(blk_site(BR_FWD, j), a.X0, d.b, d.F, o.W, o.c, kH, nullptr, a.A, st));   // Eq. 10
  EDPC_CUDA(launch_branch_gelu(a.A, d.b, d.H, d.k, a.G, st));                                  // Eqs. 11-12
  EDPC_TRY(linear_fwd(blk_site(OUT_FWD, j), a.G, d.b, d.H, o.Wo, o.co, d.F, Xin, Xout, st));   // Eq. 13
  return EDPC_OK;
}

int Model::forward(const StepIO& io, cudaStream_t st) {
  EDPC_CUDA(launch_embed(io.mode == 2 ? nullptr : io.data, io.sp, ctl, P + po.E, d.b, d.K, d.D, S[0], ctx, st));
  for (int j = 0; j < d.nloc; ++j) EDPC_TRY(block_fwd(j, S[j], S[j + 1], st));
  const float* lte_in = S[d.nloc];
  EDPC_TRY(linear_fwd(kSiteLteDownFwd, lte_in, d.b, d.F, po.W1, po.b1, d.Fp, nullptr, Xp, st));  // Eq. 14
  if (timing && ev_fdm[0]) EDPC_CUDA(record_timing(ev_fdm[0], st));
  EDPC_CUDA(launch_fdm_fwd(Xp, U, Y, d.b, d.Fp, st));                                              // Eq. 15
  if (timing && ev_fdm[1]) EDPC_CUDA(record_timing(ev_fdm[1], st));
  EDPC_TRY(linear_fwd(kSiteLteUpFwd, Y, d.b, d.Fp, po.W2, po.b2, d.F, nullptr, S[d.nloc + 1], st));  // Eq. 16
  for (int j = d.nloc; j < d.n; ++j) EDPC_TRY(block_fwd(j, S[j + 1], S[j + 2], st));
  EDPC_TRY(linear_fwd(kSiteHeadFwd, S[d.n + 1], d.b, d.F, po.Wh, po.bh, 256, nullptr, z, st));
  return EDPC_OK;
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
  h.err = &ctl->err;
  EDPC_CUDA(launch_head(h, st));
  return EDPC_OK;
}

// ------------------------------------------------------------------------------------------
// Backward (adjoint of the forward, in reverse order)
// ------------------------------------------------------------------------------------------
int Model::block_bwd(int j, const float* dOut, const float* Xin, float* dXnew, cudaStream_t st) {
  const BlockOff& o = po.blk[j];
  BlockAct& a = ba[j];
  const int kH = d.k * d.H;
  // Eq. 13: out = G Wo^T + co + X
  EDPC_TRY(linear_dw(blk_site(OUT_DW, j), dOut, d.b, d.F, a.G, d.H, o.Wo, st));
  EDPC_CUDA(launch_colsum(dOut, nullptr, d.b, d.F, d.F, G + o.co, st));
  EDPC_TRY(linear_dx(blk_site(OUT_DX, j), dOut, d.b, d.F, o.Wo, d.H, dG, st));
  // Eqs. 11-12: G = GELU(prod X_i)
  EDPC_CUDA(launch_branch_gelu_bwd(dG, a.A, d.b, d.H, d.k, dA, st));
  // Eq. 10: X_i = X0 W_i^T + c_i
  EDPC_TRY(linear_dw(blk_site(BR_DW, j), dA, d.b, kH, a.X0, d.F, o.W, st));
  EDPC_CUDA(launch_colsum(dA, nullptr, d.b, kH, kH, G + o.c, st));
  EDPC_TRY(linear_dx(blk_site(BR_DX, j), dA, d.b, kH, o.W, d.F, dX0, st));
  // Eq. 9: X0 = g * xhat + beta, plus the residual path of Eq. 13
  EDPC_CUDA(launch_colsum(dX0, a.xhat, d.b, d.F, d.F, G + o.ln_g, st));
  EDPC_CUDA(launch_colsum(dX0, nullptr, d.b, d.F, d.F, G + o.ln_b, st));
  EDPC_CUDA(launch_ln_bwd(dX0, a.xhat, a.rstd, P + o.ln_g, dOut, dXnew, d.b, d.F, st));
  (void)Xin;
  return EDPC_OK;
}

int Model::backward(const StepIO& io, cudaStream_t st) {
  // head: z = X Wh^T + bh
  const float* head_in = S[d.n + 1];
  EDPC_TRY(linear_dw(kSiteHeadDw, dz, d.b, 256, head_in, d.F, po.Wh, st));
  EDPC_CUDA(launch_colsum(dz, nullptr, d.b, 256, 256, G + po.bh, st));
  EDPC_TRY(linear_dx(kSiteHeadDx, dz, d.b, 256, po.Wh, d.F, dXa, st));
  float* cur = dXa;
  float* nxt = dXb;
  for (int j = d.n - 1; j >= d.nloc; --j) {
    EDPC_TRY(block_bwd(j, cur, S[j + 1], nxt, st));
    std::swap(cur, nxt);
  }
  // LTE up (Eq. 16)
  EDPC_TRY(linear_dw(kSiteLteUpDw, cur, d.b, d.F, Y, d.Fp, po.W2, st));
  EDPC_CUDA(launch_colsum(cur, nullptr, d.b, d.F, d.F, G + po.b2, st));
  EDPC_TRY(linear_dx(kSiteLteUpDx, cur, d.b, d.F, po.W2, d.Fp, dY, st));
  // FDM (Eq. 15): adjoint fused with the FDM's Adam update
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
  if (timing && ev_fdm[2]) EDPC_CUDA(record_timing(ev_fdm[2], st));
  EDPC_CUDA(launch_fdm_bwd(fa, st));
  if (timing && ev_fdm[3]) EDPC_CUDA(record_timing(ev_fdm[3], st));
  // LTE down (Eq. 14)
  EDPC_TRY(linear_dw(kSiteLteDownDw, dXp, d.b, d.Fp, S[d.nloc], d.F, po.W1, st));
  EDPC_CUDA(launch_colsum(dXp, nullptr, d.b, d.Fp, d.Fp, G + po.b1, st));
  EDPC_TRY(linear_dx(kSiteLteDownDx, dXp, d.b, d.Fp, po.W1, d.F, cur, st));
  for (int j = d.nloc - 1; j >= 0; --j) {
    EDPC_TRY(block_bwd(j, cur, S[j], nxt, st));
    std::swap(cur, nxt);
  }
  // embedding: scatter-add into E's rows
  EDPC_CUDA(launch_embed_bwd(ctx, cur, d.b, d.K, d.D, G + po.E, st));
  return EDPC_OK;
}

int Model::adam(cudaStream_t st) {
  EDPC_CUDA(launch_adam(P, G, M, V, nparam, ctl, st));
  if (precision == EDPC_BF16) EDPC_TRY(refresh_bf16_weights(st));
  return EDPC_OK;
}

int Model::step(const StepIO& io, cudaStream_t st) {
  EDPC_TRY(forward(io, st));
  EDPC_TRY(head(io, st));
  EDPC_TRY(backward(io, st));
  if (io.update) EDPC_TRY(adam(st));
  if (io.advance) EDPC_CUDA(launch_step_advance(ctl, io.sp, d.K, io.ring_slots, d.b, st));
  return EDPC_OK;
}

int Model::launches_per_step() const {
  const bool bf = precision == EDPC_BF16;
  // forward: embed + per block (ln, 2 GEMMs, gelu) + LTE (2 GEMMs + fdm) + head GEMM
  int fwd_gemms = 2 * d.n + 3;
  int n = 1 + 2 * d.n + fwd_gemms + 1;
  n += 1;  // head
  // backward: head (dw, colsum, dx); per block (2 dw, 2 dx, 4 colsum, gelu, ln) ; LTE (2 dw, 2 dx, 2 colsum) + fdm + embed
  int bwd_gemms = 2 + 4 * d.n + 4;
  n += bwd_gemms + 1 + 6 * d.n + 2 + 2;
  n += 1 + 1;  // adam, advance
  if (bf) {
    n += fwd_gemms;             // operand copies before forward GEMMs
    n += bwd_gemms / 2 * 2 + bwd_gemms / 2;  // dx: 1 copy, dw: 2 copies
    n += 2 * d.n + 3;           // weight refresh after Adam
  }
  return n;
}

}  // namespace edpc
