// File-set split and the stream-length autotuner (see archive.cuh).
#include <algorithm>
#include <cmath>

#include "archive.cuh"
#include "engine.cuh"

namespace edpc {

long long StreamLayout::max_len() const {
  long long m = 0;
  for (long long v : len) m = std::max(m, v);
  return m;
}

int StreamLayout::active_at(long long i) const {
  int a = 0;
  for (long long v : len) a += v > i ? 1 : 0;
  return a;
}

void archive_split(const uint64_t* sizes, size_t nfiles, uint64_t L, StreamLayout* out) {
  out->off.clear();
  out->len.clear();
  if (L < 1) L = 1;
  unsigned long long base = 0;
  for (size_t f = 0; f < nfiles; ++f) {
    const uint64_t n = sizes[f];
    const uint64_t m = (n + L - 1) / L;
    if (m) {
      const uint64_t q = n / m, rem = n % m;
      for (uint64_t j = 0; j < m; ++j) {
        out->off.push_back((long long)(base + j * q + std::min(j, rem)));
        out->len.push_back((long long)(q + (j < rem ? 1 : 0)));
      }
    }
    base += n;
  }
  if (out->len.empty()) {
    out->off.push_back(0);
    out->len.push_back(0);
  }
}

uint64_t archive_stream_count(const uint64_t* sizes, size_t nfiles, uint64_t L) {
  uint64_t c = 0;
  for (size_t f = 0; f < nfiles; ++f) c += (sizes[f] + L - 1) / L;
  return c ? c : 1;
}

uint64_t archive_stream_len(const uint64_t* sizes, size_t nfiles, uint64_t budget) {
  uint64_t mx = 0;
  bool any = false;
  for (size_t f = 0; f < nfiles; ++f)
    if (sizes[f]) {
      mx = std::max(mx, sizes[f]);
      any = true;
    }
  if (!any) return 1;
  uint64_t lo = 1, hi = mx;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    uint64_t c = 0;
    for (size_t f = 0; f < nfiles; ++f) c += (sizes[f] + mid - 1) / mid;
    if (c <= budget)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

namespace {

// Device bytes of a model of b streams and the time of one model step (mode 2:
// forward, head, adjoint, Adam), from a CUDA graph of the step replayed.
int probe(const edpc_cfg& c, int b, size_t* bytes, double* ms) {
  Model m;
  EDPC_TRY(m.init(c, b));
  *bytes = m.device_bytes();
  cudaStream_t st = nullptr;
  uint8_t* io_buf = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int r = EDPC_OK;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && r == EDPC_OK) r = fail(EDPC_ECUDA, std::string("autotune ") + what + ": " + cudaGetErrorString(e));
    return r == EDPC_OK;
  };
  if (cu(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream") &&
      cu(cudaMalloc(&io_buf, 2 * (size_t)b), "buffers") && cu(cudaMemsetAsync(io_buf, 0, b, st), "memset") &&
      cu(cudaMemsetAsync(io_buf + b, 1, b, st), "memset")) {
    r = m.set_ctl_for_step(c.context, 1, b, 1, st);
    if (r == EDPC_OK) r = m.tune_tiles(st);
  }
  Model::StepIO io;
  io.mode = 2;
  io.targets = io_buf;
  io.active = io_buf + b;
  io.advance = false;
  io.ring_slots = 1;
  if (r == EDPC_OK && cu(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture")) {
    int rs = m.step(io, st);
    if (rs == EDPC_OK) rs = m.flush(st);
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rs != EDPC_OK && r == EDPC_OK) r = rs;
    cu(ce, "capture end");
  }
  if (r == EDPC_OK && cu(cudaGraphInstantiate(&ge, g, 0), "instantiate") && cu(cudaEventCreate(&e0), "event") &&
      cu(cudaEventCreate(&e1), "event")) {
    const int warm = 3, reps = 8;
    for (int k = 0; k < warm && r == EDPC_OK; ++k) cu(cudaGraphLaunch(ge, st), "launch");
    cu(cudaEventRecord(e0, st), "record");
    for (int k = 0; k < reps && r == EDPC_OK; ++k) cu(cudaGraphLaunch(ge, st), "launch");
    cu(cudaEventRecord(e1, st), "record");
    if (cu(cudaEventSynchronize(e1), "sync")) {
      float t = 0;
      cu(cudaEventElapsedTime(&t, e0, e1), "elapsed");
      *ms = t / reps;
    }
  }
  if (st) cudaStreamSynchronize(st);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(io_buf);
  if (st) cudaStreamDestroy(st);
  return r;
}

}  // namespace

int archive_autotune(const edpc_cfg& c, const uint64_t* sizes, size_t nfiles, TunedPlan* out) {
  uint64_t mx = 0, total = 0;
  for (size_t f = 0; f < nfiles; ++f) {
    mx = std::max(mx, sizes[f]);
    total += sizes[f];
  }
  *out = TunedPlan{};
  if (mx == 0) {
    out->L = 1;
    out->streams = 1;
    return EDPC_OK;
  }
  // candidate stream lengths, longest last
  std::vector<uint64_t> cand;
  for (uint64_t L = 8192;; L *= 2) {
    cand.push_back(std::min(L, mx));
    if (L >= mx) break;
  }
  size_t free_b = 0, total_b = 0;
  EDPC_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.7 * (double)free_b;
  // session buffers besides the model: input, coder output (<= 2L + L/256 + 64
  // per stream), the coder ring (128 x 4 B per stream) and coder state
  auto session_bytes = [&](uint64_t b) { return 3.1 * (double)total + (double)b * (64 + 512 + 64); };

  // two probes of the step time (and the model's bytes per stream)
  uint64_t bmax = 0;
  for (uint64_t L : cand) {
    uint64_t b = archive_stream_count(sizes, nfiles, L);
    if (b <= 65535) bmax = std::max(bmax, b);
  }
  if (bmax == 0) return fail(EDPC_EINVAL, "the file set needs more than 65535 streams at any stream length");
  int b_lo = (int)std::max<uint64_t>(1, std::min<uint64_t>(bmax, 256));
  size_t by_lo = 0;
  double t_lo = 0;
  EDPC_TRY(probe(c, b_lo, &by_lo, &t_lo));
  const double per_upper = (double)by_lo / b_lo;
  uint64_t b_hi = std::min<uint64_t>(bmax, 4096);
  while (b_hi > (uint64_t)b_lo && per_upper * b_hi + session_bytes(b_hi) > budget) b_hi /= 2;
  double per = per_upper, fixed = 0, t0 = t_lo, cps = 0;
  if (b_hi > (uint64_t)b_lo) {
    size_t by_hi = 0;
    double t_hi = 0;
    EDPC_TRY(probe(c, (int)b_hi, &by_hi, &t_hi));
    per = (double)(by_hi - by_lo) / (double)(b_hi - b_lo);
    fixed = (double)by_lo - per * b_lo;
    cps = std::max(0.0, (t_hi - t_lo) / (double)(b_hi - b_lo));
    t0 = std::max(0.0, t_lo - cps * b_lo);
  }
  // estimates per candidate
  double best = 1e300;
  std::vector<double> est(cand.size(), -1.0);
  for (size_t j = 0; j < cand.size(); ++j) {
    const uint64_t b = archive_stream_count(sizes, nfiles, cand[j]);
    if (b > 65535) continue;
    if (fixed + per * (double)b + session_bytes(b) > budget) continue;
    StreamLayout lay;
    archive_split(sizes, nfiles, cand[j], &lay);
    const long long steps = std::max<long long>(0, lay.max_len() - (long long)c.context);
    est[j] = (double)steps * (t0 + cps * (double)b) / 1e3;
    best = std::min(best, est[j]);
  }
  if (best >= 1e299) return fail(EDPC_ENOMEM, "no stream length fits the file set's model in device memory");
  for (size_t j = cand.size(); j-- > 0;)
    if (est[j] >= 0 && est[j] <= 1.05 * best) {
      out->L = cand[j];
      out->streams = (uint32_t)archive_stream_count(sizes, nfiles, cand[j]);
      out->est_seconds = est[j];
      break;
    }
  out->step_ms_t0 = t0;
  out->step_ms_per_stream = cps;
  return EDPC_OK;
}

}  // namespace edpc
