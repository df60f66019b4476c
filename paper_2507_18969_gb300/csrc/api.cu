// C ABI of the library: configuration checks, the container format, encoder
// and decoder sessions (Algorithm 1 over b streams with the decoupled coder
// stage of Sec. 3.3), single-kernel entry points, and the model API.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "archive.cuh"
#include "engine.cuh"

using namespace edpc;

// ==========================================================================================
// errors
// ==========================================================================================
namespace edpc {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  // A failed allocation is not sticky, but the runtime keeps it as the
  // thread's last error; clear it so that later launch checks do not see it.
  if (code == EDPC_ENOMEM) (void)cudaGetLastError();
  return code;
}
}  // namespace edpc

extern "C" const char* edpc_strerror(int status) {
  switch (status) {
    case EDPC_OK: return "ok";
    case EDPC_EINVAL: return "invalid argument";
    case EDPC_ENOMEM: return "out of memory";
    case EDPC_ECORRUPT: return "corrupt bitstream";
    case EDPC_EVERSION: return "unsupported bitstream version";
    case EDPC_ECUDA: return "CUDA error";
    case EDPC_ETIMEOUT: return "device wait timed out";
    case EDPC_EARCH: return "bitstream variant not supported by this library version";
    default: return "unknown status";
  }
}

extern "C" const char* edpc_last_error(void) { return g_last_error.c_str(); }

extern "C" void edpc_free(void* p) { free(p); }

extern "C" void edpc_default_cfg(edpc_cfg* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->version = EDPC_ABI_VERSION;
  c->streams = 4;
  c->context = 16;
  c->embed_dim = 16;
  c->latent = 128;
  c->hidden = 128;
  c->blocks = 2;
  c->branches = 2;
  c->lr = 1e-3f;
  c->precision = EDPC_FP32;
  c->seed = 1;
}

// streams = 0 (autotuned stream count) is accepted for file sets only.
static int check_cfg(const edpc_cfg* c, bool auto_streams = false) {
  if (!c) return fail(EDPC_EINVAL, "cfg is NULL");
  if (c->version != EDPC_ABI_VERSION) return fail(EDPC_EINVAL, "cfg.version != EDPC_ABI_VERSION");
  if ((c->streams < 1 && !auto_streams) || c->streams > kMaxStreams)
    return fail(EDPC_EINVAL, auto_streams ? "streams must be in [0, 65535]" : "streams must be in [1, 65535]");
  if (c->context < 1 || c->context > 256) return fail(EDPC_EINVAL, "context must be in [1, 256]");
  if (c->embed_dim < 8 || c->embed_dim > 64 || c->embed_dim % 8)
    return fail(EDPC_EINVAL, "embed_dim must be a multiple of 8 in [8, 64]");
  if ((uint64_t)c->context * c->embed_dim > 2048) return fail(EDPC_EINVAL, "context * embed_dim must be <= 2048");
  if (c->latent == 0) {  // "w/o LTE": the FDM is F x F
    if ((uint64_t)c->context * c->embed_dim > 1024)
      return fail(EDPC_EINVAL, "latent = 0 (no LTE) needs context * embed_dim <= 1024");
  } else if (c->latent < 8 || c->latent > 1024 || c->latent % 8) {
    return fail(EDPC_EINVAL, "latent must be 0 or a multiple of 8 in [8, 1024]");
  }
  if (c->hidden < 8 || c->hidden > 2048 || c->hidden % 8)
    return fail(EDPC_EINVAL, "hidden must be a multiple of 8 in [8, 2048]");
  if (c->blocks < 1 || c->blocks > (uint32_t)kMaxBlocks) return fail(EDPC_EINVAL, "blocks must be in [1, 16]");
  if (c->branches < 1 || c->branches > 3) return fail(EDPC_EINVAL, "branches must be in [1, 3]");
  if (!(c->lr > 0.f) || !std::isfinite(c->lr)) return fail(EDPC_EINVAL, "lr must be finite and > 0");
  if (c->precision != EDPC_FP32 && c->precision != EDPC_BF16 && c->precision != EDPC_FP8E4M3)
    return fail(EDPC_EINVAL, "unknown precision");
  if (c->flags & EDPC_FLAG_DELAYED_UPDATE) {
    if (c->precision == EDPC_FP8E4M3) return fail(EDPC_EINVAL, "the delayed update needs FP32 or BF16");
    if (c->flags & EDPC_FLAG_OVERLAP_FDM)
      return fail(EDPC_EINVAL, "the delayed update and EDPC_FLAG_OVERLAP_FDM exclude each other");
  }
  return EDPC_OK;
}

extern "C" uint64_t edpc_param_count(const edpc_cfg* c) {
  if (check_cfg(c) != EDPC_OK) return 0;
  return make_offsets(make_dims(*c, 1)).total;
}

static int current_device_ok() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return fail(EDPC_ECUDA, "no CUDA device available");
  return EDPC_OK;
}

// ==========================================================================================
// checksums
// ==========================================================================================
namespace {

uint32_t crc32_ieee(const uint8_t* p, size_t n) {
  static uint32_t table[256];
  static bool init = false;
  if (!init) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
    init = true;
  }
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xFF] ^ (c >> 8);
  return c ^ 0xFFFFFFFFu;
}

// Data checksum: XOR over positions i of SplitMix64's finalizer applied to
// (i << 8) | x_i. Any single changed byte changes it.
__global__ void checksum_kernel(const uint8_t* __restrict__ x, unsigned long long n, unsigned long long* out) {
  unsigned long long h = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long z = (i << 8) | x[i];
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    h ^= z ^ (z >> 31);
  }
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicXor(out, h);
}

int device_checksum(const uint8_t* x, uint64_t n, unsigned long long* scratch, cudaStream_t st, uint64_t* out) {
  EDPC_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), st));
  if (n) {
    int grid = (int)std::min<uint64_t>((n + 255) / 256, 152 * 16);
    checksum_kernel<<<grid, 256, 0, st>>>(x, n, scratch);
    EDPC_CUDA(cudaGetLastError());
  }
  unsigned long long h = 0;
  EDPC_CUDA(cudaMemcpyAsync(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
  EDPC_CUDA(cudaStreamSynchronize(st));
  *out = h;
  return EDPC_OK;
}

// Copies each stream's bytes into one contiguous buffer.
__global__ void gather_streams_kernel(const uint8_t* __restrict__ src, const unsigned long long* __restrict__ src_off,
                                      const uint32_t* __restrict__ len, const unsigned long long* __restrict__ dst_off,
                                      uint8_t* __restrict__ dst) {
  const int s = blockIdx.x;
  const uint8_t* a = src + src_off[s];
  uint8_t* b = dst + dst_off[s];
  for (uint32_t i = threadIdx.x; i < len[s]; i += blockDim.x) b[i] = a[i];
}

// ------------------------------------------------------------------------------------------
// container header
// ------------------------------------------------------------------------------------------
constexpr uint32_t kMagic = 0x43504445u;  // "EDPC" little-endian
constexpr uint32_t kSchedDelayed = 1u;     // header word 11: the delayed-update schedule
constexpr size_t kFixedHeader = 88;

// Variant 0: one input, balanced split, size-heuristic GEMM tiles.
// Variant 2: as variant 0, coded by the engine of independent per-file models
//   in one batch (the file's streams padded to a multiple of 64 rows with its
//   own model; see GroupInfo): the decoder replays that engine with one group.
// Variant 1: extended header after the fixed part:
//   u64 nfiles, u64 L (stream length of the file-set split; 0 = one input
//   with the balanced split), u32 ntile, u32 0, u64 size[nfiles],
//   u8 tile[ntile] (padded to 4 bytes): the GEMM tile code of every site.
struct Header {
  edpc_cfg cfg;
  uint64_t n = 0;
  uint32_t b = 0;
  uint64_t checksum = 0;
  uint32_t variant = 0;
  uint64_t L = 0;
  std::vector<uint64_t> sizes;
  std::vector<uint8_t> tiles;
  std::vector<uint32_t> len;
  size_t header_len = 0;
};

size_t ext_bytes(const Header& h) {
  return h.variant == 1 ? 24 + 8 * h.sizes.size() + ((h.tiles.size() + 3) & ~(size_t)3) : 0;
}

template <class T>
void put(std::vector<uint8_t>& v, size_t off, T x) {
  memcpy(v.data() + off, &x, sizeof(T));
}
template <class T>
T get(const uint8_t* p, size_t off) {
  T x;
  memcpy(&x, p + off, sizeof(T));
  return x;
}

std::vector<uint8_t> write_header(const Header& h) {
  const size_t ext = ext_bytes(h);
  std::vector<uint8_t> v(kFixedHeader + ext + 4 * (size_t)h.b + 4, 0);
  put<uint32_t>(v, 0, kMagic);
  put<uint32_t>(v, 4, EDPC_FORMAT_VERSION);
  put<uint32_t>(v, 8, (uint32_t)v.size());
  put<uint32_t>(v, 12, h.cfg.precision);
  put<uint32_t>(v, 16, h.cfg.context);
  put<uint32_t>(v, 20, h.cfg.embed_dim);
  put<uint32_t>(v, 24, h.cfg.latent);
  put<uint32_t>(v, 28, h.cfg.hidden);
  put<uint32_t>(v, 32, h.cfg.blocks);
  put<uint32_t>(v, 36, h.cfg.branches);
  put<float>(v, 40, h.cfg.lr);
  put<uint32_t>(v, 44, (h.cfg.flags & EDPC_FLAG_DELAYED_UPDATE) ? kSchedDelayed : 0u);  // update schedule
  put<uint64_t>(v, 48, h.cfg.seed);
  put<uint64_t>(v, 56, h.n);
  put<uint32_t>(v, 64, h.cfg.streams);
  put<uint32_t>(v, 68, h.b);
  put<uint64_t>(v, 72, h.checksum);
  put<uint32_t>(v, 80, h.variant);
  put<uint32_t>(v, 84, 0);
  if (h.variant == 1) {
    size_t o = kFixedHeader;
    put<uint64_t>(v, o, (uint64_t)h.sizes.size());
    put<uint64_t>(v, o + 8, h.L);
    put<uint32_t>(v, o + 16, (uint32_t)h.tiles.size());
    o += 24;
    for (uint64_t sz : h.sizes) {
      put<uint64_t>(v, o, sz);
      o += 8;
    }
    if (!h.tiles.empty()) memcpy(v.data() + o, h.tiles.data(), h.tiles.size());
  }
  for (uint32_t s = 0; s < h.b; ++s) put<uint32_t>(v, kFixedHeader + ext + 4 * (size_t)s, h.len[s]);
  put<uint32_t>(v, v.size() - 4, crc32_ieee(v.data(), v.size() - 4));
  return v;
}

int read_header(const uint8_t* p, size_t n, Header* h) {
  if (!p) return fail(EDPC_EINVAL, "bitstream is NULL");
  if (n < kFixedHeader + 4) return fail(EDPC_ECORRUPT, "bitstream shorter than the header");
  if (get<uint32_t>(p, 0) != kMagic) return fail(EDPC_ECORRUPT, "bad magic");
  if (get<uint32_t>(p, 4) != EDPC_FORMAT_VERSION) return fail(EDPC_EVERSION, "unsupported format version");
  size_t hl = get<uint32_t>(p, 8);
  uint32_t b = get<uint32_t>(p, 68);
  if (b < 1 || b > (uint32_t)kMaxStreams || hl < kFixedHeader + 4 * (size_t)b + 4 || hl > n)
    return fail(EDPC_ECORRUPT, "bad header length or stream count");
  if (crc32_ieee(p, hl - 4) != get<uint32_t>(p, hl - 4)) return fail(EDPC_ECORRUPT, "header CRC mismatch");
  h->variant = get<uint32_t>(p, 80);
  size_t ext = 0;
  if (h->variant == 1) {
    if (hl < kFixedHeader + 24 + 4 * (size_t)b + 4) return fail(EDPC_ECORRUPT, "bad extended header length");
    const uint64_t nf = get<uint64_t>(p, kFixedHeader);
    h->L = get<uint64_t>(p, kFixedHeader + 8);
    const uint32_t nt = get<uint32_t>(p, kFixedHeader + 16);
    if (nf > hl / 8 || nt > (uint32_t)TcPlan::kMaxSites) return fail(EDPC_ECORRUPT, "bad extended header counts");
    h->sizes.resize(nf);
    for (uint64_t f = 0; f < nf; ++f) h->sizes[f] = get<uint64_t>(p, kFixedHeader + 24 + 8 * f);
    h->tiles.assign(p + kFixedHeader + 24 + 8 * nf, p + kFixedHeader + 24 + 8 * nf + nt);
    ext = ext_bytes(*h);
  } else if (h->variant != 0 && h->variant != 2) {
    return fail(EDPC_EARCH, "unknown header variant " + std::to_string(h->variant));
  }
  if (hl != kFixedHeader + ext + 4 * (size_t)b + 4) return fail(EDPC_ECORRUPT, "bad header length");
  edpc_default_cfg(&h->cfg);
  h->cfg.precision = get<uint32_t>(p, 12);
  h->cfg.context = get<uint32_t>(p, 16);
  h->cfg.embed_dim = get<uint32_t>(p, 20);
  h->cfg.latent = get<uint32_t>(p, 24);
  h->cfg.hidden = get<uint32_t>(p, 28);
  h->cfg.blocks = get<uint32_t>(p, 32);
  h->cfg.branches = get<uint32_t>(p, 36);
  h->cfg.lr = get<float>(p, 40);
  const uint32_t sched = get<uint32_t>(p, 44);
  if (sched & ~kSchedDelayed) return fail(EDPC_EARCH, "unknown update schedule " + std::to_string(sched));
  if (sched & kSchedDelayed) h->cfg.flags |= EDPC_FLAG_DELAYED_UPDATE;
  h->cfg.seed = get<uint64_t>(p, 48);
  h->n = get<uint64_t>(p, 56);
  h->cfg.streams = get<uint32_t>(p, 64);
  h->b = b;
  h->checksum = get<uint64_t>(p, 72);
  int r = check_cfg(&h->cfg, h->variant == 1 && h->L > 0);
  if (r != EDPC_OK) return fail(EDPC_ECORRUPT, "header holds an invalid configuration: " + g_last_error);
  if (h->variant == 2 && h->cfg.precision != EDPC_BF16)
    return fail(EDPC_ECORRUPT, "an independent-model member must be BF16");
  h->len.resize(b);
  uint64_t total = 0;
  for (uint32_t s = 0; s < b; ++s) {
    h->len[s] = get<uint32_t>(p, kFixedHeader + ext + 4 * (size_t)s);
    total += h->len[s];
  }
  h->header_len = hl;
  if (hl + total != n) return fail(EDPC_ECORRUPT, "stream lengths do not match the bitstream size");
  if (h->variant == 1 && h->L > 0) {
    uint64_t tot = 0;
    for (uint64_t sz : h->sizes) tot += sz;
    if (tot != h->n) return fail(EDPC_ECORRUPT, "file sizes do not add up to the input length");
    if (archive_stream_count(h->sizes.data(), h->sizes.size(), h->L) != b)
      return fail(EDPC_ECORRUPT, "stream count does not match the file-set split");
    return EDPC_OK;
  }
  uint32_t be = (uint32_t)std::min<uint64_t>(h->cfg.streams, std::max<uint64_t>(1, h->n / h->cfg.context));
  if (be != b) return fail(EDPC_ECORRUPT, "stream count does not match the split rule");
  return EDPC_OK;
}

Split make_split(uint64_t n, int b) {
  Split sp;
  sp.n = (long long)n;
  sp.q = (long long)(n / (uint64_t)b);
  sp.rem = (int)(n % (uint64_t)b);
  return sp;
}

int effective_streams(const edpc_cfg& c, uint64_t n) {
  return (int)std::min<uint64_t>(c.streams, std::max<uint64_t>(1, n / c.context));
}

// Rows of independent per-file models in one batch: file f (n_f bytes at
// offset off_f of the files' concatenation) gets its member's balanced split
// into b_f streams (q or q + 1 bytes, the longer first), then padding rows of
// no bytes up to a multiple of kGroupAlign rows; group f owns those rows.
struct GroupPlan {
  StreamLayout lay;
  std::vector<GroupInfo> groups;
  std::vector<uint64_t> n, off;
  std::vector<uint32_t> b;
};

int grouped_plan(const uint64_t* sizes, const uint32_t* streams, size_t nfiles, GroupPlan* gp) {
  gp->lay.off.clear();
  gp->lay.len.clear();
  gp->groups.clear();
  gp->n.assign(sizes, sizes + nfiles);
  gp->b.assign(streams, streams + nfiles);
  gp->off.resize(nfiles);
  uint64_t o = 0;
  long long rows = 0;
  for (size_t f = 0; f < nfiles; ++f) {
    const uint64_t n = sizes[f];
    const uint32_t b = streams[f];
    if (b < 1) return fail(EDPC_EINVAL, "a member has no stream");
    gp->off[f] = o;
    GroupInfo g;
    g.r0 = (int)rows;
    g.s = (int)b;
    g.q = (long long)(n / b);
    g.rem = (int)(n % b);
    for (uint32_t j = 0; j < b; ++j) {
      gp->lay.off.push_back((long long)o + (long long)j * g.q + std::min<long long>(j, g.rem));
      gp->lay.len.push_back(g.q + (j < (uint32_t)g.rem ? 1 : 0));
    }
    const long long padded = round_up(b, kGroupAlign);
    for (long long j = b; j < padded; ++j) {
      gp->lay.off.push_back((long long)(o + n));
      gp->lay.len.push_back(0);
    }
    rows += padded;
    if (rows > (long long)kMaxStreams)
      return fail(EDPC_EINVAL, "independent models in one batch: more than 65535 rows (streams plus padding)");
    g.r1 = (int)rows;
    gp->groups.push_back(g);
    o += n;
  }
  if (gp->groups.empty()) return fail(EDPC_EINVAL, "no files");
  return EDPC_OK;
}

}  // namespace

// ==========================================================================================
// sessions
// ==========================================================================================
struct edpc_session {
  bool encoder = true;
  edpc_cfg cfg{};
  Model model;
  Split sp{};
  StreamLayout lay;                    // host copy of every stream's byte range
  unsigned long long* seg = nullptr;   // device: b + 1 stream offsets (explicit split)
  ActivePoint* cp = nullptr;           // device: active-count change points
  uint32_t variant = 0;                // header variant written by the encoder
  uint64_t arch_L = 0;                 // file-set stream length (variant 1)
  std::vector<uint64_t> file_sizes;    // file-set sizes (variant 1)
  std::vector<uint8_t> tiles;          // GEMM tile codes recorded in the header
  GroupPlan gp;                        // independent per-file models in one batch (variant 2 members)
  bool grouped = false;
  int b = 0;
  uint64_t n = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaStream_t st_coder = nullptr;
  bool pipeline = true;
  bool use_graph = true;
  uint8_t* data = nullptr;
  bool own_data = false;
  unsigned long long* scratch = nullptr;

  // encoder
  uint8_t* out = nullptr;
  unsigned long long* out_off = nullptr;
  uint32_t* out_cap = nullptr;
  uint32_t* out_len = nullptr;
  EncState* es = nullptr;
  uint32_t* ring = nullptr;
  int chunk = 64;
  int ring_slots = 128;
  cudaEvent_t ev_model[2] = {}, ev_coder[2] = {}, ev_join = nullptr;
  uint64_t coded = 0;
  std::vector<unsigned long long> h_out_off;

  // decoder
  uint8_t* bits = nullptr;
  unsigned long long* bits_off = nullptr;
  uint32_t* bits_len = nullptr;
  DecState* ds = nullptr;
  uint64_t checksum_expected = 0;

  uint64_t steps_total = 0, steps_run = 0;
  bool finished = false;

  // CUDA graphs: `chunk` consecutive steps (so each step's FDM update can run
  // under the next step's first layers), instantiated twice with separate
  // timing events and launched alternately; and a one-step graph for step
  // counts that do not fill a chunk.
  cudaGraph_t g_chunk = nullptr, g_one = nullptr;
  cudaGraphExec_t x_chunk[2] = {}, x_one = nullptr;
  int graph_kernels = 0;  // kernels per step

  // FDM kernel timing: event set k of chunk execution p is tev[p * chunk + k];
  // the one-step graph (and eager steps) use the sets after those.
  bool profiling = false;
  static constexpr int kChunk = 64;
  static constexpr int kEvSets = 2 * kChunk + 1;
  static constexpr int kEv = 6;  // FDM forward, adjoint (dx'), FDM update: start/end each
  cudaEvent_t tev[kEvSets][kEv] = {};
  bool has_adam_ev = false;
  bool tev_live[kEvSets] = {};
  double fwd_ms = 0, bwd_ms = 0, adam_ms = 0;
  uint64_t samples = 0;

  Model::StepIO io;

  ~edpc_session();
  int setup_common(const edpc_cfg& c, uint64_t n_, void* stream, const StreamLayout* explicit_lay = nullptr,
                   const std::vector<GroupInfo>* groups = nullptr);
  int capture_graph();
  int capture(int nsteps, int set0, cudaGraph_t* g);
  int launch_steps(uint64_t n);
  int code_pending();
  int join();
  int harvest(int k);
};

edpc_session::~edpc_session() {
  if (st) cudaStreamSynchronize(st);
  if (st_coder) cudaStreamSynchronize(st_coder);
  for (auto& x : x_chunk)
    if (x) cudaGraphExecDestroy(x);
  if (x_one) cudaGraphExecDestroy(x_one);
  if (g_chunk) cudaGraphDestroy(g_chunk);
  if (g_one) cudaGraphDestroy(g_one);
  for (auto& e : ev_model)
    if (e) cudaEventDestroy(e);
  for (auto& e : ev_coder)
    if (e) cudaEventDestroy(e);
  if (ev_join) cudaEventDestroy(ev_join);
  for (auto& set : tev)
    for (auto& e : set)
      if (e) cudaEventDestroy(e);
  for (auto& e : model.ev_fdm) e = nullptr;  // owned by the session's tev sets
  if (own_data && data) cudaFree(data);
  cudaFree(scratch);
  cudaFree(out);
  cudaFree(out_off);
  cudaFree(out_cap);
  cudaFree(out_len);
  cudaFree(es);
  cudaFree(ring);
  cudaFree(bits);
  cudaFree(bits_off);
  cudaFree(bits_len);
  cudaFree(ds);
  cudaFree(seg);
  cudaFree(cp);
  if (st_coder) cudaStreamDestroy(st_coder);
  if (own_stream && st) cudaStreamDestroy(st);
}

int edpc_session::setup_common(const edpc_cfg& c, uint64_t n_, void* stream, const StreamLayout* explicit_lay,
                               const std::vector<GroupInfo>* groups) {
  cfg = c;
  n = n_;
  if (explicit_lay) {
    lay = *explicit_lay;
    b = lay.streams();
    if (b < 1 || b > (int)kMaxStreams) return fail(EDPC_EINVAL, "stream count out of range");
    sp = Split{(long long)n, 0, 0};
  } else {
    b = effective_streams(c, n);
    sp = make_split(n, b);
    lay.off.resize(b);
    lay.len.resize(b);
    for (int i = 0; i < b; ++i) {
      lay.off[i] = sp.off(i);
      lay.len[i] = sp.len(i);
    }
  }
  pipeline = !(c.flags & EDPC_FLAG_NO_PIPELINE);
  use_graph = !(c.flags & EDPC_FLAG_NO_GRAPH);
  if (stream) {
    st = static_cast<cudaStream_t>(stream);
  } else {
    EDPC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    own_stream = true;
  }
  EDPC_CUDA(cudaStreamCreateWithFlags(&st_coder, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    EDPC_CUDA(cudaEventCreateWithFlags(&ev_model[k], cudaEventDisableTiming));
    EDPC_CUDA(cudaEventCreateWithFlags(&ev_coder[k], cudaEventDisableTiming));
  }
  EDPC_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  EDPC_CUDA(cudaMalloc(&scratch, 64));
  if (explicit_lay) {
    // stream table and the steps at which the active count drops (Q12 masking)
    std::vector<unsigned long long> so(b + 1);
    for (int i = 0; i < b; ++i) so[i] = (unsigned long long)lay.off[i];
    so[b] = so[b - 1] + (unsigned long long)lay.len[b - 1];
    std::vector<long long> ls(lay.len);
    std::sort(ls.begin(), ls.end());
    std::vector<ActivePoint> pts;
    for (size_t k = 0; k < ls.size(); ++k) {
      if (ls[k] <= (long long)c.context || (k + 1 < ls.size() && ls[k + 1] == ls[k])) continue;
      pts.push_back({(int)ls[k], (int)(ls.size() - k - 1)});  // from step len on, the longer ones stay
    }
    EDPC_CUDA(cudaMalloc(&seg, 8 * (size_t)(b + 1)));
    EDPC_CUDA(cudaMalloc(&cp, sizeof(ActivePoint) * std::max<size_t>(1, pts.size())));
    EDPC_CUDA(cudaMemcpyAsync(seg, so.data(), 8 * (size_t)(b + 1), cudaMemcpyHostToDevice, st));
    if (!pts.empty())
      EDPC_CUDA(cudaMemcpyAsync(cp, pts.data(), sizeof(ActivePoint) * pts.size(), cudaMemcpyHostToDevice, st));
    EDPC_CUDA(cudaStreamSynchronize(st));
    sp.seg = seg;
    sp.cp = cp;
    sp.ncp = (int)pts.size();
  }
  EDPC_TRY(model.init(c, b, groups));
  long long L = lay.max_len();
  steps_total = L > (long long)c.context ? (uint64_t)(L - c.context) : 0;
  chunk = 64;
  ring_slots = 2 * chunk;
  return EDPC_OK;
}

// Captures `nsteps` model steps (timing event sets set0, set0 + 1, ...) into
// one graph that ends with every stream joined (the last FDM update waited for).
int edpc_session::capture(int nsteps, int set0, cudaGraph_t* g) {
  model.timing = true;
  EDPC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int r = EDPC_OK;
  for (int k = 0; k < nsteps && r == EDPC_OK; ++k) {
    for (int q = 0; q < kEv; ++q) model.ev_fdm[q] = tev[set0 + k][q];
    io.tick = k;  // graphs start at even steps
    r = model.step(io, st);
  }
  if (r == EDPC_OK) r = model.flush(st);
  cudaError_t ce = cudaStreamEndCapture(st, g);
  model.timing = false;
  if (r != EDPC_OK) {
    if (*g) cudaGraphDestroy(*g);
    *g = nullptr;
    return r;
  }
  if (ce != cudaSuccess) return fail(EDPC_ECUDA, std::string("stream capture: ") + cudaGetErrorString(ce));
  return EDPC_OK;
}

int edpc_session::capture_graph() {
  has_adam_ev = model.side_fdm != nullptr;
  if (!use_graph || steps_total == 0) return EDPC_OK;
  chunk = kChunk;
  EDPC_TRY(capture(1, 2 * kChunk, &g_one));
  EDPC_CUDA(cudaGraphInstantiate(&x_one, g_one, 0));
  size_t nn = 0;
  EDPC_CUDA(cudaGraphGetNodes(g_one, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  EDPC_CUDA(cudaGraphGetNodes(g_one, nodes.data(), &nn));
  graph_kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    EDPC_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++graph_kernels;
  }
  if (steps_total < (uint64_t)kChunk) return EDPC_OK;
  EDPC_TRY(capture(kChunk, 0, &g_chunk));
  EDPC_CUDA(cudaGraphInstantiate(&x_chunk[0], g_chunk, 0));
  EDPC_CUDA(cudaGraphInstantiate(&x_chunk[1], g_chunk, 0));
  // the second instantiation records into event sets kChunk .. 2 kChunk - 1
  nn = 0;
  EDPC_CUDA(cudaGraphGetNodes(g_chunk, nullptr, &nn));
  nodes.resize(nn);
  EDPC_CUDA(cudaGraphGetNodes(g_chunk, nodes.data(), &nn));
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    EDPC_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t e;
    EDPC_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &e));
    for (int k = 0; k < kChunk; ++k)
      for (int q = 0; q < kEv; ++q)
        if (e == tev[k][q]) EDPC_CUDA(cudaGraphExecEventRecordNodeSetEvent(x_chunk[1], nd, tev[kChunk + k][q]));
  }
  return EDPC_OK;
}

int edpc_session::harvest(int k) {
  if (!tev_live[k]) return EDPC_OK;
  EDPC_CUDA(cudaEventSynchronize(tev[k][3]));
  float a = 0, c = 0, m = 0;
  EDPC_CUDA(cudaEventElapsedTime(&a, tev[k][0], tev[k][1]));
  EDPC_CUDA(cudaEventElapsedTime(&c, tev[k][2], tev[k][3]));
  if (has_adam_ev) {
    EDPC_CUDA(cudaEventSynchronize(tev[k][5]));
    EDPC_CUDA(cudaEventElapsedTime(&m, tev[k][4], tev[k][5]));
  }
  fwd_ms += a;
  bwd_ms += c;
  adam_ms += m;
  ++samples;
  tev_live[k] = false;
  return EDPC_OK;
}

// Launches the next n model steps: whole chunks through the chunk graph when
// aligned, else one step at a time (one-step graph, or eagerly).
int edpc_session::launch_steps(uint64_t n) {
  uint64_t k = 0;
  while (k < n) {
    const uint64_t j = steps_run;
    if (encoder && pipeline && j % chunk == 0 && j >= (uint64_t)(2 * chunk))
      EDPC_CUDA(cudaStreamWaitEvent(st, ev_coder[(j / chunk) % 2], 0));
    uint64_t adv = 1;
    if (x_chunk[0] && j % chunk == 0 && n - k >= (uint64_t)chunk && steps_total - j >= (uint64_t)chunk) {
      const int p = (int)((j / chunk) % 2);
      if (profiling)
        for (int q = 0; q < chunk; ++q) EDPC_TRY(harvest(p * chunk + q));
      EDPC_TRY(model.flush(st));  // an eager step's FDM update may still run on its own stream
      EDPC_CUDA(cudaGraphLaunch(x_chunk[p], st));
      if (profiling)
        for (int q = 0; q < chunk; ++q) tev_live[p * chunk + q] = true;
      adv = (uint64_t)chunk;
    } else if (x_one && !model.delayed) {  // (the delayed update alternates parities: eager)
      const int set = 2 * kChunk;
      if (profiling) EDPC_TRY(harvest(set));
      EDPC_CUDA(cudaGraphLaunch(x_one, st));
      if (profiling) tev_live[set] = true;
    } else {
      const int set = (int)(j % (2 * kChunk));
      if (profiling) {
        EDPC_TRY(harvest(set));
        for (int q = 0; q < kEv; ++q) model.ev_fdm[q] = tev[set][q];
        model.timing = true;
      }
      io.tick = (int)(j & 1);
      int r = model.step(io, st);
      model.timing = false;
      if (r != EDPC_OK) return r;
      if (profiling) tev_live[set] = true;
    }
    steps_run += adv;
    k += adv;
    if (encoder && steps_run % chunk == 0) EDPC_TRY(code_pending());
  }
  return EDPC_OK;
}

// Hands the steps [coded, steps_run) to the coder stage (DPCA): on the
// coder stream after the model stream's event, or inline when pipelining is off.
int edpc_session::code_pending() {
  const uint64_t cnt = steps_run - coded;
  if (cnt == 0) return EDPC_OK;
  const int slot0 = (int)(coded % ring_slots);
  const int par = (int)((coded / chunk) % 2);
  if (pipeline) {
    EDPC_CUDA(cudaEventRecord(ev_model[par], st));
    EDPC_CUDA(cudaStreamWaitEvent(st_coder, ev_model[par], 0));
    EDPC_CUDA(launch_range_encode(es, ring, ring_slots, slot0, (int)cnt, b, out, out_off, out_cap, st_coder));
    EDPC_CUDA(cudaEventRecord(ev_coder[par], st_coder));
  } else {
    EDPC_CUDA(launch_range_encode(es, ring, ring_slots, slot0, (int)cnt, b, out, out_off, out_cap, st));
  }
  coded = steps_run;
  return EDPC_OK;
}

int edpc_session::join() {
  EDPC_TRY(model.flush(st));  // eager steps leave the last FDM update pending
  if (encoder && pipeline) {
    EDPC_CUDA(cudaEventRecord(ev_join, st_coder));
    EDPC_CUDA(cudaStreamWaitEvent(st, ev_join, 0));
  }
  return EDPC_OK;
}

static int session_prepare_events(edpc_session* s) {
  for (int k = 0; k < edpc_session::kEvSets; ++k)
    for (int q = 0; q < edpc_session::kEv; ++q) EDPC_CUDA(cudaEventCreate(&s->tev[k][q]));
  return EDPC_OK;
}

// Opens an encoder over the concatenation of `nparts` buffers (host, or
// device when data_on_device). A single device buffer is used in place.
// lay: explicit stream layout (file sets), else the balanced split.
// tune: time the GEMM tiles and record the chosen codes (header variant 1).
// gp: independent per-file models in one batch (lay is then gp->lay).
static int encoder_open_impl(const edpc_cfg* cfg, const uint8_t* const* parts, const uint64_t* part_len,
                             size_t nparts, int data_on_device, void* cuda_stream, const StreamLayout* lay,
                             uint32_t variant, uint64_t arch_L, bool tune, edpc_session** out,
                             const GroupPlan* gp = nullptr) {
  uint64_t len = 0;
  for (size_t f = 0; f < nparts; ++f) {
    if (!parts[f] && part_len[f]) return fail(EDPC_EINVAL, "data is NULL");
    len += part_len[f];
  }
  EDPC_TRY(current_device_ok());
  edpc_session* s = new (std::nothrow) edpc_session();
  if (!s) return fail(EDPC_ENOMEM, "host allocation failed");
  auto bail = [&](int r) {
    delete s;
    return r;
  };
  s->encoder = true;
  if (gp) {
    s->gp = *gp;
    s->grouped = true;
  }
  int r = gp ? s->setup_common(*cfg, len, cuda_stream, &gp->lay, &gp->groups)
             : s->setup_common(*cfg, len, cuda_stream, lay);
  if (r != EDPC_OK) return bail(r);
  if ((r = session_prepare_events(s)) != EDPC_OK) return bail(r);
  cudaStream_t st = s->st;
  s->variant = variant;
  s->arch_L = arch_L;
  if (variant == 1 && lay) s->file_sizes.assign(part_len, part_len + nparts);
  // input bytes on the device
  if (data_on_device && nparts == 1) {
    s->data = const_cast<uint8_t*>(parts[0]);
  } else {
    if (cudaMalloc(&s->data, std::max<uint64_t>(len, 1)) != cudaSuccess) return bail(fail(EDPC_ENOMEM, "input buffer"));
    s->own_data = true;
    uint64_t o = 0;
    for (size_t f = 0; f < nparts; ++f) {
      if (part_len[f] && cudaMemcpyAsync(s->data + o, parts[f], part_len[f],
                                         data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                         st) != cudaSuccess)
        return bail(fail(EDPC_ECUDA, "input copy failed"));
      o += part_len[f];
    }
  }
  // per-stream output buffers: a stream of L bytes codes to at most 2L + L/256 + 64 bytes
  const int b = s->b;
  s->h_out_off.resize(b + 1);
  std::vector<uint32_t> cap(b);
  unsigned long long tot = 0;
  for (int i = 0; i < b; ++i) {
    long long L = s->lay.len[i];
    if (L > (1ll << 31) - (1ll << 24)) return bail(fail(EDPC_EINVAL, "a stream is longer than 2 GiB - 16 MiB"));
    cap[i] = (uint32_t)(2 * L + (L >> 8) + 64);
    s->h_out_off[i] = tot;
    tot += (cap[i] + 15) & ~15u;
  }
  s->h_out_off[b] = tot;
  if (cudaMalloc(&s->out, tot) != cudaSuccess || cudaMalloc(&s->out_off, 8 * (size_t)b) != cudaSuccess ||
      cudaMalloc(&s->out_cap, 4 * (size_t)b) != cudaSuccess || cudaMalloc(&s->out_len, 4 * (size_t)b) != cudaSuccess ||
      cudaMalloc(&s->es, sizeof(EncState) * b) != cudaSuccess ||
      cudaMalloc(&s->ring, sizeof(uint32_t) * (size_t)b * s->ring_slots) != cudaSuccess)
    return bail(fail(EDPC_ENOMEM, "encoder buffers"));
  if (cudaMemcpyAsync(s->out_off, s->h_out_off.data(), 8 * (size_t)b, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->out_cap, cap.data(), 4 * (size_t)b, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return bail(fail(EDPC_ECUDA, "encoder setup copies"));
  if (tune && cfg->precision != EDPC_FP32) {
    if ((r = s->model.tune_tiles(st)) != EDPC_OK) return bail(r);
    s->tiles.assign(s->model.tile_code, s->model.tile_code + TcPlan::kMaxSites);
  }
  // Algorithm 1, first line: the first K bytes of each stream with equal probability
  if (launch_prefix_encode(s->es, s->data, s->sp, (int)cfg->context, b, s->out, s->out_off, s->out_cap, st) !=
      cudaSuccess)
    return bail(fail(EDPC_ECUDA, "prefix encode launch"));
  long long i0 = cfg->context;
  if ((r = s->model.set_ctl_for_step((int)i0, 1, s->lay.active_at(i0), s->ring_slots, st)) != EDPC_OK) return bail(r);
  s->io.mode = 0;
  s->io.data = s->data;
  s->io.sp = s->sp;
  s->io.ring = s->ring;
  s->io.ring_slots = s->ring_slots;
  if ((r = s->capture_graph()) != EDPC_OK) return bail(r);
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(EDPC_ECUDA, "encoder open sync"));
  *out = s;
  return EDPC_OK;
}

extern "C" int edpc_encoder_open(const edpc_cfg* cfg, const uint8_t* data, size_t len, int data_on_device,
                                 void* cuda_stream, edpc_session** out) {
  if (!out) return fail(EDPC_EINVAL, "out is NULL");
  *out = nullptr;
  EDPC_TRY(check_cfg(cfg));
  const uint64_t l = len;
  const bool tune = (cfg->flags & EDPC_FLAG_TUNE_TILES) != 0;
  return encoder_open_impl(cfg, &data, &l, 1, data_on_device, cuda_stream, nullptr, tune ? 1u : 0u, 0, tune, out);
}

extern "C" int edpc_session_run(edpc_session* s, uint64_t max_steps, int sync, uint64_t* steps_done) {
  if (!s) return fail(EDPC_EINVAL, "session is NULL");
  if (s->finished) return fail(EDPC_EINVAL, "session already finished");
  uint64_t left = s->steps_total - s->steps_run;
  uint64_t n = std::min(left, max_steps);
  EDPC_TRY(s->launch_steps(n));
  EDPC_TRY(s->join());
  if (sync) EDPC_CUDA(cudaStreamSynchronize(s->st));
  if (steps_done) *steps_done = n;
  return EDPC_OK;
}

extern "C" int edpc_session_remaining(const edpc_session* s, uint64_t* left) {
  if (!s || !left) return fail(EDPC_EINVAL, "NULL argument");
  *left = s->steps_total - s->steps_run;
  return EDPC_OK;
}

static int check_device_errors(edpc_session* s) {
  StepCtl c, c2;
  EDPC_CUDA(cudaMemcpyAsync(&c, s->model.ctl_of(0), sizeof(c), cudaMemcpyDeviceToHost, s->st));
  EDPC_CUDA(cudaMemcpyAsync(&c2, s->model.ctl_of(1), sizeof(c2), cudaMemcpyDeviceToHost, s->st));
  EDPC_CUDA(cudaStreamSynchronize(s->st));
  c.err |= c2.err;
  if (c.err & kErrTcTimeout) return fail(EDPC_ETIMEOUT, "a tensor-core GEMM wait expired");
  if (c.err) return fail(EDPC_ECUDA, "device error flags " + std::to_string(c.err));
  return EDPC_OK;
}

// Runs an encoder session to its end and flushes every coder; lens receives
// the byte count of each row's substream, dst their offsets when packed.
static int encoder_drain(edpc_session* s, std::vector<uint32_t>* lens, std::vector<unsigned long long>* dst,
                         uint64_t* total) {
  uint64_t done = 0;
  EDPC_TRY(edpc_session_run(s, UINT64_MAX, 0, &done));
  EDPC_TRY(s->code_pending());
  EDPC_TRY(s->join());
  const int b = s->b;
  cudaStream_t st = s->st;
  EDPC_CUDA(launch_encode_flush(s->es, b, s->out, s->out_off, s->out_cap, s->out_len, st));
  lens->resize(b);
  EDPC_CUDA(cudaMemcpyAsync(lens->data(), s->out_len, 4 * (size_t)b, cudaMemcpyDeviceToHost, st));
  EDPC_CUDA(cudaStreamSynchronize(st));
  EDPC_TRY(check_device_errors(s));
  *total = 0;
  dst->resize(b);
  for (int i = 0; i < b; ++i) {
    if ((*lens)[i] == 0xFFFFFFFFu) return fail(EDPC_ECUDA, "coder output buffer overflow");
    (*dst)[i] = *total;
    *total += (*lens)[i];
  }
  return EDPC_OK;
}

// Packs every row's substream (in row order) into host memory.
static int gather_payload(edpc_session* s, const std::vector<unsigned long long>& dst, uint64_t total, uint8_t* host) {
  if (!total) return EDPC_OK;
  const int b = s->b;
  cudaStream_t st = s->st;
  uint8_t* packed = nullptr;
  unsigned long long* dst_dev = nullptr;
  if (cudaMalloc(&packed, total) != cudaSuccess || cudaMalloc(&dst_dev, 8 * (size_t)b) != cudaSuccess) {
    cudaFree(packed);
    return fail(EDPC_ENOMEM, "packing buffer");
  }
  cudaMemcpyAsync(dst_dev, dst.data(), 8 * (size_t)b, cudaMemcpyHostToDevice, st);
  gather_streams_kernel<<<b, 256, 0, st>>>(s->out, s->out_off, s->out_len, dst_dev, packed);
  cudaError_t e = cudaMemcpyAsync(host, packed, total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(packed);
  cudaFree(dst_dev);
  if (e != cudaSuccess) return fail(EDPC_ECUDA, std::string("stream gather: ") + cudaGetErrorString(e));
  return EDPC_OK;
}

// Independent per-file models in one batch: one variant-2 container per file
// (the file's own streams, cfg.streams = its stream count, its bytes' checksum).
static int grouped_encoder_finish(edpc_session* s, std::vector<std::vector<uint8_t>>* members) {
  std::vector<uint32_t> len;
  std::vector<unsigned long long> dst;
  uint64_t total = 0;
  EDPC_TRY(encoder_drain(s, &len, &dst, &total));
  std::vector<uint8_t> payload(std::max<uint64_t>(total, 1));
  EDPC_TRY(gather_payload(s, dst, total, payload.data()));
  const GroupPlan& gp = s->gp;
  members->assign(gp.groups.size(), {});
  for (size_t f = 0; f < gp.groups.size(); ++f) {
    const GroupInfo& g = gp.groups[f];
    Header h;
    h.cfg = s->cfg;
    h.cfg.streams = gp.b[f];
    h.n = gp.n[f];
    h.b = gp.b[f];
    h.len.assign(len.begin() + g.r0, len.begin() + g.r0 + g.s);
    h.variant = 2;
    EDPC_TRY(device_checksum(s->data + gp.off[f], gp.n[f], s->scratch, s->st, &h.checksum));
    std::vector<uint8_t> hdr = write_header(h);
    uint64_t bytes = 0;
    for (uint32_t v : h.len) bytes += v;
    std::vector<uint8_t>& m = (*members)[f];
    m.resize(hdr.size() + bytes);
    memcpy(m.data(), hdr.data(), hdr.size());
    if (bytes) memcpy(m.data() + hdr.size(), payload.data() + dst[g.r0], bytes);
  }
  s->finished = true;
  return EDPC_OK;
}

extern "C" int edpc_encoder_finish(edpc_session* s, uint8_t** out, size_t* out_len) {
  if (!s || !out || !out_len) return fail(EDPC_EINVAL, "NULL argument");
  if (!s->encoder) return fail(EDPC_EINVAL, "not an encoder session");
  if (s->grouped) return fail(EDPC_EINVAL, "a batch of independent models finishes into an archive");
  *out = nullptr;
  *out_len = 0;
  std::vector<uint32_t> len;
  std::vector<unsigned long long> dst;
  uint64_t total = 0;
  EDPC_TRY(encoder_drain(s, &len, &dst, &total));
  Header h;
  h.cfg = s->cfg;
  h.n = s->n;
  h.b = (uint32_t)s->b;
  h.len = len;
  h.variant = s->variant;
  h.L = s->arch_L;
  h.sizes = s->file_sizes;
  h.tiles = s->tiles;
  EDPC_TRY(device_checksum(s->data, s->n, s->scratch, s->st, &h.checksum));
  std::vector<uint8_t> hdr = write_header(h);
  uint8_t* buf = static_cast<uint8_t*>(malloc(hdr.size() + total + 1));
  if (!buf) return fail(EDPC_ENOMEM, "output buffer");
  memcpy(buf, hdr.data(), hdr.size());
  int r = gather_payload(s, dst, total, buf + hdr.size());
  if (r != EDPC_OK) {
    free(buf);
    return r;
  }
  s->finished = true;
  *out = buf;
  *out_len = hdr.size() + total;
  return EDPC_OK;
}

extern "C" int edpc_peek(const uint8_t* bits, size_t bits_len, edpc_cfg* cfg, uint64_t* orig_len,
                         uint32_t* streams_eff) {
  Header h;
  EDPC_TRY(read_header(bits, bits_len, &h));
  if (cfg) *cfg = h.cfg;
  if (orig_len) *orig_len = h.n;
  if (streams_eff) *streams_eff = h.b;
  return EDPC_OK;
}

// Opens a decoder over `payload` (every row's substream, in row order; row r
// has row_len[r] bytes). lay: explicit layout (file sets), gp: independent
// models in one batch (rows and layout from gp), neither: the balanced split.
static int decoder_open_impl(const edpc_cfg& cfg, uint64_t n, const StreamLayout* lay, const GroupPlan* gp,
                             const uint8_t* payload, size_t payload_len, const std::vector<uint32_t>& row_len,
                             uint64_t checksum, const std::vector<uint8_t>& tiles, void* out_device,
                             void* cuda_stream, edpc_session** out) {
  EDPC_TRY(current_device_ok());
  edpc_session* s = new (std::nothrow) edpc_session();
  if (!s) return fail(EDPC_ENOMEM, "host allocation failed");
  auto bail = [&](int r) {
    delete s;
    return r;
  };
  s->encoder = false;
  if (gp) {
    s->gp = *gp;
    s->grouped = true;
  }
  int r = gp ? s->setup_common(cfg, n, cuda_stream, &gp->lay, &gp->groups) : s->setup_common(cfg, n, cuda_stream, lay);
  if (r != EDPC_OK) return bail(r);
  if ((r = session_prepare_events(s)) != EDPC_OK) return bail(r);
  cudaStream_t st = s->st;
  const int b = s->b;
  if ((int)row_len.size() != b) return bail(fail(EDPC_ECORRUPT, "stream table does not match the layout"));
  s->checksum_expected = checksum;
  // the encoder's GEMM tiles (they fix the accumulation layout of the replay)
  if (!tiles.empty() && (r = s->model.set_tiles(tiles.data(), (int)tiles.size())) != EDPC_OK) return bail(r);
  if (out_device) {
    s->data = static_cast<uint8_t*>(out_device);
  } else {
    if (cudaMalloc(&s->data, std::max<uint64_t>(n, 1)) != cudaSuccess) return bail(fail(EDPC_ENOMEM, "output"));
    s->own_data = true;
  }
  std::vector<unsigned long long> off(b);
  unsigned long long o = 0;
  for (int i = 0; i < b; ++i) {
    off[i] = o;
    o += row_len[i];
  }
  if (o != payload_len) return bail(fail(EDPC_ECORRUPT, "stream lengths do not match the payload"));
  if (cudaMalloc(&s->bits, std::max<size_t>(payload_len, 1)) != cudaSuccess ||
      cudaMalloc(&s->bits_off, 8 * (size_t)b) != cudaSuccess || cudaMalloc(&s->bits_len, 4 * (size_t)b) != cudaSuccess ||
      cudaMalloc(&s->ds, sizeof(DecState) * b) != cudaSuccess)
    return bail(fail(EDPC_ENOMEM, "decoder buffers"));
  if ((payload_len && cudaMemcpyAsync(s->bits, payload, payload_len, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaMemcpyAsync(s->bits_off, off.data(), 8 * (size_t)b, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->bits_len, row_len.data(), 4 * (size_t)b, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return bail(fail(EDPC_ECUDA, "decoder input copies"));
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(EDPC_ECUDA, "decoder input sync"));
  if (launch_dec_init(s->ds, s->bits, s->bits_off, s->bits_len, b, st) != cudaSuccess ||
      launch_prefix_decode(s->ds, s->bits, s->bits_off, s->bits_len, s->sp, (int)cfg.context, b, s->data, st) !=
          cudaSuccess)
    return bail(fail(EDPC_ECUDA, "decoder prefix launch"));
  long long i0 = cfg.context;
  if ((r = s->model.set_ctl_for_step((int)i0, 1, s->lay.active_at(i0), s->ring_slots, st)) != EDPC_OK) return bail(r);
  s->io.mode = 1;
  s->io.data = s->data;
  s->io.sp = s->sp;
  s->io.ring_slots = s->ring_slots;
  s->io.dec = s->ds;
  s->io.bits = s->bits;
  s->io.bits_off = s->bits_off;
  s->io.bits_len = s->bits_len;
  if ((r = s->capture_graph()) != EDPC_OK) return bail(r);
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(EDPC_ECUDA, "decoder open sync"));
  *out = s;
  return EDPC_OK;
}

// Rows of a batch of variant-2 members (each member's streams, then padding
// rows of no bytes) and their concatenated payload.
static int grouped_members_plan(const std::vector<Header>& hs, const std::vector<const uint8_t*>& payloads,
                                GroupPlan* gp, std::vector<uint8_t>* payload, std::vector<uint32_t>* row_len,
                                uint64_t* total_n) {
  std::vector<uint64_t> n(hs.size());
  std::vector<uint32_t> b(hs.size());
  *total_n = 0;
  size_t bytes = 0;
  for (size_t f = 0; f < hs.size(); ++f) {
    n[f] = hs[f].n;
    b[f] = hs[f].b;
    *total_n += hs[f].n;
    for (uint32_t v : hs[f].len) bytes += v;
  }
  EDPC_TRY(grouped_plan(n.data(), b.data(), hs.size(), gp));
  payload->resize(bytes);
  row_len->assign(gp->lay.streams(), 0);
  size_t o = 0;
  for (size_t f = 0; f < hs.size(); ++f) {
    size_t mb = 0;
    for (uint32_t s = 0; s < hs[f].b; ++s) {
      (*row_len)[gp->groups[f].r0 + s] = hs[f].len[s];
      mb += hs[f].len[s];
    }
    if (mb) memcpy(payload->data() + o, payloads[f], mb);
    o += mb;
  }
  return EDPC_OK;
}

extern "C" int edpc_decoder_open(const uint8_t* bits, size_t bits_len, void* out_device, void* cuda_stream,
                                 edpc_session** out) {
  if (!out) return fail(EDPC_EINVAL, "out is NULL");
  *out = nullptr;
  Header h;
  EDPC_TRY(read_header(bits, bits_len, &h));
  if (h.variant == 2) {
    // one file of an archive of independent models: its own model, replayed
    // by the batched engine with one group
    GroupPlan gp;
    std::vector<uint8_t> payload;
    std::vector<uint32_t> row_len;
    uint64_t n = 0;
    EDPC_TRY(grouped_members_plan({h}, {bits + h.header_len}, &gp, &payload, &row_len, &n));
    return decoder_open_impl(h.cfg, h.n, nullptr, &gp, payload.data(), payload.size(), row_len, h.checksum, {},
                             out_device, cuda_stream, out);
  }
  StreamLayout lay;
  const bool file_set = h.variant == 1 && h.L > 0;
  if (file_set) archive_split(h.sizes.data(), h.sizes.size(), h.L, &lay);
  return decoder_open_impl(h.cfg, h.n, file_set ? &lay : nullptr, nullptr, bits + h.header_len,
                           bits_len - h.header_len, h.len, h.checksum, h.tiles, out_device, cuda_stream, out);
}

extern "C" int edpc_decoder_finish(edpc_session* s, uint8_t* out_host) {
  if (!s) return fail(EDPC_EINVAL, "session is NULL");
  if (s->encoder) return fail(EDPC_EINVAL, "not a decoder session");
  uint64_t done = 0;
  EDPC_TRY(edpc_session_run(s, UINT64_MAX, 1, &done));
  EDPC_TRY(check_device_errors(s));
  uint64_t h = 0;
  EDPC_TRY(device_checksum(s->data, s->n, s->scratch, s->st, &h));
  if (h != s->checksum_expected) return fail(EDPC_ECORRUPT, "checksum of the decoded data does not match");
  if (out_host && s->n) {
    EDPC_CUDA(cudaMemcpyAsync(out_host, s->data, s->n, cudaMemcpyDeviceToHost, s->st));
    EDPC_CUDA(cudaStreamSynchronize(s->st));
  }
  s->finished = true;
  return EDPC_OK;
}

extern "C" int edpc_session_stats(const edpc_session* s, edpc_stats* o) {
  if (!s || !o) return fail(EDPC_EINVAL, "NULL argument");
  memset(o, 0, sizeof(*o));
  o->steps_run = s->steps_run;
  o->steps_total = s->steps_total;
  o->streams = (uint32_t)s->b;
  o->launches_per_step = (uint32_t)(s->graph_kernels ? s->graph_kernels : s->model.launches_per_step());
  o->fdm_samples = s->samples;
  o->fdm_fwd_ms = s->samples ? s->fwd_ms / s->samples : 0;
  o->fdm_bwd_ms = s->samples ? s->bwd_ms / s->samples : 0;
  o->fdm_adam_ms = s->samples ? s->adam_ms / s->samples : 0;
  return EDPC_OK;
}

extern "C" int edpc_session_profile(edpc_session* s, int on) {
  if (!s) return fail(EDPC_EINVAL, "session is NULL");
  if (!on && s->profiling) {
    for (int k = 0; k < edpc_session::kEvSets; ++k) EDPC_TRY(s->harvest(k));
  }
  if (on && !s->profiling) {
    s->fwd_ms = s->bwd_ms = s->adam_ms = 0;
    s->samples = 0;
  }
  s->profiling = on != 0;
  return EDPC_OK;
}

extern "C" void edpc_session_close(edpc_session* s) { delete s; }

extern "C" int edpc_compress(const uint8_t* buf, size_t len, const edpc_cfg* cfg, uint8_t** out, size_t* out_len) {
  if (!out || !out_len) return fail(EDPC_EINVAL, "NULL output pointer");
  edpc_session* s = nullptr;
  EDPC_TRY(edpc_encoder_open(cfg, buf, len, 0, nullptr, &s));
  int r = edpc_encoder_finish(s, out, out_len);
  edpc_session_close(s);
  return r;
}

extern "C" int edpc_decompress(const uint8_t* bits, size_t bits_len, uint8_t** out, size_t* out_len) {
  if (!out || !out_len) return fail(EDPC_EINVAL, "NULL output pointer");
  *out = nullptr;
  *out_len = 0;
  uint64_t n = 0;
  EDPC_TRY(edpc_peek(bits, bits_len, nullptr, &n, nullptr));
  uint8_t* buf = static_cast<uint8_t*>(malloc(std::max<uint64_t>(n, 1)));
  if (!buf) return fail(EDPC_ENOMEM, "output buffer");
  edpc_session* s = nullptr;
  int r = edpc_decoder_open(bits, bits_len, nullptr, nullptr, &s);
  if (r == EDPC_OK) r = edpc_decoder_finish(s, buf);
  edpc_session_close(s);
  if (r != EDPC_OK) {
    free(buf);
    return r;
  }
  *out = buf;
  *out_len = n;
  return EDPC_OK;
}

// ==========================================================================================
// file sets (archives)
// ==========================================================================================
static int plan_file_set(const size_t* lens, size_t nfiles, const edpc_cfg* cfg, edpc_split_plan* plan,
                         std::vector<uint64_t>* sizes) {
  if (!lens && nfiles) return fail(EDPC_EINVAL, "lens is NULL");
  EDPC_TRY(check_cfg(cfg, true));
  sizes->assign(lens, lens + nfiles);
  memset(plan, 0, sizeof(*plan));
  uint64_t L = 0;
  if (cfg->streams > 0) {
    L = archive_stream_len(sizes->data(), nfiles, cfg->streams);
  } else {
    EDPC_TRY(current_device_ok());
    TunedPlan tp;
    EDPC_TRY(archive_autotune(*cfg, sizes->data(), nfiles, &tp));
    L = tp.L;
    plan->est_seconds = tp.est_seconds;
    plan->step_ms_t0 = tp.step_ms_t0;
    plan->step_ms_per_stream = tp.step_ms_per_stream;
  }
  const uint64_t b = archive_stream_count(sizes->data(), nfiles, L);
  if (b > kMaxStreams) return fail(EDPC_EINVAL, "the file set needs more than 65535 streams");
  plan->stream_len = L;
  plan->streams = (uint32_t)b;
  return EDPC_OK;
}

extern "C" int edpc_archive_plan(const size_t* lens, size_t nfiles, const edpc_cfg* cfg, edpc_split_plan* plan) {
  if (!plan) return fail(EDPC_EINVAL, "plan is NULL");
  std::vector<uint64_t> sizes;
  return plan_file_set(lens, nfiles, cfg, plan, &sizes);
}

extern "C" int edpc_encoder_open_many(const edpc_cfg* cfg, const uint8_t* const* bufs, const size_t* lens,
                                      size_t nfiles, int data_on_device, void* cuda_stream, edpc_session** out) {
  if (!out) return fail(EDPC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!bufs && nfiles) return fail(EDPC_EINVAL, "bufs is NULL");
  edpc_split_plan plan;
  std::vector<uint64_t> sizes;
  EDPC_TRY(plan_file_set(lens, nfiles, cfg, &plan, &sizes));
  StreamLayout lay;
  archive_split(sizes.data(), nfiles, plan.stream_len, &lay);
  edpc_cfg c = *cfg;
  std::vector<const uint8_t*> parts(bufs, bufs + nfiles);
  return encoder_open_impl(&c, parts.data(), sizes.data(), nfiles, data_on_device, cuda_stream, &lay, 1u,
                           plan.stream_len, true, out);
}

extern "C" int edpc_compress_many(const uint8_t* const* bufs, const size_t* lens, size_t nfiles, const edpc_cfg* cfg,
                                  uint8_t** out, size_t* out_len) {
  if (!out || !out_len) return fail(EDPC_EINVAL, "NULL output pointer");
  edpc_session* s = nullptr;
  EDPC_TRY(edpc_encoder_open_many(cfg, bufs, lens, nfiles, 0, nullptr, &s));
  int r = edpc_encoder_finish(s, out, out_len);
  edpc_session_close(s);
  return r;
}

extern "C" int edpc_archive_info(const uint8_t* bits, size_t bits_len, uint64_t* nfiles, uint64_t* sizes) {
  if (!nfiles) return fail(EDPC_EINVAL, "nfiles is NULL");
  Header h;
  EDPC_TRY(read_header(bits, bits_len, &h));
  if (h.variant == 1 && h.L > 0) {
    *nfiles = h.sizes.size();
    if (sizes) memcpy(sizes, h.sizes.data(), 8 * h.sizes.size());
  } else {
    *nfiles = 1;
    if (sizes) sizes[0] = h.n;
  }
  return EDPC_OK;
}

extern "C" int edpc_decompress_many(const uint8_t* bits, size_t bits_len, uint8_t*** outs, size_t** lens,
                                    size_t* nfiles) {
  if (!outs || !lens || !nfiles) return fail(EDPC_EINVAL, "NULL output pointer");
  *outs = nullptr;
  *lens = nullptr;
  *nfiles = 0;
  uint64_t nf = 0;
  EDPC_TRY(edpc_archive_info(bits, bits_len, &nf, nullptr));
  std::vector<uint64_t> sizes(nf);
  EDPC_TRY(edpc_archive_info(bits, bits_len, &nf, sizes.data()));
  uint64_t total = 0;
  for (uint64_t v : sizes) total += v;
  // one block: nf pointers, then the files' bytes back to back
  const size_t head = sizeof(uint8_t*) * (size_t)std::max<uint64_t>(nf, 1);
  uint8_t* block = static_cast<uint8_t*>(malloc(head + std::max<uint64_t>(total, 1)));
  size_t* ls = static_cast<size_t*>(malloc(sizeof(size_t) * (size_t)std::max<uint64_t>(nf, 1)));
  if (!block || !ls) {
    free(block);
    free(ls);
    return fail(EDPC_ENOMEM, "output buffers");
  }
  uint8_t* data = block + head;
  edpc_session* s = nullptr;
  int r = edpc_decoder_open(bits, bits_len, nullptr, nullptr, &s);
  if (r == EDPC_OK) r = edpc_decoder_finish(s, data);
  edpc_session_close(s);
  if (r != EDPC_OK) {
    free(block);
    free(ls);
    return r;
  }
  uint8_t** ptrs = reinterpret_cast<uint8_t**>(block);
  uint64_t o = 0;
  for (uint64_t f = 0; f < nf; ++f) {
    ptrs[f] = data + o;
    ls[f] = (size_t)sizes[f];
    o += sizes[f];
  }
  *outs = ptrs;
  *lens = ls;
  *nfiles = (size_t)nf;
  return EDPC_OK;
}

// ==========================================================================================
// archives of independent per-file models
// ==========================================================================================
// Layout: "EDPI", u32 format version, u64 file count, u64 stream length L,
// then per file (u64 member offset, u64 member bytes, u64 file bytes), a
// CRC-32 of everything before it, then the members: member f is the
// single-input container edpc_compress gives for file f with cfg.streams =
// max(1, ceil(n_f / L)).
namespace {

constexpr uint32_t kIndepMagic = 0x49504445u;  // "EDPI"
constexpr int kIndepChunk = 128;                // model steps queued per session and round

struct IndepTable {
  uint64_t nfiles = 0, L = 0;
  std::vector<uint64_t> off, bytes, size;
  size_t header_len = 0;
};

size_t indep_header_len(uint64_t nfiles) { return 24 + 24 * (size_t)nfiles + 4; }

int read_indep(const uint8_t* p, size_t n, IndepTable* t) {
  if (!p || n < 28) return fail(EDPC_ECORRUPT, "archive too short");
  if (get<uint32_t>(p, 0) != kIndepMagic) return fail(EDPC_ECORRUPT, "not an archive of independent models");
  if (get<uint32_t>(p, 4) != EDPC_FORMAT_VERSION) return fail(EDPC_EVERSION, "unsupported format version");
  t->nfiles = get<uint64_t>(p, 8);
  t->L = get<uint64_t>(p, 16);
  if (t->nfiles > (n - 28) / 24) return fail(EDPC_ECORRUPT, "archive file table truncated");
  t->header_len = indep_header_len(t->nfiles);
  if (crc32_ieee(p, t->header_len - 4) != get<uint32_t>(p, t->header_len - 4))
    return fail(EDPC_ECORRUPT, "archive header CRC mismatch");
  t->off.resize(t->nfiles);
  t->bytes.resize(t->nfiles);
  t->size.resize(t->nfiles);
  for (uint64_t f = 0; f < t->nfiles; ++f) {
    t->off[f] = get<uint64_t>(p, 24 + 24 * f);
    t->bytes[f] = get<uint64_t>(p, 32 + 24 * f);
    t->size[f] = get<uint64_t>(p, 40 + 24 * f);
    if (t->off[f] < t->header_len || t->off[f] > n || t->bytes[f] > n - t->off[f])
      return fail(EDPC_ECORRUPT, "archive member out of range");
  }
  return EDPC_OK;
}

uint32_t indep_streams(uint64_t n, uint64_t L) {
  const uint64_t b = (n + L - 1) / L;
  return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(b, 1), kMaxStreams);
}

// Independent models run as one batch (the grouped engine) in BF16 with
// Algorithm 1's schedule; other precisions and schedules run one session per
// file, several at a time.
bool batched_independent(const edpc_cfg& c) {
  return c.precision == EDPC_BF16 && !(c.flags & (EDPC_FLAG_DELAYED_UPDATE | EDPC_FLAG_OVERLAP_FDM));
}

// Runs the sessions of `count` jobs, at most `conc` at a time, each on its
// own CUDA stream: open(j, stream, &s) opens job j's session, done(j, s)
// finishes it. Every round queues kIndepChunk model steps on each open
// session; a session whose steps are all queued is finished (which waits for
// its own stream only) and its slot reopened on the next job.
template <class Open, class Done>
int run_concurrent(size_t count, uint32_t conc, Open open, Done done) {
  if (conc == 0) conc = 8;
  conc = (uint32_t)std::min<size_t>(conc, std::max<size_t>(count, 1));
  std::vector<cudaStream_t> sts(conc, nullptr);
  std::vector<edpc_session*> ss(conc, nullptr);
  std::vector<size_t> job(conc, 0);
  int r = EDPC_OK;
  for (auto& st : sts)
    if (r == EDPC_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      r = fail(EDPC_ECUDA, "stream creation");
  size_t next = 0, finished = 0;
  while (r == EDPC_OK && finished < count) {
    for (uint32_t k = 0; k < conc && r == EDPC_OK; ++k)
      if (!ss[k] && next < count) {
        job[k] = next++;
        r = open(job[k], sts[k], &ss[k]);
      }
    for (uint32_t k = 0; k < conc && r == EDPC_OK; ++k) {
      if (!ss[k]) continue;
      uint64_t left = 0;
      r = edpc_session_remaining(ss[k], &left);
      if (r == EDPC_OK && left > 0) r = edpc_session_run(ss[k], kIndepChunk, 0, nullptr);
    }
    for (uint32_t k = 0; k < conc && r == EDPC_OK; ++k) {
      if (!ss[k]) continue;
      uint64_t left = 1;
      r = edpc_session_remaining(ss[k], &left);
      if (r == EDPC_OK && left == 0) {
        r = done(job[k], ss[k]);
        edpc_session_close(ss[k]);
        ss[k] = nullptr;
        ++finished;
      }
    }
  }
  for (uint32_t k = 0; k < conc; ++k) {
    if (ss[k]) edpc_session_close(ss[k]);
    if (sts[k]) cudaStreamDestroy(sts[k]);
  }
  return r;
}

}  // namespace

extern "C" int edpc_compress_independent(const uint8_t* const* bufs, const size_t* lens, size_t nfiles,
                                         const edpc_cfg* cfg, uint64_t stream_len, uint32_t concurrency,
                                         uint8_t** out, size_t* out_len) {
  if (!out || !out_len) return fail(EDPC_EINVAL, "NULL output pointer");
  *out = nullptr;
  *out_len = 0;
  if ((!bufs || !lens) && nfiles) return fail(EDPC_EINVAL, "bufs or lens is NULL");
  if (stream_len == 0) return fail(EDPC_EINVAL, "stream_len must be > 0");
  edpc_cfg c0 = *cfg;
  c0.streams = 1;
  EDPC_TRY(check_cfg(&c0));
  for (size_t f = 0; f < nfiles; ++f)
    if (!bufs[f] && lens[f]) return fail(EDPC_EINVAL, "data is NULL");
  EDPC_TRY(current_device_ok());
  std::vector<std::vector<uint8_t>> members(nfiles);
  if (batched_independent(*cfg) && nfiles) {
    // BF16: every file's model in one batch (grouped engine), one session
    std::vector<uint64_t> sz(lens, lens + nfiles);
    std::vector<uint32_t> bs(nfiles);
    for (size_t f = 0; f < nfiles; ++f) {
      edpc_cfg c = *cfg;
      c.streams = indep_streams(lens[f], stream_len);
      bs[f] = (uint32_t)effective_streams(c, lens[f]);
    }
    GroupPlan gp;
    EDPC_TRY(grouped_plan(sz.data(), bs.data(), nfiles, &gp));
    edpc_session* s = nullptr;
    EDPC_TRY(encoder_open_impl(&c0, bufs, sz.data(), nfiles, 0, nullptr, nullptr, 2, 0, false, &s, &gp));
    int r = grouped_encoder_finish(s, &members);
    edpc_session_close(s);
    EDPC_TRY(r);
  } else {
    auto open = [&](size_t f, cudaStream_t st, edpc_session** s) {
      edpc_cfg c = *cfg;
      c.streams = indep_streams(lens[f], stream_len);
      return edpc_encoder_open(&c, bufs[f], lens[f], 0, st, s);
    };
    auto done = [&](size_t f, edpc_session* s) {
      uint8_t* b = nullptr;
      size_t n = 0;
      EDPC_TRY(edpc_encoder_finish(s, &b, &n));
      members[f].assign(b, b + n);
      free(b);
      return EDPC_OK;
    };
    EDPC_TRY(run_concurrent(nfiles, concurrency, open, done));
  }
  const size_t hl = indep_header_len(nfiles);
  size_t total = hl;
  for (auto& m : members) total += m.size();
  std::vector<uint8_t> hdr(hl, 0);
  put<uint32_t>(hdr, 0, kIndepMagic);
  put<uint32_t>(hdr, 4, EDPC_FORMAT_VERSION);
  put<uint64_t>(hdr, 8, (uint64_t)nfiles);
  put<uint64_t>(hdr, 16, stream_len);
  uint64_t o = hl;
  for (size_t f = 0; f < nfiles; ++f) {
    put<uint64_t>(hdr, 24 + 24 * f, o);
    put<uint64_t>(hdr, 32 + 24 * f, (uint64_t)members[f].size());
    put<uint64_t>(hdr, 40 + 24 * f, (uint64_t)lens[f]);
    o += members[f].size();
  }
  put<uint32_t>(hdr, hl - 4, crc32_ieee(hdr.data(), hl - 4));
  uint8_t* buf = static_cast<uint8_t*>(malloc(total));
  if (!buf) return fail(EDPC_ENOMEM, "output buffer");
  memcpy(buf, hdr.data(), hl);
  o = hl;
  for (auto& m : members) {
    if (!m.empty()) memcpy(buf + o, m.data(), m.size());
    o += m.size();
  }
  *out = buf;
  *out_len = total;
  return EDPC_OK;
}

extern "C" int edpc_independent_info(const uint8_t* bits, size_t bits_len, uint64_t* nfiles, uint64_t* sizes) {
  if (!nfiles) return fail(EDPC_EINVAL, "nfiles is NULL");
  IndepTable t;
  EDPC_TRY(read_indep(bits, bits_len, &t));
  *nfiles = t.nfiles;
  if (sizes && t.nfiles) memcpy(sizes, t.size.data(), 8 * (size_t)t.nfiles);
  return EDPC_OK;
}

extern "C" int edpc_decompress_member(const uint8_t* bits, size_t bits_len, uint64_t index, uint8_t** out,
                                      size_t* out_len) {
  if (!out || !out_len) return fail(EDPC_EINVAL, "NULL output pointer");
  IndepTable t;
  EDPC_TRY(read_indep(bits, bits_len, &t));
  if (index >= t.nfiles) return fail(EDPC_EINVAL, "member index out of range");
  uint64_t n = 0;
  EDPC_TRY(edpc_peek(bits + t.off[index], t.bytes[index], nullptr, &n, nullptr));
  if (n != t.size[index]) return fail(EDPC_ECORRUPT, "member length does not match the file table");
  return edpc_decompress(bits + t.off[index], t.bytes[index], out, out_len);
}

// Decodes every variant-2 member of an archive in one batched session and
// checks each member's data checksum.
static int grouped_decode_all(const std::vector<Header>& hs, const uint8_t* bits, const IndepTable& t,
                              uint8_t** outs) {
  std::vector<const uint8_t*> pl(hs.size());
  for (size_t f = 0; f < hs.size(); ++f) pl[f] = bits + t.off[f] + hs[f].header_len;
  GroupPlan gp;
  std::vector<uint8_t> payload;
  std::vector<uint32_t> row_len;
  uint64_t n = 0;
  EDPC_TRY(grouped_members_plan(hs, pl, &gp, &payload, &row_len, &n));
  edpc_session* s = nullptr;
  EDPC_TRY(decoder_open_impl(hs[0].cfg, n, nullptr, &gp, payload.data(), payload.size(), row_len, 0, {}, nullptr,
                             nullptr, &s));
  uint64_t done = 0;
  int r = edpc_session_run(s, UINT64_MAX, 1, &done);
  if (r == EDPC_OK) r = check_device_errors(s);
  for (size_t f = 0; f < hs.size() && r == EDPC_OK; ++f) {
    uint64_t h = 0;
    r = device_checksum(s->data + gp.off[f], gp.n[f], s->scratch, s->st, &h);
    if (r == EDPC_OK && h != hs[f].checksum) r = fail(EDPC_ECORRUPT, "checksum of a decoded member does not match");
    if (r == EDPC_OK && gp.n[f] && cudaMemcpy(outs[f], s->data + gp.off[f], gp.n[f], cudaMemcpyDeviceToHost) !=
                                       cudaSuccess)
      r = fail(EDPC_ECUDA, "member copy");
  }
  if (r == EDPC_OK) s->finished = true;
  edpc_session_close(s);
  return r;
}

extern "C" int edpc_decompress_independent(const uint8_t* bits, size_t bits_len, uint32_t concurrency,
                                           uint8_t*** outs, size_t** lens, size_t* nfiles) {
  if (!outs || !lens || !nfiles) return fail(EDPC_EINVAL, "NULL output pointer");
  *outs = nullptr;
  *lens = nullptr;
  *nfiles = 0;
  IndepTable t;
  EDPC_TRY(read_indep(bits, bits_len, &t));
  for (uint64_t f = 0; f < t.nfiles; ++f) {
    uint64_t n = 0;
    EDPC_TRY(edpc_peek(bits + t.off[f], t.bytes[f], nullptr, &n, nullptr));
    if (n != t.size[f]) return fail(EDPC_ECORRUPT, "member length does not match the file table");
  }
  uint64_t total = 0;
  for (uint64_t v : t.size) total += v;
  const size_t head = sizeof(uint8_t*) * (size_t)std::max<uint64_t>(t.nfiles, 1);
  uint8_t* block = static_cast<uint8_t*>(malloc(head + std::max<uint64_t>(total, 1)));
  size_t* ls = static_cast<size_t*>(malloc(sizeof(size_t) * (size_t)std::max<uint64_t>(t.nfiles, 1)));
  if (!block || !ls) {
    free(block);
    free(ls);
    return fail(EDPC_ENOMEM, "output buffers");
  }
  uint8_t** ptrs = reinterpret_cast<uint8_t**>(block);
  uint64_t o = 0;
  for (uint64_t f = 0; f < t.nfiles; ++f) {
    ptrs[f] = block + head + o;
    ls[f] = (size_t)t.size[f];
    o += t.size[f];
  }
  int r = EDPC_OK;
  // members of the batched engine with one configuration decode as one batch
  std::vector<Header> hs(t.nfiles);
  bool batch = t.nfiles > 0;
  for (uint64_t f = 0; f < t.nfiles && r == EDPC_OK; ++f) {
    r = read_header(bits + t.off[f], t.bytes[f], &hs[f]);
    const edpc_cfg& a = hs[f].cfg;
    const edpc_cfg& z = hs[0].cfg;
    batch = batch && hs[f].variant == 2 && a.context == z.context && a.embed_dim == z.embed_dim &&
            a.latent == z.latent && a.hidden == z.hidden && a.blocks == z.blocks && a.branches == z.branches &&
            a.lr == z.lr && a.seed == z.seed && a.precision == z.precision && a.flags == z.flags;
  }
  if (r == EDPC_OK && batch) {
    r = grouped_decode_all(hs, bits, t, ptrs);
  } else if (r == EDPC_OK && t.nfiles) {
    r = current_device_ok();
    auto open = [&](size_t f, cudaStream_t st, edpc_session** s) {
      return edpc_decoder_open(bits + t.off[f], t.bytes[f], nullptr, st, s);
    };
    auto done = [&](size_t f, edpc_session* s) { return edpc_decoder_finish(s, ptrs[f]); };
    if (r == EDPC_OK) r = run_concurrent((size_t)t.nfiles, concurrency, open, done);
  }
  if (r != EDPC_OK) {
    free(block);
    free(ls);
    return r;
  }
  *outs = ptrs;
  *lens = ls;
  *nfiles = (size_t)t.nfiles;
  return EDPC_OK;
}

// ==========================================================================================
// single-kernel entry points
// ==========================================================================================
extern "C" int edpc_cdf_quantize(const float* p, uint32_t rows, uint32_t* freq, uint32_t* cum, void* stream) {
  if ((!p || !freq || !cum) && rows) return fail(EDPC_EINVAL, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EDPC_CUDA(launch_cdf_quantize(p, (int)rows, freq, cum, st));
  EDPC_CUDA(cudaStreamSynchronize(st));
  return EDPC_OK;
}

extern "C" int edpc_range_encode(const uint32_t* sym, uint32_t nsym, uint32_t streams, uint8_t* out, uint32_t cap,
                                 uint32_t* out_len, void* stream) {
  if (!sym || !out || !out_len || streams == 0) return fail(EDPC_EINVAL, "NULL argument or no streams");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EncState* es = nullptr;
  unsigned long long* off = nullptr;
  uint32_t* caps = nullptr;
  std::vector<unsigned long long> h_off(streams);
  std::vector<uint32_t> h_cap(streams, cap);
  for (uint32_t s = 0; s < streams; ++s) h_off[s] = (unsigned long long)s * cap;
  int r = EDPC_OK;
  if (cudaMalloc(&es, sizeof(EncState) * streams) != cudaSuccess || cudaMalloc(&off, 8 * (size_t)streams) != cudaSuccess ||
      cudaMalloc(&caps, 4 * (size_t)streams) != cudaSuccess) {
    r = fail(EDPC_ENOMEM, "coder state");
  } else {
    cudaMemcpyAsync(off, h_off.data(), 8 * (size_t)streams, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(caps, h_cap.data(), 4 * (size_t)streams, cudaMemcpyHostToDevice, st);
    Split none{0, 0, 0};
    cudaError_t e = launch_prefix_encode(es, nullptr, none, 0, (int)streams, out, off, caps, st);
    if (e == cudaSuccess) e = launch_range_encode(es, sym, (int)nsym, 0, (int)nsym, (int)streams, out, off, caps, st);
    if (e == cudaSuccess) e = launch_encode_flush(es, (int)streams, out, off, caps, out_len, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = fail(EDPC_ECUDA, std::string("range encode: ") + cudaGetErrorString(e));
    if (r == EDPC_OK) {
      std::vector<uint32_t> l(streams);
      cudaMemcpy(l.data(), out_len, 4 * (size_t)streams, cudaMemcpyDeviceToHost);
      bool over = false;
      for (auto& v : l)
        if (v == 0xFFFFFFFFu) {
          v = cap;
          over = true;
        }
      if (over) {
        cudaMemcpy(out_len, l.data(), 4 * (size_t)streams, cudaMemcpyHostToDevice);
        r = fail(EDPC_EINVAL, "a stream needs more than cap bytes");
      }
    }
  }
  cudaFree(es);
  cudaFree(off);
  cudaFree(caps);
  return r;
}

// ==========================================================================================
// model API
// ==========================================================================================
struct edpc_model {
  Model m;
  edpc_cfg cfg{};
  uint8_t* tgt = nullptr;
  uint8_t* act = nullptr;
  uint32_t t = 0;
  ~edpc_model() {
    cudaFree(tgt);
    cudaFree(act);
  }
};

extern "C" int edpc_model_create(const edpc_cfg* cfg, uint32_t streams, edpc_model** out) {
  if (!out) return fail(EDPC_EINVAL, "out is NULL");
  *out = nullptr;
  EDPC_TRY(check_cfg(cfg));
  if (streams < 1 || streams > kMaxStreams) return fail(EDPC_EINVAL, "streams must be in [1, 65535]");
  if (cfg->flags & EDPC_FLAG_DELAYED_UPDATE)
    return fail(EDPC_EINVAL, "the model API runs Algorithm 1's schedule (no EDPC_FLAG_DELAYED_UPDATE)");
  EDPC_TRY(current_device_ok());
  edpc_model* m = new (std::nothrow) edpc_model();
  if (!m) return fail(EDPC_ENOMEM, "host allocation failed");
  m->cfg = *cfg;
  int r = m->m.init(*cfg, (int)streams);
  if (r == EDPC_OK && (cudaMalloc(&m->tgt, streams) != cudaSuccess || cudaMalloc(&m->act, streams) != cudaSuccess))
    r = fail(EDPC_ENOMEM, "model buffers");
  if (r != EDPC_OK) {
    delete m;
    return r;
  }
  *out = m;
  return EDPC_OK;
}

extern "C" void edpc_model_destroy(edpc_model* m) { delete m; }

extern "C" int edpc_model_get_state(const edpc_model* mm, float* shared, float* fdm, float* m_shared, float* v_shared,
                                    float* m_fdm, float* v_fdm, uint32_t* t) {
  if (!mm) return fail(EDPC_EINVAL, "model is NULL");
  const Model& m = mm->m;
  const size_t np = m.nparam * 4, nf = (size_t)m.d.b * m.d.Fp * m.d.Fp * 4;
  EDPC_CUDA(cudaDeviceSynchronize());
  if (shared) EDPC_CUDA(cudaMemcpy(shared, m.P, np, cudaMemcpyDeviceToHost));
  if (m_shared) EDPC_CUDA(cudaMemcpy(m_shared, m.M, np, cudaMemcpyDeviceToHost));
  if (v_shared) EDPC_CUDA(cudaMemcpy(v_shared, m.V, np, cudaMemcpyDeviceToHost));
  if (fdm) EDPC_CUDA(cudaMemcpy(fdm, m.U, nf, cudaMemcpyDeviceToHost));
  if (m_fdm) EDPC_CUDA(cudaMemcpy(m_fdm, m.Um, nf, cudaMemcpyDeviceToHost));
  if (v_fdm) EDPC_CUDA(cudaMemcpy(v_fdm, m.Uv, nf, cudaMemcpyDeviceToHost));
  if (t) *t = mm->t;
  return EDPC_OK;
}

extern "C" int edpc_model_set_state(edpc_model* mm, const float* shared, const float* fdm, const float* m_shared,
                                    const float* v_shared, const float* m_fdm, const float* v_fdm, uint32_t t) {
  if (!mm) return fail(EDPC_EINVAL, "model is NULL");
  Model& m = mm->m;
  const size_t np = m.nparam * 4, nf = (size_t)m.d.b * m.d.Fp * m.d.Fp * 4;
  if (shared) EDPC_CUDA(cudaMemcpy(m.P, shared, np, cudaMemcpyHostToDevice));
  if (m_shared) EDPC_CUDA(cudaMemcpy(m.M, m_shared, np, cudaMemcpyHostToDevice));
  if (v_shared) EDPC_CUDA(cudaMemcpy(m.V, v_shared, np, cudaMemcpyHostToDevice));
  if (fdm) EDPC_CUDA(cudaMemcpy(m.U, fdm, nf, cudaMemcpyHostToDevice));
  if (m_fdm) EDPC_CUDA(cudaMemcpy(m.Um, m_fdm, nf, cudaMemcpyHostToDevice));
  if (v_fdm) EDPC_CUDA(cudaMemcpy(m.Uv, v_fdm, nf, cudaMemcpyHostToDevice));
  mm->t = t;
  if (shared && m.precision != EDPC_FP32) {
    EDPC_TRY(m.refresh_bf16_weights(0));
    EDPC_CUDA(cudaDeviceSynchronize());
  }
  return EDPC_OK;
}

static int model_prepare(edpc_model* mm, const uint8_t* ctx, const uint8_t* targets, const uint8_t* active,
                         uint32_t t, Model::StepIO* io) {
  Model& m = mm->m;
  const int b = m.d.b;
  std::vector<uint8_t> zeros(b, 0), ones(b, 1);
  EDPC_CUDA(cudaMemcpy(m.ctx, ctx, (size_t)b * m.d.K, cudaMemcpyHostToDevice));
  EDPC_CUDA(cudaMemcpy(mm->tgt, targets ? targets : zeros.data(), b, cudaMemcpyHostToDevice));
  // a forward pass without a mask predicts for every stream
  EDPC_CUDA(cudaMemcpy(mm->act, active ? active : ones.data(), b, cudaMemcpyHostToDevice));
  int bact = 0;
  for (int i = 0; i < b; ++i) bact += active ? active[i] != 0 : 1;
  EDPC_TRY(m.set_ctl_for_step(0, (int)t, bact, 1, 0));
  io->mode = 2;
  io->targets = mm->tgt;
  io->active = mm->act;
  io->advance = false;
  io->ring_slots = 1;
  return EDPC_OK;
}

extern "C" int edpc_model_forward(edpc_model* mm, const uint8_t* ctx, float* logits, float* probs) {
  if (!mm || !ctx) return fail(EDPC_EINVAL, "NULL argument");
  Model::StepIO io;
  EDPC_TRY(model_prepare(mm, ctx, nullptr, nullptr, mm->t + 1, &io));
  Model& m = mm->m;
  EDPC_TRY(m.forward(io, 0));
  EDPC_TRY(m.head(io, 0));
  EDPC_CUDA(cudaDeviceSynchronize());
  const size_t nb = (size_t)m.d.b * 256 * 4;
  if (logits) EDPC_CUDA(cudaMemcpy(logits, m.z, nb, cudaMemcpyDeviceToHost));
  if (probs) EDPC_CUDA(cudaMemcpy(probs, m.p, nb, cudaMemcpyDeviceToHost));
  return EDPC_OK;
}

extern "C" int edpc_model_backward(edpc_model* mm, const uint8_t* ctx, const uint8_t* targets, const uint8_t* active,
                                   float* g_shared, float* g_fdm) {
  if (!mm || !ctx || !targets || !active) return fail(EDPC_EINVAL, "NULL argument");
  Model& m = mm->m;
  if (!m.gU) {
    size_t nf = (size_t)m.d.b * m.d.Fp * m.d.Fp * 4;
    if (cudaMalloc(&m.gU, nf) != cudaSuccess) return fail(EDPC_ENOMEM, "FDM gradient buffer");
  }
  Model::StepIO io;
  EDPC_TRY(model_prepare(mm, ctx, targets, active, mm->t + 1, &io));
  io.update = 0;
  EDPC_TRY(m.forward(io, 0));
  EDPC_TRY(m.head(io, 0));
  EDPC_TRY(m.backward(io, 0));
  EDPC_CUDA(cudaDeviceSynchronize());
  if (g_shared) EDPC_CUDA(cudaMemcpy(g_shared, m.G, m.nparam * 4, cudaMemcpyDeviceToHost));
  if (g_fdm) EDPC_CUDA(cudaMemcpy(g_fdm, m.gU, (size_t)m.d.b * m.d.Fp * m.d.Fp * 4, cudaMemcpyDeviceToHost));
  return EDPC_OK;
}

extern "C" int edpc_model_train_step(edpc_model* mm, const uint8_t* ctx, const uint8_t* targets, const uint8_t* active) {
  if (!mm || !ctx || !targets || !active) return fail(EDPC_EINVAL, "NULL argument");
  Model& m = mm->m;
  Model::StepIO io;
  EDPC_TRY(model_prepare(mm, ctx, targets, active, mm->t + 1, &io));
  io.update = 1;
  EDPC_TRY(m.step(io, 0));
  EDPC_TRY(m.flush(0));
  EDPC_CUDA(cudaDeviceSynchronize());
  mm->t += 1;
  return EDPC_OK;
}

extern "C" int edpc_model_set_tiles(edpc_model* mm, const uint8_t* codes, uint32_t n) {
  if (!mm) return fail(EDPC_EINVAL, "model is NULL");
  EDPC_TRY(mm->m.set_tiles(codes, (int)n));
  return EDPC_OK;
}

extern "C" int edpc_model_time_gemms(edpc_model* mm, uint32_t reps, double* ms, double* flop, double* bytes,
                                     uint32_t cap, uint32_t* n) {
  if (!mm || !ms || !flop) return fail(EDPC_EINVAL, "NULL argument");
  const uint32_t k = std::min(cap, (uint32_t)TcPlan::kMaxSites);
  EDPC_TRY(mm->m.time_sites(0, (int)reps, ms, flop, bytes, (int)k));
  EDPC_CUDA(cudaDeviceSynchronize());
  if (n) *n = k;
  return EDPC_OK;
}

extern "C" int edpc_model_block_io(edpc_model* mm, uint32_t block, float* s_in, float* s_out) {
  if (!mm || !s_in || !s_out) return fail(EDPC_EINVAL, "NULL argument");
  Model& m = mm->m;
  if (block >= (uint32_t)m.d.n) return fail(EDPC_EINVAL, "block out of range");
  // residual-stream stages: blocks before the LTE read S[j], the others S[j + 1]
  const int in = (int)block < m.d.nloc ? (int)block : (int)block + 1;
  const size_t bytes = (size_t)m.d.b * m.d.F * sizeof(float);
  EDPC_CUDA(cudaDeviceSynchronize());
  EDPC_CUDA(cudaMemcpy(s_in, m.S[in], bytes, cudaMemcpyDeviceToHost));
  EDPC_CUDA(cudaMemcpy(s_out, m.S[in + 1], bytes, cudaMemcpyDeviceToHost));
  return EDPC_OK;
}

extern "C" int edpc_model_tune_tiles(edpc_model* mm, uint8_t* codes, uint32_t cap, uint32_t* n) {
  if (!mm) return fail(EDPC_EINVAL, "model is NULL");
  EDPC_TRY(mm->m.tune_tiles(0));
  EDPC_CUDA(cudaDeviceSynchronize());
  const uint32_t k = (uint32_t)TcPlan::kMaxSites;
  if (codes) memcpy(codes, mm->m.tile_code, std::min(cap, k));
  if (n) *n = k;
  return EDPC_OK;
}
