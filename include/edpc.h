/*
 * edpc.h - C ABI of the GB300-native EDPC compressor.
 *
 * EDPC ("Accelerating Lossless Compression via Lightweight Probability
 * Models and Decoupled Parallel Dataflow", ACM MM 2025) is an autoregressive
 * lossless byte compressor. Algorithm 1 codes each byte x_i with arithmetic
 * coding under Pr(i) = Model(x_{i-t..i-1}) and then takes one Adam step on
 * the cross-entropy (Sec. 2.1, Eqs. 1-2). The decoder replays the same
 * loop on the decoded bytes. The model (Sec. 3) is a byte embedding,
 * Multi-path Byte Refinement Blocks (MBRB, Sec. 3.1.2, Eqs. 9-13), and a
 * Latent Transformation Engine (LTE, Sec. 3.2, Eqs. 14-16) whose Feature
 * Distribution Matrix U is learned per stream. The input is split into b
 * streams that advance one byte per step together (Sec. 3.3). The model
 * stage and the coder stage run as a decoupled pipeline (DPCA, Sec. 3.3).
 *
 * Conventions for every entry point:
 *   - Return 0 (EDPC_OK) on success, else one of the EDPC_E* codes.
 *     edpc_strerror() names each code, and edpc_last_error() gives the
 *     detail of the last failure on the calling thread.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the current device. Input buffers are borrowed and
 *     never written. Buffers the library allocates for the caller are
 *     released with edpc_free().
 *   - All floating-point tensors are FP32, row-major, densely packed.
 *   - A NULL cuda_stream means the library's own stream. Calls return after
 *     their GPU work has completed unless stated otherwise.
 *   - Failures never leave a GPU wait spinning: every device-side wait is
 *     bounded and reports EDPC_ETIMEOUT.
 */
#ifndef EDPC_H
#define EDPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EDPC_ABI_VERSION 1u
#define EDPC_FORMAT_VERSION 1u

/* Status codes. */
#define EDPC_OK 0
#define EDPC_EINVAL 1    /* bad argument or configuration */
#define EDPC_ENOMEM 2    /* host or device allocation failed */
#define EDPC_ECORRUPT 3  /* bad magic, CRC, length or coder state in a bitstream */
#define EDPC_EVERSION 4  /* bitstream format version not supported */
#define EDPC_ECUDA 5     /* a CUDA runtime or driver call failed */
#define EDPC_ETIMEOUT 6  /* a bounded device-side wait expired */
#define EDPC_EARCH 7     /* bitstream was made by a GEMM, precision or schedule variant this
                            library version lacks */

/* Arithmetic of the model's GEMMs. Softmax, CDF quantization, optimizer
 * state and the FDM stay FP32 in every mode. */
#define EDPC_FP32 0u     /* plain FP32 (SIMT) GEMMs */
#define EDPC_BF16 1u     /* BF16 operands, FP32 accumulation (tcgen05) */
#define EDPC_FP8E4M3 2u  /* FP8 e4m3 operands with per-tensor power-of-two scales
                            (2^k, k largest with amax * 2^k <= 448, every step),
                            FP32 accumulation (tcgen05 kind::f8f6f4) */

/* cfg.flags */
#define EDPC_FLAG_NO_PIPELINE 1u  /* run the coder stage inline (DPCA off) */
#define EDPC_FLAG_NO_GRAPH 2u     /* launch every kernel eagerly (no CUDA graph) */
#define EDPC_FLAG_TUNE_TILES 4u   /* BF16: time each GEMM's N tile at open and record the
                                     choice in the header (file sets always do) */
#define EDPC_FLAG_OVERLAP_FDM 8u  /* BF16/FP8: run the FDM's Adam update as a persistent
                                     kernel on its own stream, overlapping the rest of
                                     the step and the next step's first layers (same
                                     results; slower on GB300 at the measured sizes,
                                     kept for comparison) */
#define EDPC_FLAG_DELAYED_UPDATE 16u
                                  /* FP32/BF16: delayed-update schedule, a variant of
                                     Algorithm 1 (which updates before the next
                                     prediction): the gradient of step i, taken at the
                                     parameters that predicted step i, is applied after
                                     step i + 1, theta_{i+1} = Adam(theta_i, g_{i-1}), for
                                     the shared parameters and the FDMs alike. The adjoint
                                     of step i then runs beside the forward pass of step
                                     i + 1 on a second CUDA stream, in the encoder and the
                                     decoder. A different bitstream from the default
                                     schedule, still lossless; recorded in the header.
                                     Needs twice the parameter, FDM and activation memory.
                                     Not with EDPC_FLAG_OVERLAP_FDM, FP8 or the model API. */

/*
 * Model and coder configuration. Everything here that changes the bitstream
 * is stored in the header, so edpc_decompress needs no cfg.
 *
 *   streams    b, the number of parallel streams (the paper's batch size,
 *              Sec. 4.4). The input is split into b_eff = min(b, max(1, n/K))
 *              contiguous streams of q or q+1 bytes (q = n / b_eff).
 *   context    K, history bytes per prediction (t in Algorithm 1; 16 in
 *              Sec. 4.1). The first K bytes of each stream are coded with
 *              equal probability (Algorithm 1, first line).
 *   embed_dim  D, the byte embedding width; F = K * D is the model width.
 *   latent     F' = F / r, the LTE latent width (Eq. 14); the FDM of each
 *              stream is F' x F' (Eq. 15). 0 selects the ablation "w/o LTE"
 *              of Table 4 and Sec. 4.4.3: no projections, and each stream's
 *              FDM is F x F and acts on the block output itself (F <= 1024).
 *   hidden     H, the width of each MBRB branch (Eq. 10).
 *   blocks     n MBRBs: n/2 "Local" before the LTE and n - n/2 "Global"
 *              after it (Fig. 3 caption).
 *   branches   k, the MBRB paths multiplied together (Eq. 11); 2 by default
 *              (Sec. 3.1.2), 1..3 accepted.
 *   lr         Adam learning rate (Sec. 4.1: 1e-3).
 *   precision  EDPC_FP32, EDPC_BF16 or EDPC_FP8E4M3.
 *   seed       seed of the initial parameters (SplitMix64 counter streams).
 *
 * Limits: 1 <= context <= 256; embed_dim a multiple of 8 in [8, 64];
 * latent (0, or a multiple of 8) and hidden multiples of 8; F <= 2048,
 * F' <= 1024, H <= 2048;
 * streams <= 65535; blocks <= 16.
 */
typedef struct {
  uint32_t version;     /* must be EDPC_ABI_VERSION */
  uint32_t streams;
  uint32_t context;
  uint32_t embed_dim;
  uint32_t latent;
  uint32_t hidden;
  uint32_t blocks;
  uint32_t branches;
  float lr;
  uint32_t precision;
  uint64_t seed;
  uint32_t flags;
  uint32_t reserved;
} edpc_cfg;

/* Fills *cfg with the small FP32 configuration: b = 4, K = 16, D = 16,
 * F' = 128, H = 128, n = 2, k = 2, lr = 1e-3, seed = 1. */
void edpc_default_cfg(edpc_cfg* cfg);

/* Human-readable name of a status code (static storage). */
const char* edpc_strerror(int status);

/* Detail of the last failure on the calling thread (static thread-local
 * storage, overwritten by the next failure). */
const char* edpc_last_error(void);

/* Number of shared FP32 parameters (embedding, MBRBs, LTE projections,
 * head) in the canonical flat order documented at edpc_model_get_state. */
uint64_t edpc_param_count(const edpc_cfg* cfg);

/* Releases a buffer returned by the library. NULL is ignored. */
void edpc_free(void* p);

/*
 * One-shot compression of host bytes (Algorithm 1, encoding side).
 *   buf, len   input (host). len may be 0.
 *   cfg        configuration (host, borrowed).
 *   out        receives a library-allocated host buffer holding the
 *              container: header, per-stream lengths, CRCs, substreams.
 *   out_len    receives its size in bytes.
 * Errors: EINVAL (NULL pointers, bad cfg), ENOMEM, ECUDA, ETIMEOUT.
 */
int edpc_compress(const uint8_t* buf, size_t len, const edpc_cfg* cfg,
                  uint8_t** out, size_t* out_len);

/*
 * One-shot decompression (Algorithm 1, decoding side). The configuration is
 * read from the header.
 *   bits, bits_len  container from edpc_compress (host).
 *   out, out_len    receive a library-allocated host buffer with the bytes.
 * Errors: ECORRUPT (bad magic, header CRC, lengths, or the CRC32 of the
 * decoded data does not match), EVERSION, EARCH, ENOMEM, ECUDA, ETIMEOUT.
 */
int edpc_decompress(const uint8_t* bits, size_t bits_len, uint8_t** out, size_t* out_len);

/* Reads the configuration and original length stored in a container
 * header without decoding (host only). cfg->flags carries
 * EDPC_FLAG_DELAYED_UPDATE when the container was coded with that schedule.
 * Errors: ECORRUPT, EVERSION, EARCH (an update schedule this library version lacks). */
int edpc_peek(const uint8_t* bits, size_t bits_len, edpc_cfg* cfg, uint64_t* orig_len,
              uint32_t* streams_eff);

/* ------------------------------------------------------------------------ */
/* Sessions: the same loop, advanced a bounded number of steps per call.    */
/* ------------------------------------------------------------------------ */
typedef struct edpc_session edpc_session;

/*
 * Opens an encoder over `len` input bytes.
 *   data            input bytes. If data_on_device is 0 they are host bytes,
 *                   copied to the device at open; otherwise `data` is a
 *                   device pointer that must stay valid until the session
 *                   is closed.
 *   cuda_stream     cudaStream_t on which the model stage runs (NULL: the
 *                   library's own). The coder stage runs on a second stream
 *                   of the library's and joins back before run() returns.
 * The uniform prefix (the first K bytes of each stream) is coded at open.
 */
int edpc_encoder_open(const edpc_cfg* cfg, const uint8_t* data, size_t len, int data_on_device,
                      void* cuda_stream, edpc_session** out);

/*
 * Advances the session by up to `max_steps` model steps. A model step codes
 * one byte of every active stream (one iteration of Algorithm 1's loop for
 * the whole batch). *steps_done receives the number run (0 when finished).
 * If `sync` is 0 the call may return before the GPU work finishes; the
 * work is ordered on cuda_stream.
 */
int edpc_session_run(edpc_session* s, uint64_t max_steps, int sync, uint64_t* steps_done);

/* Model steps left (total = max stream length - K, or 0). */
int edpc_session_remaining(const edpc_session* s, uint64_t* steps_left);

/* Encoder: runs any remaining steps, flushes the coders and returns the
 * container (library-allocated host buffer). */
int edpc_encoder_finish(edpc_session* s, uint8_t** out, size_t* out_len);

/*
 * Opens a decoder over a container. If out_device is non-NULL the decoded
 * bytes are written there (device, orig_len bytes, caller-owned);
 * otherwise the library allocates the device buffer.
 */
int edpc_decoder_open(const uint8_t* bits, size_t bits_len, void* out_device, void* cuda_stream,
                      edpc_session** out);

/* Decoder: runs remaining steps, checks the CRC32 of the decoded bytes and
 * copies them to `out_host` (orig_len bytes, caller-owned) if non-NULL. */
int edpc_decoder_finish(edpc_session* s, uint8_t* out_host);

/* Per-session counters. The fdm_*_ms fields are CUDA-event times of the
 * FDM kernels, averaged over the steps recorded since profiling was enabled
 * (see edpc_session_profile). */
typedef struct {
  uint64_t steps_run;
  uint64_t steps_total;
  uint32_t streams;
  uint32_t launches_per_step;    /* kernels this library launches per model step */
  double fdm_fwd_ms;             /* FDM forward (Eq. 15) */
  double fdm_bwd_ms;             /* FDM adjoint: dx' alone when the update is split off, else dx' + Adam */
  uint64_t fdm_samples;
  uint64_t coded_bytes;          /* substream bytes so far (after finish: final) */
  double fdm_adam_ms;            /* FDM Adam update when it runs as its own kernel, else 0 */
} edpc_stats;

int edpc_session_stats(const edpc_session* s, edpc_stats* st);

/* Turns on CUDA-event timing of the FDM kernels for subsequent run()
 * calls. It records events around those two launches in every step. */
int edpc_session_profile(edpc_session* s, int on);

void edpc_session_close(edpc_session* s);

/* ------------------------------------------------------------------------ */
/* File sets: many files of uneven size in one batch.                       */
/* ------------------------------------------------------------------------ */
/*
 * The paper codes one input split into parallel streams (Sec. 3.3); it has
 * no archive format. Here a file set runs as one batch under one model: with
 * stream length L, file f of n_f bytes becomes m_f = ceil(n_f / L) contiguous
 * streams of q or q + 1 bytes (q = n_f / m_f, the longer ones first),
 * numbered file by file; an empty file has none. All streams start together
 * and each stops when its bytes run out (it is then masked: no coding, no
 * gradient, no FDM update). Each stream has its own FDM, Adam moments and
 * range coder; the shared parameters learn from every active stream.
 *
 * cfg->streams chooses L:
 *   > 0  a stream budget: the smallest L whose split has at most that many
 *        streams (one stream per file when even that exceeds the budget).
 *   0    autotuned on the current GPU: candidates L = 8 KiB * 2^j, model step
 *        times measured at two stream counts (CUDA graph of the step) and
 *        fitted as t0 + c * b, models that do not fit in 70 % of free device
 *        memory dropped; the longest L within 5 % of the fastest estimate is
 *        taken (fewer streams learn from more bytes each).
 * The GEMM N tiles are also timed at open (BF16) and recorded in the header.
 * Limits as for edpc_cfg; at most 65535 streams in all.
 */
typedef struct {
  uint64_t stream_len;        /* L */
  uint32_t streams;           /* b = sum_f ceil(n_f / L) (1 if no bytes) */
  uint32_t reserved;
  double est_seconds;         /* autotuner's estimate of the encode time (0 for a budget) */
  double step_ms_t0;          /* fitted model-step time at zero streams (ms) */
  double step_ms_per_stream;  /* fitted model-step time per stream (ms) */
} edpc_split_plan;

/* The split edpc_compress_many would use (lens: host, nfiles sizes). With
 * cfg->streams = 0 this runs the autotuner's probes on the current GPU.
 * Errors: EINVAL (bad cfg, NULL, more than 65535 streams), ENOMEM, ECUDA. */
int edpc_archive_plan(const size_t* lens, size_t nfiles, const edpc_cfg* cfg, edpc_split_plan* plan);

/* One-shot compression of a file set into one container.
 *   bufs, lens  host arrays of nfiles pointers and sizes (a pointer may be
 *               NULL when its size is 0).
 * out/out_len as for edpc_compress. Errors as edpc_compress and
 * edpc_archive_plan. */
int edpc_compress_many(const uint8_t* const* bufs, const size_t* lens, size_t nfiles, const edpc_cfg* cfg,
                       uint8_t** out, size_t* out_len);

/* Encoder session over a file set (see edpc_encoder_open). bufs[f] are host
 * pointers, or device pointers when data_on_device != 0; either way the
 * files are copied, in order, into one library-owned device buffer at open.
 * edpc_decoder_open decodes the container; its output is the files' bytes
 * back to back, in order. */
int edpc_encoder_open_many(const edpc_cfg* cfg, const uint8_t* const* bufs, const size_t* lens, size_t nfiles,
                           int data_on_device, void* cuda_stream, edpc_session** out);

/* File count and sizes of a container. For a single-input container
 * *nfiles = 1 and sizes[0] = its length. sizes (host, *nfiles entries) may
 * be NULL to query the count first. Errors: ECORRUPT, EVERSION, EARCH. */
int edpc_archive_info(const uint8_t* bits, size_t bits_len, uint64_t* nfiles, uint64_t* sizes);

/* One-shot decompression of a container into its files.
 *   *outs   receives one library-allocated block: *nfiles pointers, one per
 *           file, followed by the files' bytes; release it with
 *           edpc_free(*outs).
 *   *lens   receives a library-allocated array of *nfiles sizes; release
 *           with edpc_free(*lens).
 * Errors as edpc_decompress. */
int edpc_decompress_many(const uint8_t* bits, size_t bits_len, uint8_t*** outs, size_t** lens, size_t* nfiles);

/* ------------------------------------------------------------------------ */
/* Archives of independent per-file models.                                 */
/* ------------------------------------------------------------------------ */
/*
 * A file set in which every file has its own model (the paper codes one
 * input under one model, Algorithm 1 and Sec. 3.3, over a batch of streams;
 * an archive whose files share one model, as edpc_compress_many makes, can
 * only be decoded whole). File f is split as edpc_compress would split it
 * with cfg->streams = max(1, ceil(n_f / stream_len)), and each member is a
 * single-input container, so any file decodes alone.
 *   BF16 with Algorithm 1's schedule: all files' models run as one batch.
 *     File f's streams take rows padded to a multiple of 64; every kernel of
 *     the step indexes the parameters of the row's own file (the GEMMs run
 *     one launch over all files: tile lists with per-file weights, and
 *     weight gradients contracting each file's rows only), and the CE mean of
 *     Eq. 2 is over the file's own active streams. Each member is a header
 *     variant 2 container; edpc_decompress replays it with the same engine
 *     and one file, and a member's bytes do not depend on the other files of
 *     the batch. `concurrency` is unused.
 *   Other precisions or schedules: member f is exactly edpc_compress's
 *     container for file f; the files' sessions run `concurrency` at a time
 *     (0: 8), each on its own CUDA stream.
 *
 * Container: "EDPI", u32 format version, u64 file count, u64 stream_len,
 * per file (u64 member offset, u64 member bytes, u64 file bytes), u32 CRC-32
 * of the preceding bytes, then the members.
 *
 *   edpc_compress_independent  bufs/lens: host arrays of nfiles pointers and
 *                              sizes (NULL allowed for size 0). out/out_len as
 *                              for edpc_compress. cfg->streams is ignored.
 *                              Errors: EINVAL (bad cfg, NULL, stream_len 0; a
 *                              batch above 65535 padded rows), ENOMEM, ECUDA,
 *                              ETIMEOUT.
 *   edpc_independent_info      file count and sizes (sizes may be NULL).
 *                              Errors: ECORRUPT, EVERSION.
 *   edpc_decompress_member     decodes file `index` alone into a
 *                              library-allocated buffer (edpc_free).
 *                              Errors: EINVAL (index), and as edpc_decompress.
 *   edpc_decompress_independent  every file: members of the batched engine
 *                              with one configuration in one batch (each
 *                              member's checksum checked), others
 *                              `concurrency` at a time; outputs as for
 *                              edpc_decompress_many.
 */
int edpc_compress_independent(const uint8_t* const* bufs, const size_t* lens, size_t nfiles, const edpc_cfg* cfg,
                              uint64_t stream_len, uint32_t concurrency, uint8_t** out, size_t* out_len);
int edpc_independent_info(const uint8_t* bits, size_t bits_len, uint64_t* nfiles, uint64_t* sizes);
int edpc_decompress_member(const uint8_t* bits, size_t bits_len, uint64_t index, uint8_t** out, size_t* out_len);
int edpc_decompress_independent(const uint8_t* bits, size_t bits_len, uint32_t concurrency, uint8_t*** outs,
                                size_t** lens, size_t* nfiles);


/* ------------------------------------------------------------------------ */
/* Single kernels on device buffers, for tests and benchmarks.              */
/* ------------------------------------------------------------------------ */

/*
 * CDF quantization of `rows` FP32 probability vectors, the coder's input
 * (Sec. 2.1 "Data Encoding"; the paper leaves the rule open, this is the
 * library's rule).
 *   p     device, rows x 256 FP32.
 *   freq  device, rows x 256 uint32 out: f_j = 1 + floor(fl32(p_j * 65280)),
 *         remainder 65536 - sum(f) added to the first largest f.
 *   cum   device, rows x 257 uint32 out: exclusive prefix sums, cum[256] = 65536.
 */
int edpc_cdf_quantize(const float* p, uint32_t rows, uint32_t* freq, uint32_t* cum,
                      void* cuda_stream);

/*
 * Range-encodes `nsym` symbols for each of `streams` independent coders
 * (one 32-bit range coder per stream, the arithmetic coding of Sec. 2.1).
 *   sym   device, nsym x streams uint32, step-major: sym[t*streams + s] =
 *         cum | (freq - 1) << 16 of stream s's t-th symbol, or 0xFFFFFFFF
 *         to skip. cum + freq <= 65536.
 *   out   device, streams x cap bytes: stream s writes at out + s*cap.
 *   out_len device, streams uint32 out: bytes written per stream.
 * Errors: EINVAL if some stream needs more than cap bytes (its output is
 * then truncated and out_len holds cap).
 */
int edpc_range_encode(const uint32_t* sym, uint32_t nsym, uint32_t streams, uint8_t* out,
                      uint32_t cap, uint32_t* out_len, void* cuda_stream);

/*
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory per call, such as services that reserve
 * their whole GPU memory budget at start-up and refuse later allocations, or
 * loops that cannot absorb the device-wide synchronisation cudaFree may do.
 *
 * Same arguments, layout and result as edpc_range_encode, but the per-stream
 * coder state, output offsets and capacities live in a fixed scratch array
 * compiled into the library (EDPC_NOALLOC_MAX_STREAMS streams, about 176 KiB,
 * held on every GPU that loads the library until the process exits). The
 * call makes no device or host allocation.
 *   - streams must be <= EDPC_NOALLOC_MAX_STREAMS; larger counts return
 *     EDPC_EINVAL before any GPU work.
 *   - The first call on each device looks up the scratch's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device. The address is kept for the
 *     life of the process, so after a cudaDeviceReset of a device this entry
 *     point must not be called on that device again.
 *   - Every call on a device uses the same scratch and re-initialises it.
 *     Calls whose GPU work overlaps (different streams or threads, same
 *     device) race on it and must be serialised by the caller.
 *   - Returns after the work on cuda_stream has completed.
 */
#define EDPC_NOALLOC_MAX_STREAMS 4096u
int edpc_range_encode_noalloc(const uint32_t* sym, uint32_t nsym, uint32_t streams, uint8_t* out,
                              uint32_t cap, uint32_t* out_len, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Model: one training step at a given state (gradient and parity checks).  */
/* ------------------------------------------------------------------------ */
typedef struct edpc_model edpc_model;

/* A model for `streams` rows with cfg's dims and precision, initialised
 * from cfg.seed exactly as the encoder initialises it. Its steps follow
 * Algorithm 1: cfg.flags with EDPC_FLAG_DELAYED_UPDATE gives EDPC_EINVAL. */
int edpc_model_create(const edpc_cfg* cfg, uint32_t streams, edpc_model** out);
void edpc_model_destroy(edpc_model* m);

/*
 * State exchange (host buffers; NULL skips that part).
 *   shared  edpc_param_count(cfg) floats in the canonical order:
 *           E[256][D];
 *           for each block j = 0..n-1: ln_g[F], ln_b[F], W[k*H][F] (branch i
 *             in rows i*H..i*H+H-1), c[k*H], Wo[F][H], co[F];
 *           LTE W1[F'][F], b1[F'], W2[F][F'], b2[F];
 *           head Wh[256][F], bh[256].
 *   fdm     streams x F' x F' floats, U_s[i][j] at (s*F' + i)*F' + j.
 *   m_*, v_* Adam moments in the same layouts. t = Adam steps taken.
 */
int edpc_model_get_state(const edpc_model* m, float* shared, float* fdm, float* m_shared,
                         float* v_shared, float* m_fdm, float* v_fdm, uint32_t* t);
int edpc_model_set_state(edpc_model* m, const float* shared, const float* fdm, const float* m_shared,
                         const float* v_shared, const float* m_fdm, const float* v_fdm, uint32_t t);

/*
 * Forward pass (Eqs. 9-16 and the head) on host inputs.
 *   ctx     host, streams x K bytes, oldest first.
 *   logits  host out, streams x 256 (may be NULL).
 *   probs   host out, streams x 256 FP32 softmax (may be NULL).
 */
int edpc_model_forward(edpc_model* m, const uint8_t* ctx, float* logits, float* probs);

/*
 * Gradient of the mean cross-entropy over the active rows (Eq. 2) at the
 * current state, without updating it.
 *   targets  host, streams bytes.   active  host, streams bytes (0/1).
 *   g_shared host out (param_count floats, canonical order) or NULL.
 *   g_fdm    host out (streams x F' x F') or NULL.
 */
int edpc_model_backward(edpc_model* m, const uint8_t* ctx, const uint8_t* targets,
                        const uint8_t* active, float* g_shared, float* g_fdm);

/* Forward, backward and one Adam step (Sec. 4.1), exactly as one model step
 * of the encoder: inactive rows leave their FDM and its moments unchanged. */
int edpc_model_train_step(edpc_model* m, const uint8_t* ctx, const uint8_t* targets,
                          const uint8_t* active);

/*
 * GEMM N tiles of a BF16 model (no effect in FP32). Each tcgen05 GEMM site
 * has a code: 0 = chosen from the problem size, 1/2/4/8 = N tile of
 * 32/64/128/256 (for the fused branch GEMM of Eqs. 10-12: 32 * code hidden
 * units of each branch per tile, at most 256 columns in all).
 * The codes fix how each output tile is accumulated, so a decoder must use
 * the encoder's (containers record them when tuned). There is no such
 * choice in the paper; it is a GPU implementation parameter.
 *   edpc_model_set_tiles   sets codes[0..n) (the rest 0). Errors: EARCH for
 *                          a code the site does not accept.
 *   edpc_model_tune_tiles  times every accepted code at every site on the
 *                          model's buffers (before a step: it overwrites
 *                          activations and gradients), keeps the fastest, and
 *                          copies up to cap codes to `codes` (host, may be
 *                          NULL); *n receives the number of sites.
 */
int edpc_model_set_tiles(edpc_model* m, const uint8_t* codes, uint32_t n);
int edpc_model_tune_tiles(edpc_model* m, uint8_t* codes, uint32_t cap, uint32_t* n);

/*
 * Measurement of the model's Linear layers (Eqs. 10, 13, 14, 16, the head and
 * their adjoints; the paper reports no per-layer timing). Each tcgen05 GEMM
 * site of a BF16 or FP8 model is launched alone: one warm-up launch, then
 * `reps` launches between two CUDA events on the default stream. ms[i] (host)
 * receives the mean milliseconds per launch of site i, flop[i] its 2*M*N*K
 * and, when bytes is not NULL, bytes[i] its compulsory memory traffic (A and
 * B, the residual or saved branch outputs its epilogue reads, and every
 * output it writes, each counted once); unused sites get 0. Writes
 * min(cap, site count) entries and that count to *n. Like
 * edpc_model_tune_tiles it overwrites activations and gradients (call it
 * between steps). Errors: EINVAL (NULL ms or flop, FP32 model), ECUDA.
 */
int edpc_model_time_gemms(edpc_model* m, uint32_t reps, double* ms, double* flop, double* bytes, uint32_t cap,
                          uint32_t* n);

/*
 * The residual-stream input and output of MBRB `block` (0 .. blocks-1) from
 * the last edpc_model_forward: the skip S and the fused output S + X^(k) of
 * Sec. 3.1.1 (Eq. 13: the block adds G W_o^T + c_o to its input). s_in and
 * s_out are host arrays of streams * F floats (FP32, [stream][feature]).
 * Errors: EINVAL (NULL, block out of range), ECUDA.
 */
int edpc_model_block_io(edpc_model* m, uint32_t block, float* s_in, float* s_out);

/*
 * Kraskov's k-nearest-neighbour estimate of the mutual information I(Z; Y)
 * that Sec. 3.1.1 uses to compare branch counts (IFR_{k1->k2} =
 * I^(k1) / I^(k2)). Z (N x dz) and Y (N x dy) are FP32 row-major device
 * arrays of paired samples. For each sample i, eps(i) is the k-th smallest
 * distance max(|z_i - z_j|_inf, |y_i - y_j|_inf) over j != i, and c_z(i),
 * c_y(i) (written to the device arrays cz, cy of N counts) are the numbers of
 * j != i strictly closer than eps(i) in z and in y alone; distances and counts
 * are exact functions of the FP32 samples. *mi (host) receives
 * psi(k) + psi(N) - mean_i(psi(c_z(i) + 1) + psi(c_y(i) + 1)) in nats, FP64.
 * Runs on cuda_stream (NULL: the default stream) and waits for it.
 * Limits: 2 <= N <= 8192, 1 <= k <= min(64, N - 1), dz + dy <= 8192.
 * Errors: EINVAL, ECUDA.
 */
int edpc_ksg_mi(const float* Z, const float* Y, uint32_t N, uint32_t dz, uint32_t dy, uint32_t k, uint32_t* cz,
                uint32_t* cy, double* mi, void* cuda_stream);

/*
 * Self-test of the bounded-wait error path (fault detection without a GPU
 * fault). One CTA waits on a shared-memory mbarrier that nothing arrives on;
 * the wait gives up after about 50 ms of SM clock (or 2^20 polls), records an
 * error bit and returns, as every bounded wait of the library's kernels does.
 * Runs on cuda_stream (NULL: the default stream) and waits for it, then runs
 * a further copy on the stream to show the context still works.
 * Returns EDPC_ETIMEOUT when the wait expired (the expected result), ECUDA if
 * the wait completed or a CUDA call failed.
 */
int edpc_selftest_wait_timeout(void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EDPC_H */
