// Many files in one batch: the split of a file set into streams, the stream
// length for a stream budget, and the autotuner that picks the stream length
// (and with it the stream count) from measured step times.
#pragma once

#include <vector>

#include "common.cuh"

namespace edpc {

// Per-stream byte ranges of an input: stream s is [off[s], off[s] + len[s]).
struct StreamLayout {
  std::vector<long long> off, len;
  int streams() const { return (int)len.size(); }
  long long max_len() const;
  int active_at(long long i) const;  // streams with len > i
};

// File f of n_f bytes becomes m_f = ceil(n_f / L) contiguous streams of q or
// q + 1 bytes (q = n_f / m_f, the longer ones first), numbered file by file
// with offsets into the files' concatenation. An empty file has no stream; a
// set with no bytes has one empty stream.
void archive_split(const uint64_t* sizes, size_t nfiles, uint64_t L, StreamLayout* out);

// Number of streams archive_split makes for stream length L.
uint64_t archive_stream_count(const uint64_t* sizes, size_t nfiles, uint64_t L);

// The smallest L >= 1 whose split has at most `budget` streams; the largest
// file size when even one stream per file exceeds the budget.
uint64_t archive_stream_len(const uint64_t* sizes, size_t nfiles, uint64_t budget);

// Autotuned stream length for cfg's model on the current device.
//   Candidates: L = 8 KiB * 2^j (every stream of a file longer than 8 KiB
//   then holds at least 4 KiB) up to the largest file, with at most 65535
//   streams whose model fits in 70 % of the free device memory.
//   Cost model: the time of one model step at b streams is measured at two
//   stream counts (a CUDA graph of the whole step, replayed) and fitted as
//   t(b) = t0 + c b; a candidate's encode time is (longest stream - K) t(b).
//   Choice: the longest L (fewest streams, so each stream's FDM learns from
//   more bytes) whose estimate is within 5 % of the fastest candidate's.
struct TunedPlan {
  uint64_t L = 0;
  uint32_t streams = 0;
  double est_seconds = 0;   // estimated encode time of the whole set
  double step_ms_t0 = 0;    // fitted t0 (ms)
  double step_ms_per_stream = 0;  // fitted c (ms per stream)
};
int archive_autotune(const edpc_cfg& cfg, const uint64_t* sizes, size_t nfiles, TunedPlan* out);

}  // namespace edpc
