"""Algorithm 1 over b parallel streams (oracle side).

Algorithm 1 (Sec. 2.1) codes one byte stream: the first t bytes with equal
probability, then for each later byte x_i it predicts Pr(i) from the
previous t bytes, codes x_i, and takes one optimizer step on the
cross-entropy (Eq. 2). Decoding replays the same loop on decoded bytes.

The batch of Sec. 3.3 / Sec. 4.4 splits the input into b segments
("streams") that advance one byte per step together through one shared
model. Each stream has its own FDM slice U_s (Sec. 3.2) and, here, its own
range coder; that replaces the paper's pool of encoding subprocesses.

Readings:
  * Split: b_eff = min(b, max(1, n // K)) streams. With q, rem =
    divmod(n, b_eff), stream s has q + (s < rem) bytes and starts at
    s*q + min(s, rem).
  * Step i (0-based) is active for stream s when K <= i < len_s. The uniform
    prefix covers i < K (each byte costs exactly 8 bits, f = 256).
  * The loss of a step is the mean over its active streams.
  * A file set (archive) is cut file by file into streams of at most L
    bytes (``archive_split``); all its streams start together and share the
    model, exactly as the streams of one input do.
  * Delayed update (``delayed=True``; a schedule outside Algorithm 1, which
    updates before the next prediction): the gradient of step i is still
    taken at the parameters theta_i that predicted step i, but it is
    applied one step later, theta_{i+1} = Adam(theta_i, g_{i-1}), with
    theta_{K+1} = theta_K (no gradient exists before the first step). The
    shared parameters and every stream's FDM follow the same rule; the FDM
    rows updated are those active at step i - 1. Adam's step counter counts
    applied updates. Encoder and decoder run the same schedule, so the
    result stays lossless; it lets the adjoint of step i run beside the
    forward of step i + 1.

Parity: the round trip is an invariant, checked here on every call that
decodes. The code length is checked against the ideal plus truncation bound,
and the bits/byte against the closed-form entropy of seeded sources
(tests/test_oracle_compress.py). The delayed schedule is pinned by its
definition built from independent pieces: no update after the first step,
the first update equal to Algorithm 1's first, and the second one taken
from a fresh model's gradient at the stale parameters
(tests/test_oracle_delayed.py).
"""
from __future__ import annotations

import numpy as np

from .coder import RangeDecoder, RangeEncoder, quantize_cdf
from .model import Config, Model, softmax


def split_streams(n: int, b: int, K: int):
    """(b_eff, offsets, lengths) of the contiguous stream split."""
    b_eff = min(b, max(1, n // K)) if K > 0 else b
    b_eff = max(1, b_eff)
    q, rem = divmod(n, b_eff)
    lengths = np.array([q + (1 if s < rem else 0) for s in range(b_eff)], dtype=np.int64)
    offsets = np.array([s * q + min(s, rem) for s in range(b_eff)], dtype=np.int64)
    return b_eff, offsets, lengths


def archive_split(sizes, L: int):
    """(b, offsets, lengths) of a file set cut into streams of at most L bytes.

    Reading for many files in one batch (Sec. 3.3's parallel streams over a
    file set): file f of n_f bytes becomes m_f = ceil(n_f / L) contiguous
    streams; with q, rem = divmod(n_f, m_f) the first rem of them have q + 1
    bytes and the others q. Streams are numbered file by file, offsets are
    into the files' concatenation, and an empty file has no stream. If no
    file has a byte, there is one empty stream (as for an empty input).
    """
    assert L >= 1
    offsets, lengths = [], []
    base = 0
    for n in sizes:
        n = int(n)
        m = -(-n // L)
        if m:
            q, rem = divmod(n, m)
            for j in range(m):
                offsets.append(base + j * q + min(j, rem))
                lengths.append(q + (1 if j < rem else 0))
        base += n
    if not lengths:
        offsets, lengths = [0], [0]
    return len(lengths), np.array(offsets, dtype=np.int64), np.array(lengths, dtype=np.int64)


def archive_stream_len(sizes, budget: int) -> int:
    """The smallest L >= 1 with sum_f ceil(n_f / L) <= budget (budget >= the
    number of non-empty files, else the largest file size)."""
    sizes = [int(n) for n in sizes if int(n) > 0]
    if not sizes:
        return 1

    def count(L):
        return sum(-(-n // L) for n in sizes)

    lo, hi = 1, max(sizes)
    while lo < hi:
        mid = (lo + hi) // 2
        if count(mid) <= budget:
            hi = mid
        else:
            lo = mid + 1
    return lo


def _contexts(buf, offsets, rows, i, K):
    idx = offsets[rows][:, None] + (i - K) + np.arange(K)[None, :]
    return buf[idx]


def _update(model: Model, g, dU, rows, pending, delayed: bool):
    """The optimizer step after a model step; returns the new pending update.

    Algorithm 1: Adam on this step's gradient now. Delayed: Adam on the
    previous step's gradient (none after the first step), and this step's
    gradient waits for the next step.
    """
    if not delayed:
        model.adam(g, dU, rows)
        return None
    if pending is not None:
        model.adam(*pending)
    return (g, dU, rows)


def oracle_compress(data, cfg: Config, streams: int, max_steps: int | None = None,
                    model: Model | None = None, split=None, delayed: bool = False):
    """Encodes ``data`` (uint8) with Algorithm 1 over ``streams`` streams.

    Returns a dict: ``streams`` (list of bytes), ``b``, ``lengths``,
    ``offsets``, ``ideal_bits`` and ``trunc_bits`` per stream, ``model``
    (the final state), ``steps`` (model steps run). With ``max_steps``, only
    that many model steps run and the coders are flushed there (a prefix
    run, used for timing and for comparing bits/byte on a prefix).
    ``split`` = (b, offsets, lengths) replaces the contiguous split (for
    example ``archive_split`` of a file set; ``streams`` is then ignored).
    ``delayed`` selects the delayed-update schedule (module header).
    """
    data = np.asarray(data, dtype=np.uint8)
    n = data.size
    K = cfg.context
    b, offsets, lengths = split_streams(n, streams, K) if split is None else split
    if model is None:
        model = Model(cfg, b)
    encs = [RangeEncoder() for _ in range(b)]
    # Algorithm 1, first line: the first t bytes with equal probability.
    for s in range(b):
        for i in range(min(K, int(lengths[s]))):
            encs[s].encode(256 * int(data[offsets[s] + i]), 256)
    L = int(lengths.max()) if b else 0
    steps = 0
    pending = None
    for i in range(K, L):
        if max_steps is not None and steps >= max_steps:
            break
        rows = np.nonzero(lengths > i)[0]
        ctx = _contexts(data, offsets, rows, i, K)
        x = data[offsets[rows] + i].astype(np.int64)
        # Model(x_{i-t..i-1}) -> Pr(i); encode x_i with Pr(i).
        z, cache = model.forward(ctx, rows)
        p = softmax(z)
        f, cum = quantize_cdf(p.astype(np.float32))
        for r_, s in enumerate(rows):
            encs[s].encode(int(cum[r_, x[r_]]), int(f[r_, x[r_]]))
        # loss = CrossEntropy(Pr(i), x_i); backward; update.
        dz = p.copy()
        dz[np.arange(len(rows)), x] -= 1.0
        dz /= len(rows)
        g, dU = model.backward(cache, dz)
        pending = _update(model, g, dU, rows, pending, delayed)
        steps += 1
    out = [e.finish() for e in encs]
    return dict(streams=out, b=b, lengths=lengths, offsets=offsets,
                ideal_bits=np.array([e.ideal_bits for e in encs]),
                trunc_bits=np.array([e.trunc_bits for e in encs]),
                model=model, steps=steps)


def oracle_decompress(streams, n: int, cfg: Config, b_req: int, split=None, delayed: bool = False) -> np.ndarray:
    """Decodes the per-stream bitstreams of ``oracle_compress`` back to ``n`` bytes."""
    K = cfg.context
    b, offsets, lengths = split_streams(n, b_req, K) if split is None else split
    assert len(streams) == b
    model = Model(cfg, b)
    decs = [RangeDecoder(s) for s in streams]
    buf = np.zeros(n, dtype=np.uint8)
    for s in range(b):
        for i in range(min(K, int(lengths[s]))):
            buf[offsets[s] + i] = decs[s].decode_uniform()
    L = int(lengths.max()) if b else 0
    pending = None
    for i in range(K, L):
        rows = np.nonzero(lengths > i)[0]
        ctx = _contexts(buf, offsets, rows, i, K)
        z, cache = model.forward(ctx, rows)
        p = softmax(z)
        f, cum = quantize_cdf(p.astype(np.float32))
        x = np.empty(len(rows), dtype=np.int64)
        for r_, s in enumerate(rows):
            x[r_] = decs[s].decode(cum[r_])
            buf[offsets[s] + i] = x[r_]
        dz = p.copy()
        dz[np.arange(len(rows)), x] -= 1.0
        dz /= len(rows)
        g, dU = model.backward(cache, dz)
        pending = _update(model, g, dU, rows, pending, delayed)
    return buf
