"""Seeded synthetic byte sources shaped like the paper's workloads.

This module only draws input bytes. It holds none of the compressor's
arithmetic, so the CPU oracle, the tests and the benchmark can all use it
without coupling the oracle to the CUDA path.

The paper measures on datasets that are not available here (Table 1:
text, sound, images, floats, backups). These generators stand in for them:

* ``markov_bytes``: order-k Markov chain over 256 symbols. Each transition
  row is Dirichlet(alpha). Used for the small FP32 workload (order 2,
  alpha 0.1) and for i.i.d. sources (order 0).
* ``image_bytes``: 8-bit 512x512 grayscale images. Each is a smooth 2-D
  gradient plus a low-frequency cosine plus Gaussian noise (sigma 4),
  clipped to [0, 255].
* ``pcm_bytes``: 16-bit little-endian PCM at 44.1 kHz. Each 65536-sample
  segment holds 3 sines (50-4000 Hz) plus Gaussian noise (sigma 200).
* ``text_bytes``: order-3 Markov bytes with Dirichlet(0.05) rows. The
  context's 3 bytes are hashed into a fixed table of rows.
* ``multimedia_mix``: images, PCM and text in equal contiguous thirds.
* ``uneven_files``: many files with log-uniform sizes, each a mix drawn
  with its own random weights.

Every function is a pure function of its arguments and seed.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "markov_table",
    "markov_bytes",
    "image_bytes",
    "pcm_bytes",
    "text_bytes",
    "multimedia_mix",
    "uneven_files",
    "MIB",
]

MIB = 1 << 20


def markov_table(order: int, alpha: float, seed: int, rows: int | None = None) -> np.ndarray:
    """Transition rows of an order-``order`` chain, shape (rows, 256), float64.

    Row ``c`` is a Dirichlet(alpha) draw (normalised Gamma(alpha) variates).
    By default there is one row per context (256**order rows).
    """
    if rows is None:
        rows = 256 ** order
    rng = np.random.default_rng([seed, order, 0xD1])
    g = rng.gamma(alpha, 1.0, size=(rows, 256))
    s = g.sum(axis=1, keepdims=True)
    # A row whose Gamma draws all underflow is replaced by a point mass.
    bad = s[:, 0] <= 0
    if np.any(bad):
        g[bad] = 0.0
        g[bad, 0] = 1.0
        s = g.sum(axis=1, keepdims=True)
    return g / s


def _guide(table: np.ndarray):
    """(flat CDF, guide table) of the inverse-CDF sampler for ``table``'s rows."""
    rows = table.shape[0]
    cum = np.cumsum(table, axis=1)
    cum[:, -1] = 1.0
    grid = np.arange(256) / 256.0
    # guide[r, g] = #{j : cum[r, j] <= g / 256}, found with one search over
    # rows shifted apart by 2r.
    flat = (cum + 2.0 * np.arange(rows)[:, None]).ravel()
    q = (grid[None, :] + 2.0 * np.arange(rows)[:, None]).ravel()
    guide = (np.searchsorted(flat, q, side="right").reshape(rows, 256)
             - 256 * np.arange(rows)[:, None]).astype(np.int64)
    return cum.ravel(), guide


def _sample_chains(table: np.ndarray, ctx_index, n_steps: int, state: np.ndarray,
                   rng: np.random.Generator, order: int, prep=None) -> np.ndarray:
    """Runs ``len(state)`` chains in lockstep for ``n_steps`` steps.

    ``state`` is (chains, order) uint8, the last ``order`` bytes of each chain.
    ``ctx_index`` maps that state, given as a list of ``order`` int64 columns
    (oldest first), to a row of ``table``.
    Sampling is by inverse CDF: the symbol is the first j with CDF_j > u.
    A 256-entry guide table per row gives the starting j for u's bucket.
    ``prep`` is ``_guide(table)`` when the caller has it already.
    Returns a (chains, n_steps) uint8 array.
    """
    cum_flat, guide = _guide(table) if prep is None else prep
    chains = state.shape[0]
    out = np.empty((n_steps, chains), dtype=np.uint8)
    cols = [state[:, k].astype(np.int64) for k in range(order)]
    guide_flat = guide.ravel()
    # The uniforms are drawn in blocks of steps: the generator yields the same
    # sequence as one (n_steps, chains) draw, with bounded memory.
    blk = max(1, min(n_steps, (1 << 24) // max(1, chains)))
    for t in range(n_steps):
        if t % blk == 0:
            u = rng.random((min(blk, n_steps - t), chains))
            bucket = (u * 256).astype(np.int64)
        ut = u[t % blk]
        r = ctx_index(cols) if order > 0 else np.zeros(chains, dtype=np.int64)
        base = r * 256
        j = np.minimum(guide_flat[base + bucket[t % blk]], 255)
        # The symbol is the first j >= guide start with CDF_j > u. A few linear
        # steps settle most chains; the rest take a binary search for the
        # count of CDF entries <= u (the same answer: the CDF is nondecreasing).
        for _ in range(3):
            adv = cum_flat[base + j] <= ut
            if not adv.any():
                break
            j = np.minimum(j + adv, 255)
        else:
            left = np.nonzero(cum_flat[base + j] <= ut)[0]
            if left.size:
                lo = np.zeros(left.size, np.int64)
                hi = np.full(left.size, 256, np.int64)
                bl, ul = base[left], ut[left]
                for _ in range(9):
                    mid = (lo + hi) // 2
                    le = cum_flat[bl + np.minimum(mid, 255)] <= ul
                    lo = np.where((lo < hi) & le, mid + 1, lo)
                    hi = np.where((lo < hi) & ~le, mid, hi)
                j[left] = np.minimum(np.maximum(j[left], lo), 255)
        out[t] = j
        if order > 0:
            cols = cols[1:] + [j]
    return np.ascontiguousarray(out.T)


def markov_bytes(n: int, order: int, alpha: float, seed: int,
                 table: np.ndarray | None = None) -> np.ndarray:
    """``n`` bytes from one order-``order`` Markov chain with Dirichlet rows.

    The first ``order`` bytes are uniform. The table (from ``markov_table``)
    can be passed in to avoid redrawing it.
    """
    if table is None:
        table = markov_table(order, alpha, seed)
    rng = np.random.default_rng([seed, order, 0xD2])
    if n <= order:
        return rng.integers(0, 256, size=n, dtype=np.uint8)
    init = rng.integers(0, 256, size=(1, order), dtype=np.uint8)

    def index(cols):
        r = np.zeros(cols[0].shape[0], dtype=np.int64)
        for c in cols:
            r = r * 256 + c
        return r

    body = _sample_chains(table, index, n - order, init, rng, order)[0]
    return np.concatenate([init[0], body]).astype(np.uint8)


def markov_entropy_rate(table: np.ndarray, order: int, iters: int = 4000,
                        tol: float = 1e-13) -> float:
    """Entropy rate in bits/symbol of the chain: sum_c pi(c) H(row_c).

    pi is the stationary distribution over the 256**order contexts, found by
    power iteration. For order 0 this is the entropy of the single row.
    """
    with np.errstate(divide="ignore", invalid="ignore"):
        h_rows = -np.where(table > 0, table * np.log2(table), 0.0).sum(axis=1)
    if order == 0:
        return float(h_rows[0])
    if order == 1:
        pi = np.full(256, 1.0 / 256)
        for _ in range(iters):
            nxt = pi @ table
            if np.abs(nxt - pi).sum() < tol:
                pi = nxt
                break
            pi = nxt
        return float(pi @ h_rows)
    if order == 2:
        p3 = table.reshape(256, 256, 256)  # [a, b, c] = P(c | a, b)
        pi = np.full((256, 256), 1.0 / 65536)
        for _ in range(iters):
            nxt = np.einsum("ab,abc->bc", pi, p3)
            if np.abs(nxt - pi).sum() < tol:
                pi = nxt
                break
            pi = nxt
        return float((pi.ravel() * h_rows).sum())
    raise ValueError("entropy rate implemented for order <= 2")


def image_bytes(n_images: int, seed: int, side: int = 512) -> np.ndarray:
    """``n_images`` raw 8-bit grayscale images of ``side`` x ``side``, concatenated."""
    rng = np.random.default_rng([seed, 0x1A])
    y, x = np.mgrid[0:side, 0:side].astype(np.float64)
    out = np.empty((n_images, side, side), dtype=np.uint8)
    for k in range(n_images):
        a, b = rng.uniform(-0.25, 0.25, size=2)
        c = rng.uniform(64.0, 192.0)
        amp = rng.uniform(10.0, 40.0)
        fx, fy = rng.uniform(0.5, 3.0, size=2)
        ph = rng.uniform(0.0, 2 * np.pi)
        img = a * (x - side / 2) + b * (y - side / 2) + c
        img += amp * np.cos(2 * np.pi * (fx * x + fy * y) / side + ph)
        img += rng.normal(0.0, 4.0, size=(side, side))
        out[k] = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    return out.reshape(-1)


def pcm_bytes(n_bytes: int, seed: int, rate: int = 44100, segment: int = 65536) -> np.ndarray:
    """``n_bytes`` (even) of 16-bit little-endian PCM.

    Every ``segment`` samples, 3 new sines are drawn: frequency U(50, 4000) Hz,
    amplitude U(1000, 8000), phase U(0, 2 pi). Gaussian noise (sigma 200) is
    added and the result is clipped to int16.
    """
    if n_bytes % 2:
        raise ValueError("PCM byte count must be even")
    n = n_bytes // 2
    rng = np.random.default_rng([seed, 0x2B])
    out = np.empty(n, dtype="<i2")
    for s0 in range(0, n, segment):
        m = min(segment, n - s0)
        t = np.arange(m, dtype=np.float64) / rate
        sig = np.zeros(m)
        for _ in range(3):
            f = rng.uniform(50.0, 4000.0)
            amp = rng.uniform(1000.0, 8000.0)
            ph = rng.uniform(0.0, 2 * np.pi)
            sig += amp * np.sin(2 * np.pi * f * t + ph)
        sig += rng.normal(0.0, 200.0, size=m)
        out[s0:s0 + m] = np.clip(np.rint(sig), -32768, 32767).astype("<i2")
    return out.view(np.uint8).copy()


def text_bytes(n_bytes: int, seed: int, alpha: float = 0.05, chains: int = 2048,
               table_rows: int = 1 << 12, table: np.ndarray | None = None, prep=None) -> np.ndarray:
    """``n_bytes`` of order-3 Markov bytes with Dirichlet(alpha) rows.

    The 3-byte context is hashed into ``table_rows`` rows. Each row is a
    Dirichlet(alpha) draw, so the source is still an order-3 chain.
    ``chains`` independent chains run in lockstep and are laid out
    one after another. ``table`` (with ``prep = _guide(table)``) replaces
    the seed's own table, so several texts can share one source.
    """
    if n_bytes == 0:
        return np.zeros(0, dtype=np.uint8)
    if table is None:
        table = markov_table(3, alpha, seed, rows=table_rows)
        prep = None
    table_rows = table.shape[0]
    rng = np.random.default_rng([seed, 0x3C])
    # long texts get more chains (about 64 KiB each) so the lockstep loop stays short
    chains = max(1, min(chains, n_bytes // 64 or 1), n_bytes >> 16)
    per = -(-n_bytes // chains)
    init = rng.integers(0, 256, size=(chains, 3), dtype=np.uint8)

    def index(cols):
        h = (cols[0] * 65599 + cols[1]) * 65599 + cols[2]
        h = (h * 0x9E3779B1) & 0xFFFFFFFF
        return (h >> 16) % table_rows

    body = _sample_chains(table, index, per, init, rng, 3, prep)
    return body.reshape(-1)[:n_bytes].copy()


def multimedia_mix(total: int, seed: int) -> np.ndarray:
    """``total`` bytes: images, PCM and text in equal contiguous thirds.

    The image third holds whole 512x512 images; PCM holds an even number of
    bytes; text takes the remainder.
    """
    third = total // 3
    n_img = third // (512 * 512)
    img = image_bytes(n_img, seed) if n_img else np.zeros(0, np.uint8)
    pcm = pcm_bytes((third // 2) * 2, seed)
    txt = text_bytes(total - img.size - pcm.size, seed)
    out = np.concatenate([img, pcm, txt])
    assert out.size == total
    return out


def uneven_files(n_files: int, seed: int, lo: int = 4096, hi: int = 16 * MIB,
                 max_total: int | None = None) -> list[np.ndarray]:
    """``n_files`` files with sizes log-uniform in [lo, hi].

    Each file mixes image, PCM and text bytes. The weights are Dirichlet(1, 1, 1)
    per file; the parts are laid out contiguously. All files' text comes from
    one order-3 source (one Dirichlet(0.05) table for the set, hashed contexts
    as in ``text_bytes``), sampled as chains of 4 KiB run in lockstep; each
    file takes its own consecutive chains.
    ``max_total`` caps the total size by truncating the list.
    """
    rng = np.random.default_rng([seed, 0x4D])
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_files)).astype(np.int64)
    parts = []
    total = 0
    for k, sz in enumerate(sizes):
        if max_total is not None and total + sz > max_total:
            break
        w = rng.dirichlet([1.0, 1.0, 1.0])
        n_img_b = int(sz * w[0])
        n_img = n_img_b // (512 * 512)
        img = image_bytes(n_img, seed * 7919 + k) if n_img else np.zeros(0, np.uint8)
        rem_img = n_img_b - img.size
        pcm_n = (int(sz * w[1]) + rem_img) // 2 * 2
        pcm = pcm_bytes(pcm_n, seed * 7919 + k)
        parts.append((img, pcm, int(sz) - img.size - pcm.size))
        total += int(sz)
    # all text in one lockstep run: file k owns ceil(n_txt / 4096) chains
    chunk = 4096
    nch = [-(-t // chunk) for _, _, t in parts]
    table = markov_table(3, 0.05, seed, rows=1 << 12)
    trng = np.random.default_rng([seed, 0x3D])
    body = np.zeros((0, chunk), np.uint8)
    if sum(nch):
        init = trng.integers(0, 256, size=(sum(nch), 3), dtype=np.uint8)

        def index(cols):
            h = (cols[0] * 65599 + cols[1]) * 65599 + cols[2]
            h = (h * 0x9E3779B1) & 0xFFFFFFFF
            return (h >> 16) % table.shape[0]

        body = _sample_chains(table, index, chunk, init, trng, 3)
    files = []
    c0 = 0
    for (img, pcm, t), m in zip(parts, nch):
        txt = body[c0:c0 + m].reshape(-1)[:t]
        c0 += m
        files.append(np.concatenate([img, pcm, txt]).astype(np.uint8))
    return files
