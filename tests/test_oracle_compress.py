"""Pins for Algorithm 1 as run by the oracle (CPU only)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle.coder import T, RangeDecoder, RangeEncoder, quantize_cdf
from oracle.compress import (archive_split, archive_stream_len, oracle_compress, oracle_decompress,
                             split_streams)
from oracle.model import Config, Model, softmax

TINY = dict(embed_dim=4, latent=8, hidden=8, blocks=2, branches=2, lr=1e-3)


def tiny(K=2, seed=1, **kw):
    d = dict(TINY)
    d.update(kw)
    return Config(context=K, seed=seed, **d)


@pytest.mark.parametrize("n,b,K", [(0, 4, 2), (1, 4, 2), (7, 4, 2), (100, 3, 5), (1001, 8, 3), (64, 64, 1)])
def test_split_partitions_input(n, b, K):
    be, off, ln = split_streams(n, b, K)
    assert 1 <= be <= b
    assert ln.sum() == n and np.all(ln.max() - ln.min() <= 1)
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(ln)[:-1]]))
    if n >= K:
        assert be <= n // K


@pytest.mark.parametrize("sizes,L", [([], 4), ([0, 0], 3), ([5], 1), ([5], 5), ([5], 2), ([10, 0, 3, 17], 4),
                                     ([4096, 70000, 1, 65536], 65536), ([9, 8, 7], 100)])
def test_archive_split_partitions_each_file(sizes, L):
    b, off, ln = archive_split(sizes, L)
    assert b == len(ln) == len(off)
    if sum(sizes) == 0:
        assert b == 1 and ln[0] == 0
        return
    assert b == sum(-(-n // L) for n in sizes)
    # the streams tile the concatenation in order, none crossing a file boundary
    assert off[0] == 0 and np.array_equal(off[1:], off[:-1] + ln[:-1])
    ends = np.cumsum(sizes)
    starts = ends - np.array(sizes)
    s = 0
    for n, a, e in zip(sizes, starts, ends):
        m = -(-n // L)
        piece = ln[s:s + m]
        assert piece.sum() == n and (m == 0 or piece.max() - piece.min() <= 1)
        assert np.all(piece <= L) and np.all(np.diff(piece) <= 0)
        assert np.all((off[s:s + m] >= a) & (off[s:s + m] + piece <= e))
        s += m


@pytest.mark.parametrize("sizes", [[1], [7, 3], [100, 1, 50, 0, 33], [4096, 9000, 70000]])
def test_archive_stream_len_is_the_smallest_that_fits(sizes):
    count = lambda L: sum(-(-n // L) for n in sizes if n)
    for budget in (1, 2, 3, 5, 17, 64, 10 ** 6):
        L = archive_stream_len(sizes, budget)
        nz = sum(1 for n in sizes if n)
        if budget >= nz:
            assert count(L) <= budget
            assert L == 1 or count(L - 1) > budget
        else:
            assert L == max(sizes)


def test_archive_roundtrip_with_uneven_streams():
    """Streams of very different lengths (some shorter than K, one empty file)."""
    rng = np.random.default_rng(5)
    sizes = [1, 0, 40, 7, 95]
    data = rng.integers(0, 256, size=sum(sizes)).astype(np.uint8)
    cfg = tiny(3)
    sp = archive_split(sizes, 32)
    r = oracle_compress(data, cfg, 0, split=sp)
    assert r["b"] == 1 + 2 + 1 + 3
    y = oracle_decompress(r["streams"], data.size, cfg, 0, split=sp)
    assert np.array_equal(y, data)


@pytest.mark.parametrize("n,b,K,latent", [(0, 2, 2, 8), (1, 2, 2, 8), (5, 3, 2, 8), (300, 4, 3, 8), (257, 5, 2, 8),
                                           (300, 4, 3, 0)])
def test_roundtrip_small(n, b, K, latent):
    # latent = 0: the "w/o LTE" variant of Table 4
    x = np.random.default_rng(n + b).integers(0, 256, size=n).astype(np.uint8)
    cfg = tiny(K, latent=latent)
    r = oracle_compress(x, cfg, b)
    y = oracle_decompress(r["streams"], n, cfg, b)
    assert np.array_equal(x, y)


def test_code_length_bound_per_stream():
    x = synth.markov_bytes(3000, 1, 0.05, 7)
    cfg = tiny(3)
    r = oracle_compress(x, cfg, 3)
    for s, bs in enumerate(r["streams"]):
        assert 8 * len(bs) <= r["ideal_bits"][s] + r["trunc_bits"][s] + 16
        # and no better than the information content by more than a byte
        assert 8 * len(bs) >= r["ideal_bits"][s] - 8


def test_exact_rational_interval_on_short_inputs():
    """<= 8-byte inputs: the output value lies in the coder's nested interval
    (as exact integers), and its length is fixed by the rational width."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(1, 9))
        K = int(rng.integers(1, 3))
        x = rng.integers(0, 256, size=n).astype(np.uint8)
        cfg = tiny(K, seed=trial)
        m = Model(cfg, 1)
        pairs = [(256 * int(v), 256) for v in x[:K]]
        for i in range(K, n):
            z, cache = m.forward(x[None, i - K:i].astype(np.int64), [0])
            p = softmax(z)
            f, cum = quantize_cdf(p.astype(np.float32))
            pairs.append((int(cum[0, x[i]]), int(f[0, x[i]])))
            dz = p.copy()
            dz[0, x[i]] -= 1
            g, dU = m.backward(cache, dz)
            m.adam(g, dU, [0])
        r = oracle_compress(x, cfg, 1)
        out = r["streams"][0]
        # exact nested intervals with unbounded integers
        BL, R, k = 0, 0xFFFFFFFF, 0
        W = Fraction(1)
        for c, f in pairs:
            r_ = R >> 16
            BL += r_ * c
            R = R - r_ * c if c + f == T else r_ * f
            W *= Fraction(f, T)
            while R < (1 << 24):
                R, BL, k = R << 8, BL << 8, k + 1
        V = int.from_bytes(out.ljust(4 + k, b"\x00")[:4 + k], "big") if out else 0
        assert len(out) <= 4 + k
        assert BL <= V < BL + R
        info = math.log2(W.denominator) - math.log2(W.numerator)
        assert 8 * len(out) <= info + r["trunc_bits"][0] + 16


def test_all_two_byte_inputs_are_distinct_and_decode():
    """b = 1, K = 1: every one of the 65536 two-byte inputs gets its own code."""
    cfg = tiny(1, seed=3)
    m = Model(cfg, 1)
    z, _ = m.forward(np.arange(256)[:, None], rows=np.zeros(256, dtype=np.int64))
    f, cum = quantize_cdf(softmax(z).astype(np.float32))
    codes = {}
    for a in range(256):
        for x in range(256):
            e = RangeEncoder()
            e.encode(256 * a, 256)
            e.encode(int(cum[a, x]), int(f[a, x]))
            codes[(a, x)] = e.finish()
    assert len(set(codes.values())) == 65536
    rng = np.random.default_rng(0)
    for a, x in rng.integers(0, 256, size=(300, 2)):
        d = RangeDecoder(codes[(a, x)])
        assert d.decode_uniform() == a
        assert d.decode(cum[a]) == x
    # the full pipeline agrees with the direct coding on a sample
    for a, x in rng.integers(0, 256, size=(20, 2)):
        r = oracle_compress(np.array([a, x], dtype=np.uint8), cfg, 1)
        assert r["streams"][0] == codes[(a, x)]


# ---- entropy pins ---------------------------------------------------------------------

def test_uniform_random_bytes_cost_at_least_8_bits():
    n = 4096
    x = np.random.default_rng(12).integers(0, 256, size=n).astype(np.uint8)
    r = oracle_compress(x, tiny(2), 4)
    bits = 8 * sum(len(s) for s in r["streams"])
    # No code beats the entropy of uniform bytes by k bits except with
    # probability 2^-k; allow 64 bits.
    assert bits >= 8 * n - 64
    assert bits <= 8.2 * n


def test_constant_input_floor_from_quantizer_cap():
    n, b, K = 4096, 2, 2
    x = np.full(n, 65, dtype=np.uint8)
    r = oracle_compress(x, tiny(K), b)
    bits = 8 * sum(len(s) for s in r["streams"])
    # f <= T - 255 caps p at (T-255)/T, so each model-coded byte costs at least
    # -log2((T-255)/T) bits; the K prefix bytes of each stream cost 8 bits.
    floor = b * K * 8 + (n - b * K) * -math.log2((T - 255) / T)
    assert bits >= floor - 16 * b
    assert bits / n < 0.5


def test_iid_source_approaches_entropy():
    tab = synth.markov_table(0, 0.3, 21)
    H = synth.markov_entropy_rate(tab, 0)
    n = 16384
    x = synth.markov_bytes(n, 0, 0.3, 21, table=tab)
    emp = np.bincount(x, minlength=256) / n
    with np.errstate(divide="ignore", invalid="ignore"):
        H_emp = -np.nansum(np.where(emp > 0, emp * np.log2(emp), 0))
    r = oracle_compress(x, tiny(2, seed=5), 4)
    bpb = 8 * sum(len(s) for s in r["streams"]) / n
    # A sequential code for i.i.d. data does not beat the sample's empirical
    # entropy except by chance; adaptive learning on 16 KiB costs at most
    # ~1 bit/byte here.
    assert bpb >= H_emp - 0.05
    assert bpb <= H + 1.0, (bpb, H)
