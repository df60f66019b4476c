"""Pins for the oracle's quantizer and range coder (CPU only)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.coder import T, RangeDecoder, RangeEncoder, quantize_cdf


# ---- quantizer ------------------------------------------------------------------

def test_quantize_uniform_closed_form():
    p = np.full(256, 1.0 / 256, dtype=np.float32)
    f, cum = quantize_cdf(p)
    # 1 + floor(65280/256) = 256 for every symbol, and the total is already T.
    assert np.all(f == 256)
    assert np.array_equal(cum, np.arange(257) * 256)


def test_quantize_one_hot_closed_form():
    p = np.zeros(256, dtype=np.float32)
    p[77] = 1.0
    f, cum = quantize_cdf(p)
    assert f[77] == T - 255 and np.all(np.delete(f, 77) == 1)
    assert cum[-1] == T


@pytest.mark.parametrize("idx,pmax,rest,fmax,frest,rem", [
    # two symbols tie at the largest frequency; the other 254 share the rest
    ((3, 7), 0.4, 0.2 / 254, 26113, 52, 102),
    ((9, 200), 0.4, 0.2 / 254, 26113, 52, 102),
    # a three-way tie that includes the first and the last symbol
    ((0, 128, 255), 0.3, 0.1 / 253, 19585, 26, 203),
])
def test_quantize_tie_gives_the_remainder_to_the_lowest_index(idx, pmax, rest, fmax, frest, rem):
    """Tied largest frequencies: the remainder T - sum(f) lands on the lowest
    tied index only (the quantizer's tie rule). Hand arithmetic: fl32(0.4) *
    65280 = 26112.0004 rounds to 26112.0 in FP32, so f = 26113;
    fl32(0.2/254) * 65280 = 51.40, f = 52; 2 * 26113 + 254 * 52 = 65434, so
    the remainder is 102. fl32(0.3) * 65280 = 19584.0008 -> 19584.0, f = 19585;
    fl32(0.1/253) * 65280 = 25.80, f = 26; 3 * 19585 + 253 * 26 = 65333,
    remainder 203."""
    p = np.full(256, rest, dtype=np.float32)
    p[list(idx)] = pmax
    f, cum = quantize_cdf(p)
    expect = np.full(256, frest, dtype=np.int64)
    expect[list(idx)] = fmax
    expect[min(idx)] += rem
    assert np.array_equal(f, expect)
    assert cum[-1] == T


def test_quantize_strict_maximum_after_a_tie_takes_the_remainder():
    """The remainder goes to the largest f even when a pair of smaller f tie
    earlier: p[1] = p[2] = 0.2 and p[250] = 0.4; the rest share 0.2."""
    p = np.full(256, 0.2 / 253, dtype=np.float32)
    p[[1, 2]] = 0.2
    p[250] = 0.4
    f, _ = quantize_cdf(p)
    # 1 + floor(fl32(0.2) * 65280) = 1 + 13056; 1 + floor(fl32(0.2/253) * 65280) = 1 + 51
    assert f[1] == f[2] == 13057
    base = 2 * 13057 + 26113 + 253 * 52
    assert f[250] == 26113 + (T - base)
    assert np.all(np.delete(f, [1, 2, 250]) == 52)


@pytest.mark.parametrize("alpha", [0.01, 0.1, 1.0, 10.0])
def test_quantize_invariants_and_error_bound(alpha):
    rng = np.random.default_rng(3)
    p = rng.dirichlet(np.full(256, alpha), size=400).astype(np.float32)
    f, cum = quantize_cdf(p)
    assert np.all(f >= 1)
    assert np.all(f.sum(1) == T)
    assert np.all(np.diff(cum, axis=1) == f)
    assert np.all(cum[:, 0] == 0) and np.all(cum[:, -1] == T)
    # f_j - 1 = floor(65280 p_j) gives |f_j/T - p_j| <= 256/T, except for the
    # symbol that takes the remainder (at most 256 more, or a few less).
    am = np.argmax(f, axis=1)
    err = np.abs(f / T - p.astype(np.float64))
    err[np.arange(len(am)), am] = 0
    assert err.max() <= 256 / T + 1e-7


def test_quantize_handles_sum_above_one():
    # FP32 probabilities can sum to slightly more than 1: the remainder is then
    # negative and comes off the largest frequency.
    p = np.full(256, np.float32(1.0 / 256) * np.float32(1.0000001), dtype=np.float32)
    p[0] = np.float32(0.5)
    p[1:] = np.float32(0.5 / 255 * 1.0001)
    f, cum = quantize_cdf(p)
    assert f.sum() == T and np.all(f >= 1)


# ---- range coder ------------------------------------------------------------------

def _random_symbols(rng, n, peaked):
    """n (cum, f, cdf) triples from random quantized CDFs."""
    out = []
    for _ in range(n):
        a = 0.02 if peaked else 1.0
        p = rng.dirichlet(np.full(256, a)).astype(np.float32)
        f, cum = quantize_cdf(p)
        s = int(rng.choice(256, p=f / f.sum()))
        out.append((s, int(cum[s]), int(f[s]), cum))
    return out


def _bigint_encode(pairs):
    """Unbounded-integer statement of the same interval arithmetic.

    The interval is [BL, BL + R) in units of 2^-(32 + 8k); renormalising
    scales both by 256. Carries need no handling here. The flush value is BL
    rounded up to a multiple of 2^24, written on 4 + k bytes.
    """
    BL, R, k = 0, 0xFFFFFFFF, 0
    for c, f in pairs:
        r = R >> 16
        BL += r * c
        R = R - r * c if c + f == T else r * f
        while R < (1 << 24):
            R <<= 8
            BL <<= 8
            k += 1
    V = (BL + (1 << 24) - 1) >> 24 << 24
    assert BL <= V < BL + R
    return V.to_bytes(4 + k, "big").rstrip(b"\x00")


@pytest.mark.parametrize("seed,peaked,n", [(0, False, 300), (1, True, 300), (2, True, 2000), (3, False, 1)])
def test_encoder_matches_unbounded_integer_coder(seed, peaked, n):
    rng = np.random.default_rng(seed)
    syms = _random_symbols(rng, n, peaked)
    enc = RangeEncoder()
    for _, c, f, _ in syms:
        enc.encode(c, f)
    out = enc.finish()
    assert out == _bigint_encode([(c, f) for _, c, f, _ in syms])
    dec = RangeDecoder(out)
    assert [dec.decode(cdf) for *_, cdf in syms] == [s for s, *_ in syms]


def test_carry_and_pending_ff_paths():
    # Symbols at the very top of the CDF push low towards 2^32, which forces
    # 0xFF pending bytes and carries; check against the unbounded coder.
    rng = np.random.default_rng(9)
    pairs = []
    for _ in range(3000):
        f = int(rng.integers(1, 40))
        c = T - f if rng.random() < 0.7 else int(rng.integers(0, T - f))
        pairs.append((c, f))
    enc = RangeEncoder()
    for c, f in pairs:
        enc.encode(c, f)
    out = enc.finish()
    assert out == _bigint_encode(pairs)
    assert b"\xff" in out


def test_empty_and_uniform_streams():
    assert RangeEncoder().finish() == b""
    rng = np.random.default_rng(4)
    data = rng.integers(0, 256, size=100)
    enc = RangeEncoder()
    for x in data:
        enc.encode(256 * int(x), 256)
    out = enc.finish()
    # Each uniform byte costs 8 bits plus the R >> 16 truncation loss.
    assert 8 * len(out) <= enc.ideal_bits + enc.trunc_bits + 16
    assert enc.ideal_bits == 800
    dec = RangeDecoder(out)
    assert [dec.decode_uniform() for _ in range(100)] == list(data)


def test_code_length_within_ideal_plus_truncation():
    rng = np.random.default_rng(5)
    for n in (10, 200, 5000):
        syms = _random_symbols(rng, n, True)
        enc = RangeEncoder()
        exact = Fraction(1)
        for _, c, f, _ in syms:
            enc.encode(c, f)
            exact *= Fraction(f, T)
        out = enc.finish()
        info = -(math.log2(exact.numerator) - math.log2(exact.denominator))
        assert abs(info - enc.ideal_bits) < 1e-6 * max(1.0, info)
        assert 8 * len(out) <= enc.ideal_bits + enc.trunc_bits + 16
        assert enc.trunc_bits <= n * 0.0057
