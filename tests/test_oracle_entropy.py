"""Entropy pins of the oracle's code length on the small order-2 Markov
workload (64 KiB, every transition row Dirichlet(0.1); CPU only).

What fixes the numbers, with no implementation to compare against:

* Lower bound (competitive optimality of the source code, Barron 1985): for
  any uniquely decodable code and any c > 0, the probability under the source
  that L(x) < -log2 P(x) - c is at most 2^-c. The oracle's output for x (the
  per-stream byte strings plus their 32-bit lengths, n and b being known) is
  such a code, and P(x) is known exactly: the chain's first two bytes are
  uniform and every later byte has probability table[ctx, x_i]. With c = 20
  a correct oracle fails this with probability below 1e-6, while an oracle
  whose prediction sees the byte it codes (an off-by-one context) drops far
  below it.
* The entropy rate H (power iteration over the 65,536 contexts) and the
  sample's own log-loss agree within 3 sigma of the per-byte log-loss.
* Reference: the adaptive Krichevsky-Trofimov code of order k has the
  closed-form length sum over contexts of log2 of the Dirichlet(1/2)-
  multinomial, written here from the sample's counts and pinned against its
  sequential definition (product of (n_c + 1/2) / (N + 128)).
* Upper bound (reading, see the design notes): Algorithm 1 has no escape to
  the uniform code, so an online-learned model may expand a source it cannot
  learn within its length; on this sample the closed-form order-1 KT code
  expands too (8.24 bits/byte). The bound allows one bit per byte of
  learning cost: <= 9 bits/byte. A gradient of the wrong sign (planted in the
  oracle on a prefix) breaks it.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import gammaln

import synth
from oracle.compress import oracle_compress
from oracle.model import Config, Model

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_c0.json")
DATA_SEED = 20250718
C0 = Config(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=1)
BARRON_C = 20.0
UPPER_BPB = 9.0


def kt_bits(x, order, a=0.5):
    """Length in bits of the adaptive order-`order` Dirichlet(a)-multinomial
    code of x (the first `order` bytes cost 8 bits each)."""
    x = np.asarray(x, dtype=np.int64)
    n = x.size
    if n <= order:
        return 8.0 * n
    ctx = np.zeros(n - order, np.int64)
    for k in range(order):
        ctx = ctx * 256 + x[k:n - order + k]
    key = ctx * 256 + x[order:]
    _, cnt = np.unique(key, return_counts=True)
    _, tot = np.unique(ctx, return_counts=True)
    nats = (gammaln(256 * a + tot) - gammaln(256 * a)).sum() - (gammaln(a + cnt) - gammaln(a)).sum()
    return nats / math.log(2) + 8.0 * order


def kt_bits_sequential(x, order, a=0.5):
    """The same code length by its definition: each byte costs
    -log2((n_c(x_i) + a) / (N_c + 256 a)) with the counts seen so far."""
    counts = {}
    bits = 8.0 * min(order, len(x))
    for i in range(order, len(x)):
        c = tuple(int(v) for v in x[i - order:i])
        row = counts.setdefault(c, np.zeros(256))
        bits -= math.log2((row[x[i]] + a) / (row.sum() + 256 * a))
        row[x[i]] += 1
    return bits


def source_bits(x, table):
    """-log2 P(x) under the order-2 source (two uniform bytes, then the rows)."""
    x = np.asarray(x, dtype=np.int64)
    ctx = x[:-2] * 256 + x[1:-1]
    return 16.0 + float(-np.log2(table[ctx, x[2:]]).sum())


@pytest.fixture(scope="module")
def c0():
    table = synth.markov_table(2, 0.1, DATA_SEED)
    x = synth.markov_bytes(65536, 2, 0.1, DATA_SEED, table=table)
    with open(GOLD) as f:
        gold = json.load(f)
    return table, x, gold


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("a", [0.5, 0.1])
def test_kt_closed_form_equals_sequential_definition(order, a):
    rng = np.random.default_rng(order)
    x = rng.integers(0, 6, size=300)  # few symbols: contexts repeat
    assert kt_bits(x, order, a) == pytest.approx(kt_bits_sequential(x, order, a), rel=1e-12)


def test_kt_special_cases():
    # one byte costs 8 bits at order 0; a constant run of n bytes costs
    # -sum_i log2((i + 1/2) / (i + 128))
    assert kt_bits(np.array([7]), 0) == pytest.approx(8.0)
    n = 50
    want = -sum(math.log2((i + 0.5) / (i + 128)) for i in range(n))
    assert kt_bits(np.full(n, 9), 0) == pytest.approx(want, rel=1e-12)


def log_loss_var(table, x):
    """Per-byte variance of -log2 P(x_i | ctx) over the sample's contexts
    (the i.i.d. approximation of the chain's log-loss variance)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        lg = np.where(table > 0, -np.log2(table), 0.0)
    h_rows = (table * lg).sum(axis=1)
    m2_rows = (table * lg * lg).sum(axis=1)
    ctx = x[:-2].astype(np.int64) * 256 + x[1:-1]
    return float(m2_rows[ctx].mean() - h_rows[ctx].mean() ** 2)


def test_entropy_rate_matches_the_sample_log_loss(c0):
    table, x, gold = c0
    H = synth.markov_entropy_rate(table, 2)
    assert H == pytest.approx(gold["entropy_rate_bits"], rel=1e-9)
    n = x.size - 2
    ll = source_bits(x, table) - 16.0
    assert abs(ll - n * H) <= 3.0 * math.sqrt(n * log_loss_var(table, x))


def test_c0_code_length_is_above_the_source_bound(c0):
    """Lower pins: the oracle's stored 64 KiB result against -log2 P(x) - 20
    bits (Barron) and against n (H - 3 sigma)."""
    table, x, gold = c0
    assert bytes(x[:64]).hex() == gold["input_sha_prefix"]
    code_bits = 8.0 * sum(gold["stream_bytes"]) + 32.0 * len(gold["stream_bytes"])
    assert code_bits >= source_bits(x, table) - BARRON_C
    H = gold["entropy_rate_bits"]
    sigma = math.sqrt(log_loss_var(table, x) / x.size)  # of the per-byte mean
    assert gold["bits_per_byte"] >= H - 3 * sigma


def test_c0_code_length_upper_reading(c0):
    """Upper pin (reading): at most 9 bits/byte. Beside it, the closed-form
    references on the same sample: order-0 and order-2 KT lie below 8 bits/byte,
    order-1 KT above (an adaptive code expands this input too)."""
    table, x, gold = c0
    assert gold["bits_per_byte"] <= UPPER_BPB
    n = x.size
    kt = [kt_bits(x, k) / n for k in (0, 1, 2)]
    assert kt[0] < 8.05 and kt[2] < 8.0 < kt[1]
    # the stored stream lengths reproduce the stored bits/byte
    assert gold["bits_per_byte"] == pytest.approx(8.0 * sum(gold["stream_bytes"]) / n)


def _prefix_run(x, flip=False):
    if not flip:
        return oracle_compress(x, C0, 4)
    orig = Model.adam

    def ascent(self, grads, dU, rows=None):  # planted mistake: the gradient's sign
        return orig(self, {k: -v for k, v in grads.items()}, -dU, rows)

    Model.adam = ascent
    try:
        return oracle_compress(x, C0, 4)
    finally:
        Model.adam = orig


def test_c0_prefix_fresh_run_within_both_bounds_and_planted_sign_breaks_upper(c0):
    """A fresh oracle run on the first 2 KiB of the chain (4 streams) lies
    between the lower and the upper pin; the same run with the gradient's sign
    flipped in the oracle's update exceeds the upper pin."""
    table, x, _ = c0
    xs = x[:2048].copy()
    lo = source_bits(xs, table) - BARRON_C
    r = _prefix_run(xs)
    bits = 8.0 * sum(len(s) for s in r["streams"]) + 32.0 * len(r["streams"])
    assert lo <= bits and 8.0 * sum(len(s) for s in r["streams"]) / xs.size <= UPPER_BPB
    rf = _prefix_run(xs, flip=True)
    assert 8.0 * sum(len(s) for s in rf["streams"]) / xs.size > UPPER_BPB
