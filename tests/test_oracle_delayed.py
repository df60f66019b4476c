"""Pins for the oracle's delayed-update schedule (CPU only).

The schedule: step i predicts with theta_i, its gradient g_i is taken at
theta_i, and the update after step i applies g_{i-1}:
theta_{i+1} = Adam(theta_i, g_{i-1}), theta_{K+1} = theta_K. The pins build
that trajectory from pieces the schedule does not share (Algorithm 1's own
first step, and a fresh model's gradient at the stale parameters), so an
update applied on time, a gradient taken at the updated parameters, a wrong
Adam counter, or FDM rows taken from the wrong step fails one of them.
"""
import numpy as np
import pytest

import synth
from oracle.coder import T, quantize_cdf
from oracle.compress import _contexts, oracle_compress, oracle_decompress, split_streams
from oracle.model import Config, Model, softmax

TINY = dict(embed_dim=4, latent=8, hidden=8, blocks=2, branches=2, lr=1e-2)


def tiny(K=3, seed=3, **kw):
    d = dict(TINY)
    d.update(kw)
    return Config(context=K, seed=seed, **d)


def state(m: Model):
    return np.concatenate([m.flat("P"), m.flat("m"), m.flat("v"), m.U.ravel(), m.mU.ravel(), m.vU.ravel()]), m.t


def same_state(a: Model, b: Model):
    sa, ta = state(a)
    sb, tb = state(b)
    return ta == tb and np.array_equal(sa, sb)


def data(n=600, seed=4):
    return synth.markov_bytes(n, 1, 0.1, seed)


@pytest.mark.parametrize("n,b,K", [(0, 3, 3), (5, 3, 3), (600, 3, 3), (601, 4, 2), (257, 7, 4)])
def test_delayed_round_trip(n, b, K):
    x = data(n, n) if n else np.zeros(0, dtype=np.uint8)
    cfg = tiny(K)
    r = oracle_compress(x, cfg, b, delayed=True)
    y = oracle_decompress(r["streams"], n, cfg, b, delayed=True)
    assert np.array_equal(x, y)


def test_delayed_round_trip_with_ragged_file_set():
    from oracle.compress import archive_split
    sizes = [40, 7, 95, 0, 3]
    x = data(sum(sizes), 9)
    sp = archive_split(sizes, 30)
    cfg = tiny(3)
    r = oracle_compress(x, cfg, 0, split=sp, delayed=True)
    assert np.array_equal(oracle_decompress(r["streams"], x.size, cfg, 0, split=sp, delayed=True), x)


def test_no_update_after_the_first_step():
    x = data()
    cfg = tiny()
    r = oracle_compress(x, cfg, 3, max_steps=1, delayed=True)
    assert same_state(r["model"], Model(cfg, r["b"]))


def test_first_update_is_algorithm_1s_first():
    # theta_{K+2} = Adam(theta_K, g_K): Algorithm 1's state after one step.
    x = data()
    cfg = tiny()
    d = oracle_compress(x, cfg, 3, max_steps=2, delayed=True)["model"]
    a = oracle_compress(x, cfg, 3, max_steps=1)["model"]
    assert same_state(d, a)


def test_second_update_uses_the_gradient_at_the_stale_parameters():
    # theta_{K+3} = Adam_2(theta_{K+2}, g_{K+1}) with g_{K+1} taken at
    # theta_{K+1} = theta_K, i.e. by a fresh model on step K+1's contexts.
    x = data()
    cfg = tiny()
    b, off, ln = split_streams(x.size, 3, cfg.context)
    i = cfg.context + 1
    rows = np.nonzero(ln > i)[0]
    ctx = _contexts(x, off, rows, i, cfg.context)
    tgt = x[off[rows] + i].astype(np.int64)
    fresh = Model(cfg, b)
    _, g, dU, _ = fresh.grad_step(ctx, tgt, rows)
    want = oracle_compress(x, cfg, 3, max_steps=1)["model"]  # theta_{K+2}, t = 1
    want.adam(g, dU, rows)
    got = oracle_compress(x, cfg, 3, max_steps=3, delayed=True)["model"]
    assert same_state(got, want)
    # and the gradient at the updated parameters would give another state
    other = oracle_compress(x, cfg, 3, max_steps=1)["model"]
    _, g2, dU2, _ = oracle_compress(x, cfg, 3, max_steps=1)["model"].grad_step(ctx, tgt, rows)
    other.adam(g2, dU2, rows)
    assert not same_state(got, other)


def test_prediction_of_step_k_plus_2_uses_the_first_update():
    # The ideal code length of the first three model steps (quantized CDF):
    # steps K and K+1 are predicted by theta_K, step K+2 by Algorithm 1's
    # theta after one step.
    x = data()
    cfg = tiny()
    b, off, ln = split_streams(x.size, 3, cfg.context)
    K = cfg.context
    fresh = Model(cfg, b)
    one = oracle_compress(x, cfg, 3, max_steps=1)["model"]
    bits = 0.0
    for i, m in ((K, fresh), (K + 1, fresh), (K + 2, one)):
        rows = np.nonzero(ln > i)[0]
        z, _ = m.forward(_contexts(x, off, rows, i, K), rows)
        f, _ = quantize_cdf(softmax(z).astype(np.float32))
        bits += float(-np.log2(f[np.arange(len(rows)), x[off[rows] + i]] / T).sum())
    r = oracle_compress(x, cfg, 3, max_steps=3, delayed=True)
    # ideal_bits adds the uniform prefix (8 bits per byte) to the model-coded bytes
    assert abs(float(r["ideal_bits"].sum()) - 8.0 * K * b - bits) < 1e-6 * bits


def test_zero_learning_rate_makes_both_schedules_equal():
    x = data(800, 5)
    cfg = tiny(lr=0.0)
    a = oracle_compress(x, cfg, 4)
    d = oracle_compress(x, cfg, 4, delayed=True)
    assert a["streams"] == d["streams"]


def test_delayed_schedule_still_learns():
    # An i.i.d. source of entropy H = 3.74 bits: both schedules end within
    # 0.25 bit/byte of H, and the delayed one within 1 % of Algorithm 1
    # (an informative bound, not a property of the method).
    tab = synth.markov_table(0, 0.05, 11)
    H = synth.markov_entropy_rate(tab, 0)
    x = synth.markov_bytes(6000, 0, 0.05, 11, table=tab)
    cfg = tiny(2, lr=1e-2)
    a = oracle_compress(x, cfg, 2)
    d = oracle_compress(x, cfg, 2, delayed=True)
    ba = 8 * sum(len(s) for s in a["streams"]) / x.size
    bd = 8 * sum(len(s) for s in d["streams"]) / x.size
    assert ba < H + 0.25 and bd < H + 0.25, (H, ba, bd)
    assert abs(bd - ba) <= 0.01 * ba, (ba, bd)


def test_delayed_update_uses_the_rows_active_at_the_gradients_step():
    # Stream 0 (K + 2 bytes) is active at steps K and K + 1 only, stream 1
    # (K + 6 bytes) throughout. The update after step K + 2 applies g_{K+1},
    # so stream 0's FDM still moves then, with its own gradient of step K + 1.
    from oracle.compress import archive_split
    cfg = tiny(3)
    K = cfg.context
    sizes = [K + 2, K + 6]
    sp = archive_split(sizes, 100)
    x = data(sum(sizes), 13)
    b, off, ln = sp
    i = K + 1
    rows = np.nonzero(ln > i)[0]
    assert list(rows) == [0, 1]
    _, g, dU, _ = Model(cfg, b).grad_step(_contexts(x, off, rows, i, K), x[off[rows] + i].astype(np.int64), rows)
    want = oracle_compress(x, cfg, 0, split=sp, max_steps=1)["model"]
    want.adam(g, dU, rows)
    got = oracle_compress(x, cfg, 0, split=sp, max_steps=3, delayed=True)["model"]
    assert same_state(got, want)
    # stream 0's FDM did change in that update (it is inactive at step K + 2)
    before = oracle_compress(x, cfg, 0, split=sp, max_steps=2, delayed=True)["model"]
    assert not np.array_equal(got.U[0], before.U[0])
