"""The "w/o LTE" variant of Table 4 (cfg latent = 0) against the FP64 oracle (needs a GPU).

Without the LTE each stream's FDM is F x F and acts on the last Local block's
output directly (y_s = x_s U_s, no projections). Checked through the C ABI:
  * initial state bit-identical to the oracle's (the canonical order has no
    LTE tensors, so the head's tensor ids move up);
  * logits and every tensor's gradient, FP32 (1e-4 / 1e-3) and BF16
    (3e-2 / 6e-2), with an inactive stream whose FDM gradient must be zero;
  * compress / decompress round trips, and FP32 bits/byte within 2 % of the
    oracle's on the same small input.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.compress import oracle_compress  # noqa: E402
from oracle.model import Config, Model as OModel, softmax  # noqa: E402

pytestmark = pytest.mark.gpu

DIMS = dict(context=8, embed_dim=16, latent=0, hidden=64, blocks=3, branches=2, lr=1e-3, seed=13)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


def test_initial_state_is_bit_identical():
    b = 5
    m = edpc.Model(edpc.make_cfg(**DIMS), b)
    om = OModel(Config(**DIMS), b)
    st = m.get_state()
    assert np.array_equal(st["P"], om.flat().astype(np.float32))
    assert np.array_equal(st["U"], om.U.reshape(-1).astype(np.float32))
    assert edpc.param_count(edpc.make_cfg(**DIMS)) == om.flat().size
    m.close()


@pytest.mark.parametrize("prec,tz,tg", [(edpc.EDPC_FP32, 1e-4, 1e-3), (edpc.EDPC_BF16, 3e-2, 6e-2)],
                         ids=["fp32", "bf16"])
@pytest.mark.parametrize("blocks", [3, 1])
def test_forward_and_gradient_parity(prec, tz, tg, blocks):
    dims = dict(DIMS, blocks=blocks)
    b = 9
    m = edpc.Model(edpc.make_cfg(precision=prec, **dims), b)
    o = Config(**dims)
    om = OModel(o, b)
    rng = np.random.default_rng(blocks)
    for _ in range(2):  # move every tensor off its initial value
        m.train_step(rng.integers(0, 256, size=(b, o.context)).astype(np.uint8),
                     rng.integers(0, 256, size=b).astype(np.uint8), np.ones(b, np.uint8))
    st = m.get_state()
    om.set_flat(st["P"].astype(np.float64))
    om.U = st["U"].astype(np.float64).reshape(om.U.shape).copy()
    ctx = rng.integers(0, 256, size=(b, o.context)).astype(np.uint8)
    z, _ = m.forward(ctx)
    zo, _ = om.forward(ctx.astype(np.int64))
    assert np.abs(z - zo).max() <= tz * np.abs(zo).max()
    t = rng.integers(0, 256, size=b).astype(np.uint8)
    active = np.ones(b, np.uint8)
    active[-1] = 0
    g, gu = m.backward(ctx, t, active)
    rows = np.nonzero(active)[0]
    dz = softmax(zo[rows])
    dz[np.arange(len(rows)), t[rows]] -= 1
    dz /= len(rows)
    _, cache = om.forward(ctx[rows].astype(np.int64), rows)
    go, dUo = om.backward(cache, dz)
    off = 0
    for name, shape, _ in om.layout:
        n = int(np.prod(shape))
        ref = go[name].ravel()
        if np.linalg.norm(ref) > 1e-12:
            assert _rel(g[off:off + n], ref) <= tg, (name, _rel(g[off:off + n], ref))
        off += n
    F = o.F
    gu = gu.reshape(b, F, F)
    assert _rel(gu[rows], dUo) <= tg
    assert not gu[active == 0].any()
    m.close()


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
def test_roundtrip_and_bits_per_byte(prec):
    x = synth.markov_bytes(4000, 1, 0.1, 3)
    dims = dict(DIMS, context=4, embed_dim=16, hidden=32, blocks=2)
    cfg = edpc.make_cfg(streams=4, precision=prec, **dims)
    bits = edpc.compress(x, cfg)
    assert np.array_equal(edpc.decompress(bits), x)
    if prec == edpc.EDPC_FP32:
        ref = oracle_compress(x, Config(**dims), 4)
        ref_bits = 8 * sum(len(s) for s in ref["streams"])
        _, n, be = edpc.peek(bits)
        got = 8 * (len(bits) - (88 + 4 * be + 4))
        assert abs(got - ref_bits) <= 0.005 * ref_bits, (got, ref_bits)
