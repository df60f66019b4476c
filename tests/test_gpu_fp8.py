"""FP8 e4m3 GEMMs (per-tensor power-of-two scales, FP32 accumulation; needs a GPU).

Tolerances follow from the format: e4m3 keeps 3 fraction bits, so each
quantized operand carries a relative error of at most 2^-4 (6.25 %), about
3.6 % RMS for uniformly spread mantissas, and a product of two quantized
operands about 5 % RMS. Summed over many terms with independent errors a
GEMM output keeps about that relative RMS error, and the model stacks about
ten GEMMs (with residual paths) before the logits. The checks are therefore
relative norms: logits within 15 %, every tensor's gradient within 30 % of
the FP64 oracle's; and compression stays lossless with bits/byte within 3 %
of the oracle's on the small workload.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.model import Config, Model as OModel, softmax  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


@pytest.mark.parametrize("dims,b", [(dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2,
                                          lr=1e-3, seed=1), 64),
                                    (dict(context=8, embed_dim=16, latent=136, hidden=200, blocks=3, branches=3,
                                          lr=1e-3, seed=5), 300)])
def test_fp8_forward_and_gradients_against_oracle(dims, b):
    c = edpc.make_cfg(precision=edpc.EDPC_FP8E4M3, **dims)
    m = edpc.Model(c, b)
    om = OModel(Config(**dims), b)
    rng = np.random.default_rng(b)
    K = dims["context"]
    ctx = rng.integers(0, 256, size=(b, K)).astype(np.uint8)
    z, _ = m.forward(ctx)
    zo, cache = om.forward(ctx.astype(np.int64))
    ez = _rel(z, zo)
    tg = rng.integers(0, 256, size=b).astype(np.uint8)
    g, gu = m.backward(ctx, tg, np.ones(b, np.uint8))
    dz = softmax(zo)
    dz[np.arange(b), tg] -= 1
    dz /= b
    go, dUo = om.backward(cache, dz)
    gf = OModel.flat_grads(om.layout, go)
    errs = {}
    off = 0
    for name, shape, _ in om.layout:
        n = int(np.prod(shape))
        if np.linalg.norm(gf[off:off + n]) > 1e-12:
            errs[name] = _rel(g[off:off + n], gf[off:off + n])
        off += n
    eu = _rel(gu.reshape(dUo.shape), dUo)
    print("fp8 rel errors: logits %.4f fdm %.4f worst grad %.4f (%s)" %
          (ez, eu, max(errs.values()), max(errs, key=errs.get)))
    assert ez <= 0.15
    assert eu <= 0.30
    for k, v in errs.items():
        assert v <= 0.30, (k, v)
    m.close()


def test_fp8_is_closer_to_bf16_than_the_format_bound():
    """The FP8 and BF16 paths agree to the FP8 rounding level on one forward."""
    dims = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=2)
    b = 128
    ctx = np.random.default_rng(3).integers(0, 256, size=(b, 16)).astype(np.uint8)
    z8, _ = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_FP8E4M3, **dims), b).forward(ctx)
    zb, _ = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_BF16, **dims), b).forward(ctx)
    assert 0 < _rel(z8, zb) <= 0.15


@pytest.mark.parametrize("code", [1, 2, 4, 8, 17, 24])
def test_fp8_tile_codes(code):
    dims = dict(context=8, embed_dim=16, latent=136, hidden=200, blocks=2, branches=2, lr=1e-3, seed=6)
    b = 200
    m = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_FP8E4M3, **dims), b)
    m.set_tiles(np.full(144, code, np.uint8))
    om = OModel(Config(**dims), b)
    ctx = np.random.default_rng(code).integers(0, 256, size=(b, 8)).astype(np.uint8)
    z, _ = m.forward(ctx)
    zo, _ = om.forward(ctx.astype(np.int64))
    assert _rel(z, zo) <= 0.15
    m.close()


def test_fp8_small_workload_roundtrip_and_bits_per_byte():
    g = json.load(open(os.path.join(GOLDEN, "oracle_c0.json")))
    table = synth.markov_table(2, 0.1, g["data_seed"])
    x = synth.markov_bytes(g["n"], 2, 0.1, g["data_seed"], table=table)
    c = edpc.make_cfg(streams=g["streams"], precision=edpc.EDPC_FP8E4M3, **g["cfg"])
    bits = edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(bits), x)
    _, n, b = edpc.peek(bits)
    bpb = 8 * (len(bits) - (88 + 4 * b + 4)) / n
    print("fp8 bits/byte %.4f oracle %.4f" % (bpb, g["bits_per_byte"]))
    assert abs(bpb - g["bits_per_byte"]) <= 0.03 * g["bits_per_byte"]


def test_fp8_multimedia_roundtrip():
    x = synth.multimedia_mix(1 << 20, 20250719)
    c = edpc.make_cfg(streams=512, context=32, embed_dim=16, latent=256, hidden=256, blocks=4,
                      precision=edpc.EDPC_FP8E4M3, seed=1)
    bits = edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(bits), x)
