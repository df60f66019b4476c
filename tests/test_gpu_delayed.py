"""Delayed-update schedule on the GPU (EDPC_FLAG_DELAYED_UPDATE) against the
oracle's delayed schedule, through the C ABI (needs a GPU).

The schedule applies the gradient of step i, taken at the parameters that
predicted step i, after step i + 1; the adjoint of step i runs on a second
stream beside the forward pass of step i + 1. Checks:
  * lossless round trips (empty, shorter than K, ragged, several 64-step
    graph chunks plus an eager tail), FP32 and BF16;
  * the same bitstream from the graph and the eager launch paths and with
    the coder stage inline;
  * the code length within 0.5 % of the FP64 oracle's delayed schedule: the
    64 KiB order-2 Markov input (FP32), the 512-stream prefix of the 64 MiB
    mix (FP32 and BF16), and an uneven file set whose active streams drop
    out step by step (FP32), 2048 streams (BF16) and the 1 GiB workload's
    model dimensions (FP32);
  * the method variants (no LTE, three branches, one block) and a BF16 file set
    with tuned GEMM tiles stay lossless and deterministic;
  * the flag is recorded in the header and changes the bitstream;
  * rejected with FP8, with EDPC_FLAG_OVERLAP_FDM and by the model API.
"""
import json
import os

import numpy as np
import pytest

pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.compress import archive_split, archive_stream_len, oracle_compress  # noqa: E402
from oracle.model import Config  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DL = edpc.EDPC_FLAG_DELAYED_UPDATE
SMALL = dict(embed_dim=8, latent=64, hidden=64, blocks=2, seed=9)


def _payload(bits):
    _, n, b = edpc.peek(bits)
    return len(bits) - (88 + 4 * b + 4), n


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("n,b,K", [(0, 4, 4), (3, 4, 4), (1000, 7, 8), (4099, 16, 16), (20000, 64, 8),
                                   (60000, 8, 8)])
def test_delayed_round_trip(prec, n, b, K):
    x = np.random.default_rng(n).integers(0, 256, size=n).astype(np.uint8)
    if n > 100:
        x[: n // 2] = synth.markov_bytes(n // 2, 1, 0.05, n)
    c = edpc.make_cfg(streams=b, context=K, precision=prec, flags=DL, **SMALL)
    bits = edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(bits), x)


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
def test_delayed_launch_paths_give_one_bitstream(prec):
    # 30000 bytes over 8 streams: 58 chunks of 64 steps and an eager tail
    x = synth.markov_bytes(30000, 1, 0.05, 1)
    outs = []
    for extra in (0, edpc.EDPC_FLAG_NO_PIPELINE, edpc.EDPC_FLAG_NO_GRAPH):
        c = edpc.make_cfg(streams=8, context=8, precision=prec, flags=DL | extra, **SMALL)
        outs.append(edpc.compress(x, c))
    assert outs[0] == outs[1] == outs[2]
    assert np.array_equal(edpc.decompress(outs[0]), x)


def test_delayed_flag_is_in_the_header_and_changes_the_code():
    x = synth.markov_bytes(20000, 1, 0.05, 3)
    a = edpc.compress(x, edpc.make_cfg(streams=8, context=8, **SMALL))
    d = edpc.compress(x, edpc.make_cfg(streams=8, context=8, flags=DL, **SMALL))
    assert a != d
    assert a[44:48] == b"\0\0\0\0" and d[44:48] == b"\1\0\0\0"
    # the decoder takes the schedule from the header alone
    assert np.array_equal(edpc.decompress(d), x) and np.array_equal(edpc.decompress(a), x)


def test_delayed_small_workload_matches_oracle():
    g = json.load(open(os.path.join(GOLDEN, "oracle_c0_delayed.json")))
    tab = synth.markov_table(2, 0.1, g["data_seed"])
    x = synth.markov_bytes(g["n"], 2, 0.1, g["data_seed"], table=tab)
    assert bytes(x[:64]).hex() == g["input_sha_prefix"]
    c = edpc.make_cfg(streams=g["streams"], flags=DL, **g["cfg"])
    bits = edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(bits), x)
    code, n = _payload(bits)
    bpb = 8 * code / n
    assert abs(bpb - g["bits_per_byte"]) <= 0.005 * g["bits_per_byte"], (bpb, g["bits_per_byte"])


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
def test_delayed_mix_prefix_matches_oracle(prec):
    g = json.load(open(os.path.join(GOLDEN, "oracle_mix_prefix_delayed.json")))
    x = synth.multimedia_mix(g["total"], g["data_seed"])
    q = x.size // g["streams"]
    per = g["cfg"]["context"] + g["steps"]
    xp = np.ascontiguousarray(x[: q * g["streams"]].reshape(g["streams"], q)[:, :per]).reshape(-1)
    assert bytes(xp[:64]).hex() == g["input_sha_prefix"] and xp.size == g["n"]
    c = edpc.make_cfg(streams=g["streams"], precision=prec, flags=DL, **g["cfg"])
    bits = edpc.compress(xp, c)
    assert np.array_equal(edpc.decompress(bits), xp)
    code, _ = _payload(bits)
    delta = code / g["code_bytes"] - 1
    print("delayed, precision %d: delta %+.3f %%" % (prec, 100 * delta))
    assert abs(delta) <= 0.005


def test_delayed_file_set_matches_oracle():
    C0 = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=1)
    rng = np.random.default_rng(11)
    sizes = np.exp(rng.uniform(np.log(600), np.log(9000), size=14)).astype(np.int64)
    sizes[::7] = 0
    sizes[1] = 5
    x = synth.multimedia_mix(int(sizes.sum()), 11)
    files, o = [], 0
    for s in sizes:
        files.append(x[o:o + s].copy())
        o += s
    budget = 40
    sp = archive_split([int(s) for s in sizes], archive_stream_len([int(s) for s in sizes], budget))
    ref = oracle_compress(x, Config(**C0), 0, split=sp, delayed=True)
    o_bytes = sum(len(s) for s in ref["streams"])
    cfg = edpc.make_cfg(streams=budget, precision=edpc.EDPC_FP32, flags=DL, **C0)
    bits = edpc.compress_many(files, cfg)
    back = edpc.decompress_many(bits)
    for a, b in zip(files, back):
        assert np.array_equal(a, b)
    _, n, b = edpc.peek(bits)
    assert b == sp[0]
    g_bytes = len(bits) - (88 + 24 + 8 * len(files) + 4 * b + 4)
    assert abs(g_bytes - o_bytes) <= 0.005 * o_bytes, (g_bytes, o_bytes)


def test_delayed_rejected_combinations():
    x = np.zeros(100, dtype=np.uint8)
    for prec, extra in ((edpc.EDPC_FP8E4M3, 0), (edpc.EDPC_BF16, edpc.EDPC_FLAG_OVERLAP_FDM)):
        with pytest.raises(edpc.EdpcError):
            edpc.compress(x, edpc.make_cfg(streams=4, context=8, precision=prec, flags=DL | extra, **SMALL))
    with pytest.raises(edpc.EdpcError):
        edpc.Model(edpc.make_cfg(streams=4, context=8, flags=DL, **SMALL), 4)


@pytest.mark.parametrize("dims,b,steps,prec", [
    (dict(context=16, embed_dim=8, latent=128, hidden=128, blocks=2), 2048, 48, edpc.EDPC_BF16),
    (dict(context=64, embed_dim=16, latent=512, hidden=512, blocks=6), 8, 64, edpc.EDPC_FP32),
], ids=["2048-streams-bf16", "1g-model-dims-fp32"])
def test_delayed_against_oracle_at_large_batch_and_large_model(dims, b, steps, prec):
    # From 2048 streams the BF16 FDM adjoint also waits for the side stream;
    # the model of the 1 GiB workload (K = 64, F' = 512, 6 MBRBs of 512) takes
    # the F' = 512 kernels. Both against the oracle's delayed schedule on
    # prefix inputs (the oracle runs here, a minute or two of CPU).
    cfg = dict(branches=2, lr=1e-3, seed=1, **dims)
    x = synth.multimedia_mix(b * (dims["context"] + steps) * 4, 5)
    q = x.size // b
    xp = np.ascontiguousarray(x[: q * b].reshape(b, q)[:, : dims["context"] + steps]).reshape(-1)
    ref = oracle_compress(xp, Config(**cfg), b, delayed=True)
    o_bytes = sum(len(s) for s in ref["streams"])
    bits = edpc.compress(xp, edpc.make_cfg(streams=b, precision=prec, flags=DL, **cfg))
    assert np.array_equal(edpc.decompress(bits), xp)
    code, _ = _payload(bits)
    print("delayed %d: %d code bytes, oracle %d (%+.3f %%)" % (prec, code, o_bytes, 100 * (code / o_bytes - 1)))
    assert abs(code - o_bytes) <= 0.005 * o_bytes, (code, o_bytes)


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("variant", [dict(latent=0), dict(branches=3), dict(blocks=1)], ids=["no-lte", "k3", "one-block"])
def test_delayed_with_method_variants(prec, variant):
    # the variants of Table 4 / Table 5 under the delayed schedule: lossless and
    # deterministic (two encoder runs give one bitstream)
    dims = dict(context=8, embed_dim=8, latent=64, hidden=64, blocks=2, branches=2, seed=4)
    dims.update(variant)
    x = synth.markov_bytes(24000, 1, 0.05, 6)
    c = edpc.make_cfg(streams=16, precision=prec, flags=DL, **dims)
    a = edpc.compress(x, c)
    assert a == edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(a), x)


def test_delayed_tuned_file_set_round_trip_bf16():
    # BF16 file sets time every GEMM's tile at open (on parity 1's plan, whose
    # buffers stay zero); the decoder sets the recorded tiles without timing
    rng = np.random.default_rng(8)
    sizes = np.exp(rng.uniform(np.log(300), np.log(20000), size=9)).astype(np.int64)
    sizes[3] = 0
    x = synth.multimedia_mix(int(sizes.sum()), 8)
    files, o = [], 0
    for s in sizes:
        files.append(x[o:o + s].copy())
        o += s
    cfg = edpc.make_cfg(streams=64, precision=edpc.EDPC_BF16, flags=DL, context=16, embed_dim=8, latent=128,
                        hidden=128, blocks=2)
    bits = edpc.compress_many(files, cfg)
    for a, b in zip(files, edpc.decompress_many(bits)):
        assert np.array_equal(a, b)
