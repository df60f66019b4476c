"""File sets (many files of uneven size in one batch) and GEMM tile codes (needs a GPU).

The split rule is pinned on the CPU against the oracle (tests/test_abi.py);
here the GPU path is checked for:
  * per-file round trip of uneven sets (empty files, files shorter than K,
    long files cut into several streams), with a stream budget and with the
    autotuned stream count, FP32 and BF16;
  * code length against the FP64 oracle on the same split (FP32, within
    0.5 % of the oracle's total, as for the single-input workload);
  * GEMM tile codes: every N tile (32 to 256) at every site, and the split-K
    weight-gradient GEMMs, give the oracle's logits and gradients within the
    BF16 tolerance, the tuner returns valid codes, and a container made with
    tuned tiles decodes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.compress import archive_split, archive_stream_len, oracle_compress  # noqa: E402
from oracle.model import Config, Model as OModel, softmax  # noqa: E402

pytestmark = pytest.mark.gpu

C0 = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=1)


def _uneven(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)).astype(np.int64)
    sizes[::7] = 0
    sizes[1] = 5  # shorter than K
    x = synth.multimedia_mix(int(sizes.sum()) + 3, seed)
    out, o = [], 0
    for s in sizes:
        out.append(x[o:o + s].copy())
        o += s
    return out


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
def test_file_set_roundtrip_with_budget(prec):
    files = _uneven(3, 23, 200, 40000)
    cfg = edpc.make_cfg(streams=64, precision=prec, **C0)
    bits = edpc.compress_many(files, cfg)
    assert edpc.archive_info(bits) == [f.size for f in files]
    back = edpc.decompress_many(bits)
    assert len(back) == len(files)
    for a, b in zip(files, back):
        assert np.array_equal(a, b)
    _, n, b = edpc.peek(bits)
    L = archive_stream_len([f.size for f in files], 64)
    assert n == sum(f.size for f in files) and b == archive_split([f.size for f in files], L)[0]


def test_empty_file_set_and_single_file():
    cfg = edpc.make_cfg(streams=8, **C0)
    bits = edpc.compress_many([], cfg)
    assert edpc.archive_info(bits) == [] and edpc.decompress_many(bits) == []
    one = [np.arange(3000, dtype=np.uint8)]
    back = edpc.decompress_many(edpc.compress_many(one, cfg))
    assert len(back) == 1 and np.array_equal(back[0], one[0])


def test_file_set_code_length_matches_oracle_fp32():
    files = _uneven(11, 14, 600, 9000)
    sizes = [f.size for f in files]
    data = np.concatenate(files)
    budget = 40
    L = archive_stream_len(sizes, budget)
    sp = archive_split(sizes, L)
    o = oracle_compress(data, Config(**C0), 0, split=sp)
    o_bytes = sum(len(s) for s in o["streams"])
    cfg = edpc.make_cfg(streams=budget, precision=edpc.EDPC_FP32, **C0)
    bits = edpc.compress_many(files, cfg)
    _, n, b = edpc.peek(bits)
    assert b == sp[0]
    hdr = 88 + 24 + 8 * len(files) + 4 * b + 4  # FP32: no tile codes
    g_bytes = len(bits) - hdr
    assert abs(g_bytes - o_bytes) <= 0.005 * o_bytes, (g_bytes, o_bytes)


def test_autotuned_file_set_roundtrip_bf16():
    files = _uneven(5, 30, 4096, 65536)
    cfg = edpc.make_cfg(streams=0, precision=edpc.EDPC_BF16, context=32, embed_dim=16, latent=256, hidden=256,
                        blocks=4)
    plan = edpc.archive_plan([f.size for f in files], cfg)
    mx = max(f.size for f in files)
    assert plan.stream_len == mx or plan.stream_len % 8192 == 0
    assert plan.streams == archive_split([f.size for f in files], plan.stream_len)[0]
    assert plan.est_seconds > 0 and plan.step_ms_t0 >= 0 and plan.step_ms_per_stream >= 0
    bits = edpc.compress_many(files, cfg)
    back = edpc.decompress_many(bits)
    for a, b in zip(files, back):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("code,k,b", [(1, 3, 300), (2, 3, 300), (4, 3, 300), (8, 3, 300), (4, 2, 300), (8, 2, 300),
                                      (8, 1, 300), (1, 2, 2100), (8, 2, 2100), (17, 3, 300), (24, 2, 300),
                                      (18, 2, 2100), (24, 2, 2100), (20, 1, 300), (17, 2, 2100)])
def test_every_tile_code_matches_oracle(code, k, b):
    """Every N tile (32-256; branch sections 32-128) at every site, one-tile
    and persistent (codes + 16) kernels, and, with 2100 streams, the split-K
    weight-gradient GEMMs (K = streams). Gradients are compared tensor by
    tensor, so a wrong small tensor (a bias, an LN parameter) cannot hide
    under the norm of a large weight."""
    dims = dict(context=8, embed_dim=16, latent=136, hidden=200, blocks=2, branches=k, lr=1e-3, seed=5)
    c = edpc.make_cfg(precision=edpc.EDPC_BF16, **dims)
    m = edpc.Model(c, b)
    m.set_tiles(np.full(512, code, np.uint8)[:200])
    om = OModel(Config(**dims), b)
    rng = np.random.default_rng(code)
    ctx = rng.integers(0, 256, size=(b, 8)).astype(np.uint8)
    z, _ = m.forward(ctx)
    zo, cache = om.forward(ctx.astype(np.int64))
    assert np.abs(z - zo).max() <= 3e-2 * np.abs(zo).max()
    tg = rng.integers(0, 256, size=b).astype(np.uint8)
    g, gu = m.backward(ctx, tg, np.ones(b, np.uint8))
    dz = softmax(zo)
    dz[np.arange(b), tg] -= 1
    dz /= b
    go, dUo = om.backward(cache, dz)
    gf = OModel.flat_grads(om.layout, go)
    off = 0
    for name, shape, _ in om.layout:
        n = int(np.prod(shape))
        ref = gf[off:off + n]
        if np.linalg.norm(ref) > 1e-12:
            assert np.linalg.norm(g[off:off + n] - ref) <= 6e-2 * np.linalg.norm(ref), name
        off += n
    gu = gu.reshape(dUo.shape)
    assert np.linalg.norm(gu - dUo) <= 6e-2 * np.linalg.norm(dUo)
    m.close()


@pytest.mark.parametrize("code", [48, 49, 56, 80, 81, 88, 32, 3])
def test_retired_and_invalid_tile_codes_are_refused(code):
    """Codes of kernels that are not built (cluster variants 48-88) and
    malformed codes are refused with EDPC_EARCH, and the model stays usable."""
    dims = dict(context=8, embed_dim=16, latent=16, hidden=64, blocks=2, branches=2, lr=1e-3, seed=9)
    m = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_BF16, **dims), 64)
    with pytest.raises(edpc.EdpcError) as ei:
        m.set_tiles(np.full(200, code, np.uint8))
    assert edpc._lib.STATUS[ei.value.code] == "EDPC_EARCH"
    m.set_tiles(np.full(200, 17, np.uint8))
    z, _ = m.forward(np.zeros((64, 8), np.uint8))
    assert np.isfinite(z).all()
    m.close()


@pytest.mark.parametrize("w", [1, 2, 4, 8])
def test_persistent_gemm_is_bit_identical(w):
    """The persistent kernel (every CTA walks several tiles and alternates two
    TMEM accumulators) gives bit-identical logits and gradients to the
    one-tile kernel (20000 streams: 157 M tiles, and the weight-gradient GEMMs
    are split)."""
    dims = dict(context=8, embed_dim=16, latent=16, hidden=64, blocks=2, branches=2, lr=1e-3, seed=9)
    b = 20000
    rng = np.random.default_rng(w)
    ctx = rng.integers(0, 256, size=(b, 8)).astype(np.uint8)
    tg = rng.integers(0, 256, size=b).astype(np.uint8)
    out = []
    for code in (w, w + 16):
        m = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_BF16, **dims), b)
        m.set_tiles(np.full(200, code, np.uint8))
        z, _ = m.forward(ctx)
        g, gu = m.backward(ctx, tg, np.ones(b, np.uint8))
        out.append((z, g, gu))
        m.close()
    for o in out[1:]:
        for a, c in zip(out[0], o):
            assert np.array_equal(a, c)


def test_tuned_tiles_single_input_roundtrip():
    m = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_BF16, **C0), 512)
    codes = m.tune_tiles()
    ok = {0} | {w + v for w in (1, 2, 4, 8) for v in (0, 16)}
    assert set(np.unique(codes)) <= ok and np.any(codes)
    m.close()
    x = synth.multimedia_mix(200000, 8)
    cfg = edpc.make_cfg(streams=64, precision=edpc.EDPC_BF16, flags=edpc.EDPC_FLAG_TUNE_TILES, **C0)
    bits = edpc.compress(x, cfg)
    assert np.array_equal(edpc.decompress(bits), x)
