"""Archives of independent per-file models (needs a GPU).

Every file gets its own model, so each member must be byte-identical to
compressing that file alone with edpc_compress (same cfg, streams =
max(1, ceil(n_f / stream_len))), decode alone, and the whole archive must
round-trip whatever the number of concurrent sessions; a damaged table is
refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

C0 = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=1)


def _files(seed):
    rng = np.random.default_rng(seed)
    sizes = [0, 5, 17, 3000, 9000, 40000, 1, 70000, 12345]
    x = synth.multimedia_mix(sum(sizes) + 3, seed)
    out, o = [], 0
    for n in sizes:
        out.append(x[o:o + n].copy())
        o += n
    rng.shuffle(out)
    return out


@pytest.mark.parametrize("prec,conc", [(edpc.EDPC_FP32, 3), (edpc.EDPC_BF16, 4), (edpc.EDPC_BF16, 1)],
                         ids=["fp32-3", "bf16-4", "bf16-1"])
def test_members_match_single_file_compression(prec, conc):
    files = _files(5)
    L = 8192
    cfg = edpc.make_cfg(precision=prec, **C0)
    bits = edpc.compress_independent(files, cfg, stream_len=L, concurrency=conc)
    assert edpc.independent_info(bits) == [f.size for f in files]
    back = edpc.decompress_independent(bits, concurrency=conc)
    for f, g in zip(files, back):
        assert np.array_equal(f, g)
    # each member is what the file alone compresses to, and decodes alone
    raw = np.frombuffer(bits, np.uint8)
    n = len(files)
    for i, f in enumerate(files):
        off = int(raw[24 + 24 * i: 32 + 24 * i].view(np.uint64)[0])
        nb = int(raw[32 + 24 * i: 40 + 24 * i].view(np.uint64)[0])
        alone = edpc.compress(f, edpc.make_cfg(streams=max(1, -(-f.size // L)), precision=prec, **C0))
        assert bytes(raw[off:off + nb]) == alone
        assert np.array_equal(edpc.decompress_member(bits, i), f)
    assert 24 + 24 * n + 4 <= len(bits)


def test_empty_archive_and_damage():
    cfg = edpc.make_cfg(precision=edpc.EDPC_BF16, **C0)
    bits = edpc.compress_independent([], cfg)
    assert edpc.independent_info(bits) == []
    assert edpc.decompress_independent(bits) == []
    bits = bytearray(edpc.compress_independent(_files(6)[:3], cfg, stream_len=4096))
    bits[30] ^= 1  # inside the file table: CRC mismatch
    with pytest.raises(edpc.EdpcError):
        edpc.independent_info(bytes(bits))
    with pytest.raises(edpc.EdpcError):
        edpc.decompress_member(bytes(bits), 0)
