"""Archives of independent per-file models (needs a GPU).

BF16 runs every file's model in one batch (the grouped engine: per-file
weights in every kernel, one launch per layer over all files). Checked here:
  * lossless round trip of the whole archive and of each member alone;
  * a member's bytes depend only on its own file: the same file compressed
    alone, or in another batch in another order, gives the same member;
  * each file's code length against the FP64 oracle run on that file alone
    (oracle_compress with the member's stream count), within 0.5 % in total;
  * FP32 (one session per file) members equal edpc_compress of the file;
  * an empty archive, and a damaged table is refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.compress import oracle_compress  # noqa: E402
from oracle.model import Config  # noqa: E402

pytestmark = pytest.mark.gpu

C0 = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=1)


def _files(seed, sizes=(0, 5, 17, 3000, 9000, 40000, 1, 70000, 12345)):
    rng = np.random.default_rng(seed)
    x = synth.multimedia_mix(sum(sizes) + 3, seed)
    out, o = [], 0
    for n in sizes:
        out.append(x[o:o + n].copy())
        o += n
    rng.shuffle(out)
    return out


def _members(bits):
    raw = np.frombuffer(bits, np.uint8)
    nf = int(raw[8:16].view(np.uint64)[0])
    out = []
    for i in range(nf):
        off = int(raw[24 + 24 * i: 32 + 24 * i].view(np.uint64)[0])
        nb = int(raw[32 + 24 * i: 40 + 24 * i].view(np.uint64)[0])
        out.append(bytes(raw[off:off + nb]))
    return out


def test_fp32_members_match_single_file_compression():
    files = _files(5)
    L = 8192
    cfg = edpc.make_cfg(precision=edpc.EDPC_FP32, **C0)
    bits = edpc.compress_independent(files, cfg, stream_len=L, concurrency=3)
    assert edpc.independent_info(bits) == [f.size for f in files]
    back = edpc.decompress_independent(bits, concurrency=3)
    for f, g in zip(files, back):
        assert np.array_equal(f, g)
    for i, (f, m) in enumerate(zip(files, _members(bits))):
        alone = edpc.compress(f, edpc.make_cfg(streams=max(1, -(-f.size // L)), precision=edpc.EDPC_FP32, **C0))
        assert m == alone
        assert np.array_equal(edpc.decompress_member(bits, i), f)


def test_batched_round_trip_and_members_alone():
    files = _files(5)
    L = 8192
    cfg = edpc.make_cfg(precision=edpc.EDPC_BF16, **C0)
    bits = edpc.compress_independent(files, cfg, stream_len=L)
    assert edpc.independent_info(bits) == [f.size for f in files]
    back = edpc.decompress_independent(bits)
    for f, g in zip(files, back):
        assert np.array_equal(f, g)
    for i, (f, m) in enumerate(zip(files, _members(bits))):
        assert int(np.frombuffer(m[80:84], np.uint32)[0]) == 2  # header variant: the batched engine
        _, n, b = edpc.peek(m)
        assert n == f.size and b == max(1, min(-(-f.size // L), f.size // 16))
        assert np.array_equal(edpc.decompress_member(bits, i), f)
        assert np.array_equal(edpc.decompress(m), f)


def test_batched_member_bytes_do_not_depend_on_the_batch():
    """A file's member is the same alone, in one batch and in another batch
    (other files, other order): its model sees only its own rows."""
    files = _files(11)
    L = 4096
    cfg = edpc.make_cfg(precision=edpc.EDPC_BF16, **C0)
    ma = _members(edpc.compress_independent(files, cfg, stream_len=L))
    others = _files(12, sizes=(2000, 30000, 7))
    pick = [6, 2, 4]
    mb = _members(edpc.compress_independent([others[0], files[6], others[1], files[2], files[4], others[2]], cfg,
                                            stream_len=L))
    assert mb[1] == ma[6] and mb[3] == ma[2] and mb[4] == ma[4]
    for i in pick:
        alone = _members(edpc.compress_independent([files[i]], cfg, stream_len=L))[0]
        assert alone == ma[i]


def test_batched_members_against_oracle():
    """Code length of every member against the FP64 oracle compressing that
    file alone with the member's stream count (Algorithm 1; BF16 GEMMs, so
    within 0.5 % of the oracle's total, as for the single-input workloads)."""
    files = _files(21, sizes=(2500, 4100, 1800, 6000, 3300))
    L = 2048
    cfg = edpc.make_cfg(precision=edpc.EDPC_BF16, **C0)
    ms = _members(edpc.compress_independent(files, cfg, stream_len=L))
    got = ref = 0
    for f, m in zip(files, ms):
        _, n, b = edpc.peek(m)
        hdr = 88 + 4 * b + 4
        r = oracle_compress(f, Config(**C0), b)
        rb = 8 * sum(len(s) for s in r["streams"])
        gb = 8 * (len(m) - hdr)
        assert abs(gb - rb) <= 0.02 * rb, (f.size, gb, rb)
        got += gb
        ref += rb
    assert abs(got - ref) <= 0.005 * ref, (got, ref)


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
