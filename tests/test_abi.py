"""The C-ABI library loads and exports what include/edpc.h declares (CPU only)."""
import ctypes as C
import os
import re
import struct
import zlib

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "edpc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(edpc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_18969_gb300 import _build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        _build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    from paper_2507_18969_gb300 import _lib
    assert sorted(_lib.PROTOS) == declared_functions()


def test_cfg_layout_and_defaults(lib):
    from paper_2507_18969_gb300._lib import Cfg
    assert C.sizeof(Cfg) == 56
    c = Cfg()
    lib.edpc_default_cfg(C.byref(c))
    assert (c.version, c.streams, c.context, c.embed_dim, c.latent, c.hidden, c.blocks, c.branches) == \
        (1, 4, 16, 16, 128, 128, 2, 2)
    assert abs(c.lr - 1e-3) < 1e-9 and c.seed == 1


@pytest.mark.parametrize("blocks,branches,latent", [(2, 2, 128), (4, 2, 256), (6, 3, 512), (1, 1, 64)])
def test_param_count_matches_canonical_layout(lib, blocks, branches, latent):
    from oracle.model import Config, param_layout
    import paper_2507_18969_gb300 as pkg
    cfg = pkg.make_cfg(context=32, embed_dim=16, latent=latent, hidden=256, blocks=blocks, branches=branches)
    o = Config(context=32, embed_dim=16, latent=latent, hidden=256, blocks=blocks, branches=branches)
    assert pkg.param_count(cfg) == sum(int(np.prod(s)) for _, s, _ in param_layout(o))


def test_invalid_cfg_is_rejected(lib):
    import paper_2507_18969_gb300 as pkg
    bad = pkg.make_cfg(embed_dim=12)
    assert pkg.param_count(bad) == 0
    out = C.c_void_p()
    n = C.c_size_t()
    r = lib.edpc_compress(None, 0, C.byref(bad), C.byref(out), C.byref(n))
    assert r == 1  # EDPC_EINVAL
    assert b"embed_dim" in lib.edpc_last_error()


def test_strerror_names_every_code(lib):
    for code in range(8):
        assert lib.edpc_strerror(code)
    assert lib.edpc_strerror(99) == b"unknown status"


def test_peek_rejects_garbage(lib):
    import paper_2507_18969_gb300 as pkg
    with pytest.raises(pkg.EdpcError) as e:
        pkg.peek(b"not a container at all" * 10)
    assert e.value.code == 3


def test_file_set_plan_matches_the_oracle_split(lib):
    """The library's stream budget rule (host code) against the oracle's, on
    random file sets: the same stream length and stream count."""
    import paper_2507_18969_gb300 as pkg
    from oracle.compress import archive_split, archive_stream_len
    rng = np.random.default_rng(9)
    for trial in range(40):
        nf = int(rng.integers(1, 30))
        sizes = np.exp(rng.uniform(0, np.log(1 << 22), size=nf)).astype(np.int64)
        sizes[rng.random(nf) < 0.1] = 0
        budget = int(rng.integers(1, 2000))
        plan = pkg.archive_plan(list(sizes), pkg.make_cfg(streams=budget))
        L = archive_stream_len(list(sizes), budget)
        b, _, _ = archive_split(list(sizes), L)
        assert (plan.stream_len, plan.streams) == (L, b), (trial, budget)
        assert plan.est_seconds == 0


def test_file_set_plan_rejects_too_many_streams(lib):
    import paper_2507_18969_gb300 as pkg
    with pytest.raises(pkg.EdpcError):
        pkg.archive_plan([1] * 70000, pkg.make_cfg(streams=65535))
    with pytest.raises(pkg.EdpcError):
        pkg.archive_plan([10, 20], pkg.make_cfg(streams=70000))


def _fmt():
    from paper_2507_18969_gb300 import _lib
    return _lib.EDPC_FORMAT_VERSION


def _indep(nfiles, members, L=65536, crc_ok=True, magic=0x49504445, version=None):
    """An archive of independent models built by hand (table + members)."""
    import struct
    import zlib
    version = _fmt() if version is None else version
    hl = 24 + 24 * nfiles + 4
    head = struct.pack("<IIQQ", magic, version, nfiles, L)
    o = hl
    for m, size in members:
        head += struct.pack("<QQQ", o, len(m), size)
        o += len(m)
    crc = zlib.crc32(head) & 0xFFFFFFFF
    head += struct.pack("<I", crc if crc_ok else crc ^ 1)
    return head + b"".join(m for m, _ in members)


def test_independent_archive_table_is_checked(lib):
    """The archive reader (host only) accepts a well-formed table and refuses a
    bad magic, a bad CRC, a truncated table and members out of range."""
    import paper_2507_18969_gb300 as edpc
    assert edpc.independent_info(_indep(0, [])) == []
    with pytest.raises(edpc.EdpcError) as ev:  # a container of a format version this library lacks
        edpc.independent_info(_indep(0, [], version=_fmt() + 1))
    assert ev.value.code == 4  # EDPC_EVERSION
    assert edpc.independent_info(_indep(2, [(b"ab", 7), (b"", 0)])) == [7, 0]
    for bad in (_indep(0, [], magic=0x12345678), _indep(1, [(b"xy", 3)], crc_ok=False),
                _indep(2, [(b"ab", 7), (b"", 0)])[:40]):
        with pytest.raises(edpc.EdpcError) as e:
            edpc.independent_info(bad)
        assert e.value.code == 3  # EDPC_ECORRUPT
    # a member that runs past the end of the archive
    import struct
    import zlib
    head = struct.pack("<IIQQ", 0x49504445, _fmt(), 1, 4096) + struct.pack("<QQQ", 52, 1000, 5)
    head += struct.pack("<I", zlib.crc32(head) & 0xFFFFFFFF)
    with pytest.raises(edpc.EdpcError):
        edpc.independent_info(head + b"short")
    with pytest.raises(edpc.EdpcError) as e:
        edpc.decompress_member(_indep(1, [(b"xy", 3)]), 1)
    assert e.value.code == 1  # EDPC_EINVAL: index out of range


def _header(sched, precision=1, n=100):
    # variant-0 container of one empty stream: fixed header, one length word, CRC
    b = 1
    hl = 88 + 4 * b + 4
    h = struct.pack("<IIIIIIIIIIf", 0x43504445, _fmt(), hl, precision, 16, 16, 128, 128, 2, 2, 1e-3)
    h += struct.pack("<IQQIIQII", sched, 1, n, 1, b, 0, 0, 0)
    h += struct.pack("<I", 0)
    assert len(h) == hl - 4
    return h + struct.pack("<I", zlib.crc32(h) & 0xFFFFFFFF)


def test_header_update_schedule_word(lib):
    import paper_2507_18969_gb300 as pkg
    c, n, b = pkg.peek(_header(0))
    assert (n, b) == (100, 1) and not (c.flags & pkg.EDPC_FLAG_DELAYED_UPDATE)
    c, _, _ = pkg.peek(_header(1))
    assert c.flags & pkg.EDPC_FLAG_DELAYED_UPDATE
    with pytest.raises(pkg.EdpcError) as e:
        pkg.peek(_header(2))
    assert e.value.code == 7  # EDPC_EARCH: a schedule this library version lacks
    with pytest.raises(pkg.EdpcError) as e:
        pkg.peek(_header(1, precision=2))  # the delayed update with FP8 is not a valid configuration
    assert e.value.code == 3


def test_delayed_update_flag_combinations_are_checked(lib):
    import paper_2507_18969_gb300 as pkg
    D = pkg.EDPC_FLAG_DELAYED_UPDATE
    assert pkg.param_count(pkg.make_cfg(precision=pkg.EDPC_BF16, flags=D)) > 0
    assert pkg.param_count(pkg.make_cfg(precision=pkg.EDPC_FP32, flags=D)) > 0
    for bad in (pkg.make_cfg(precision=pkg.EDPC_FP8E4M3, flags=D),
                pkg.make_cfg(precision=pkg.EDPC_BF16, flags=D | pkg.EDPC_FLAG_OVERLAP_FDM)):
        assert pkg.param_count(bad) == 0
        out = C.c_void_p()
        n = C.c_size_t()
        assert lib.edpc_compress(None, 0, C.byref(bad), C.byref(out), C.byref(n)) == 1
        assert b"delayed" in lib.edpc_last_error()


def test_host_allocation_failure_is_enomem(lib):
    # A valid header whose original length (2^62 bytes) no host allocation can
    # hold: edpc_decompress fails on its output buffer before any device work.
    bits = _header(0, n=1 << 62)
    out = C.c_void_p()
    n = C.c_size_t()
    buf = (C.c_uint8 * len(bits)).from_buffer_copy(bits)
    assert lib.edpc_decompress(buf, len(bits), C.byref(out), C.byref(n)) == 2  # EDPC_ENOMEM
    assert b"output buffer" in lib.edpc_last_error()
    assert not out.value and n.value == 0
