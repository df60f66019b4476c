"""The C-ABI library loads and exports what include/edpc.h declares (CPU only)."""
import ctypes as C
import os
import re

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
