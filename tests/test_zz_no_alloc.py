"""The allocation-free range encoder against the allocating one (needs a GPU).

edpc_range_encode_noalloc serves callers that may not allocate device memory
per call; it keeps its scratch in a fixed array inside the library. It must
produce exactly the bytes edpc_range_encode produces, call after call, even
though every call reuses (and must reset) the same scratch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
from oracle.coder import quantize_cdf  # noqa: E402

pytestmark = pytest.mark.gpu


def _symbols(rng, nsym, streams):
    sym = np.empty((nsym, streams), dtype=np.uint32)
    for t in range(nsym):
        p = rng.dirichlet(np.full(256, 0.05), size=streams).astype(np.float32)
        f, cum = quantize_cdf(p)
        x = np.where(rng.random(streams) < 0.5, np.argmax(f, axis=1), rng.integers(0, 256, size=streams))
        x[rng.random(streams) < 0.1] = 255
        c = cum[np.arange(streams), x]
        fr = f[np.arange(streams), x]
        sym[t] = (c | ((fr - 1) << 16)).astype(np.uint32)
        sym[t, rng.random(streams) < 0.03] = 0xFFFFFFFF
    return sym


def _encode(fn, sym, streams, cap):
    nsym = sym.shape[0]
    sd = torch.from_numpy(sym.view(np.int32)).cuda()
    out = torch.full((streams * cap,), 0xAB, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(streams, dtype=torch.int32, device="cuda")
    fn(sd.data_ptr(), nsym, streams, out.data_ptr(), cap, ln.data_ptr())
    return out.cpu().numpy(), ln.cpu().numpy()


def test_noalloc_matches_allocating_encoder_on_consecutive_calls():
    rng = np.random.default_rng(2024)
    # Two calls in a row; the second uses fewer streams, so stale coder states
    # left in the shared scratch by the first call must not leak into it.
    for streams, nsym in ((700, 400), (97, 900)):
        sym = _symbols(rng, nsym, streams)
        cap = 2 * nsym + 64
        ref_out, ref_len = _encode(edpc.range_encode, sym, streams, cap)
        out, ln = _encode(edpc.range_encode_noalloc, sym, streams, cap)
        assert np.array_equal(ln, ref_len)
        for s in range(streams):
            assert bytes(out[s * cap:s * cap + ln[s]]) == bytes(ref_out[s * cap:s * cap + ref_len[s]]), s


def test_noalloc_rejects_more_streams_than_its_scratch_holds():
    n = edpc.NOALLOC_MAX_STREAMS + 1
    sym = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(edpc.EdpcError) as e:
        edpc.range_encode_noalloc(sym.data_ptr(), 1, n, out.data_ptr(), 16, ln.data_ptr())
    assert e.value.code == 1
    assert "EDPC_NOALLOC_MAX_STREAMS" in str(e.value)


def _encode_status(fn, sym, streams, cap):
    """Like _encode, but returns the error code (0 if none) with the outputs."""
    nsym = sym.shape[0]
    sd = torch.from_numpy(sym.view(np.int32)).cuda()
    out = torch.full((streams * cap,), 0xAB, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(streams, dtype=torch.int32, device="cuda")
    code = 0
    try:
        fn(sd.data_ptr(), nsym, streams, out.data_ptr(), cap, ln.data_ptr())
    except edpc.EdpcError as e:
        code = e.code
    return code, out.cpu().numpy(), ln.cpu().numpy().view(np.uint32)


def test_noalloc_overflow_matches_allocating_encoder():
    """Streams that need more than cap bytes: both entry points report
    EDPC_EINVAL, clamp those streams' lengths to cap, and write identical bytes
    for every stream (the overflowing ones truncated at cap)."""
    streams, nsym, cap = 301, 300, 300
    sym = np.empty((nsym, streams), dtype=np.uint32)
    sym[:, 0::2] = 0 | (65534 << 16)  # cum 0, f 65535: almost free
    sym[:, 1::2] = 100                # cum 100, f 1: 16 bits per symbol, 600 bytes > cap
    sym[::7, 2::3] = 0xFFFFFFFF       # some skipped steps
    ref = _encode_status(edpc.range_encode, sym, streams, cap)
    got = _encode_status(edpc.range_encode_noalloc, sym, streams, cap)
    assert ref[0] == got[0] == 1  # EDPC_EINVAL
    assert np.array_equal(got[2], ref[2])
    over = sym[:, :] == 100
    odd_full = np.array([over[:, s].sum() * 2 > cap for s in range(streams)])
    assert np.all(ref[2][odd_full] == cap) and np.all(ref[2][~odd_full] < cap)
    for s in range(streams):
        n = int(ref[2][s])
        assert bytes(got[1][s * cap:s * cap + n]) == bytes(ref[1][s * cap:s * cap + n]), s
    # a clean call right after the failed one matches again (the shared flag was reset)
    sym_ok = np.full((40, 5), 0 | (65534 << 16), dtype=np.uint32)
    a = _encode_status(edpc.range_encode, sym_ok, 5, 64)
    b = _encode_status(edpc.range_encode_noalloc, sym_ok, 5, 64)
    assert a[0] == b[0] == 0 and np.array_equal(a[2], b[2])
