"""GB300-native EDPC: an online-learning lossless byte compressor.

Python binding of the C ABI in include/edpc.h (libedpc.so, built in-tree by
``_build.build()``). Every function here only marshals arguments; the
method itself runs in the library's CUDA kernels. The library must be
built: importing this package does not build it, and a missing library
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import (EDPC_BF16, EDPC_FP8E4M3, EDPC_FLAG_DELAYED_UPDATE, EDPC_FLAG_NO_GRAPH, EDPC_FLAG_OVERLAP_FDM, EDPC_FLAG_NO_PIPELINE, EDPC_FLAG_TUNE_TILES, EDPC_FP32, Cfg,
                   EdpcError, SplitPlan, Stats, check, load)

__all__ = [
    "Cfg", "EdpcError", "EDPC_FP32", "EDPC_BF16", "EDPC_FP8E4M3", "EDPC_FLAG_NO_PIPELINE", "EDPC_FLAG_NO_GRAPH",
    "EDPC_FLAG_TUNE_TILES", "EDPC_FLAG_OVERLAP_FDM", "EDPC_FLAG_DELAYED_UPDATE", "make_cfg", "compress", "decompress", "peek", "param_count", "Encoder", "Decoder",
    "Model", "archive_plan", "compress_many", "decompress_many", "archive_info", "SplitPlan",
    "cdf_quantize", "range_encode", "range_encode_noalloc", "NOALLOC_MAX_STREAMS", "load",
]


def make_cfg(streams=4, context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2,
             lr=1e-3, precision=EDPC_FP32, seed=1, flags=0) -> Cfg:
    c = Cfg()
    load().edpc_default_cfg(C.byref(c))
    c.streams, c.context, c.embed_dim = streams, context, embed_dim
    c.latent, c.hidden, c.blocks, c.branches = latent, hidden, blocks, branches
    c.lr, c.precision, c.seed, c.flags = lr, precision, seed, flags
    return c


def _buf(x) -> np.ndarray:
    return np.ascontiguousarray(np.frombuffer(x, dtype=np.uint8) if isinstance(x, (bytes, bytearray)) else x,
                                dtype=np.uint8)


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a.size else C.c_void_p(0)


def param_count(cfg: Cfg) -> int:
    return int(load().edpc_param_count(C.byref(cfg)))


def compress(data, cfg: Cfg) -> bytes:
    lib = load()
    a = _buf(data)
    out = C.c_void_p()
    n = C.c_size_t()
    check(lib.edpc_compress(_ptr(a), a.size, C.byref(cfg), C.byref(out), C.byref(n)), "edpc_compress")
    try:
        return C.string_at(out, n.value)
    finally:
        lib.edpc_free(out)


def decompress(bits) -> np.ndarray:
    lib = load()
    a = _buf(bits)
    out = C.c_void_p()
    n = C.c_size_t()
    check(lib.edpc_decompress(_ptr(a), a.size, C.byref(out), C.byref(n)), "edpc_decompress")
    try:
        return np.frombuffer(C.string_at(out, n.value), dtype=np.uint8).copy()
    finally:
        lib.edpc_free(out)


def peek(bits):
    lib = load()
    a = _buf(bits)
    c = Cfg()
    n = C.c_uint64()
    b = C.c_uint32()
    check(lib.edpc_peek(_ptr(a), a.size, C.byref(c), C.byref(n), C.byref(b)), "edpc_peek")
    return c, n.value, b.value


def _files(files):
    """(keep-alive arrays, pointer array, size array) of a list of byte buffers."""
    keep = [_buf(f) for f in files]
    n = len(keep)
    ptrs = (C.c_void_p * max(1, n))(*[a.ctypes.data if a.size else None for a in keep])
    lens = (C.c_size_t * max(1, n))(*[a.size for a in keep])
    return keep, ptrs, lens


def archive_plan(sizes, cfg: Cfg) -> SplitPlan:
    """The stream split edpc_compress_many would use for files of ``sizes``
    (cfg.streams = budget, or 0 to autotune on the GPU)."""
    n = len(sizes)
    lens = (C.c_size_t * max(1, n))(*[int(x) for x in sizes])
    plan = SplitPlan()
    check(load().edpc_archive_plan(lens, n, C.byref(cfg), C.byref(plan)), "edpc_archive_plan")
    return plan


def compress_many(files, cfg: Cfg) -> bytes:
    """One container for a list of files (bytes or uint8 arrays)."""
    lib = load()
    keep, ptrs, lens = _files(files)
    out = C.c_void_p()
    n = C.c_size_t()
    check(lib.edpc_compress_many(ptrs, lens, len(keep), C.byref(cfg), C.byref(out), C.byref(n)), "edpc_compress_many")
    try:
        return C.string_at(out, n.value)
    finally:
        lib.edpc_free(out)


def archive_info(bits) -> list[int]:
    """File sizes stored in a container."""
    lib = load()
    a = _buf(bits)
    nf = C.c_uint64()
    check(lib.edpc_archive_info(_ptr(a), a.size, C.byref(nf), C.c_void_p(0)), "edpc_archive_info")
    sizes = np.zeros(max(1, nf.value), np.uint64)
    check(lib.edpc_archive_info(_ptr(a), a.size, C.byref(nf), _ptr(sizes)), "edpc_archive_info")
    return [int(x) for x in sizes[:nf.value]]


def decompress_many(bits) -> list[np.ndarray]:
    """The files of a container, as uint8 arrays."""
    lib = load()
    a = _buf(bits)
    outs = C.c_void_p()
    lens = C.c_void_p()
    nf = C.c_size_t()
    check(lib.edpc_decompress_many(_ptr(a), a.size, C.byref(outs), C.byref(lens), C.byref(nf)),
          "edpc_decompress_many")
    try:
        ptrs = C.cast(outs, C.POINTER(C.c_void_p))
        ls = C.cast(lens, C.POINTER(C.c_size_t))
        return [np.frombuffer(C.string_at(ptrs[i], ls[i]), np.uint8).copy() if ls[i] else np.zeros(0, np.uint8)
                for i in range(nf.value)]
    finally:
        lib.edpc_free(outs)
        lib.edpc_free(lens)


def ksg_mi(z_dev: int, y_dev: int, n: int, dz: int, dy: int, k: int, cz_dev: int, cy_dev: int,
           stream: int = 0) -> float:
    """Kraskov estimate of I(Z; Y) in nats from FP32 device arrays Z (n x dz) and Y (n x dy);
    the per-sample counts c_z, c_y go to the device arrays cz_dev, cy_dev (n uint32 each)."""
    mi = C.c_double()
    check(load().edpc_ksg_mi(C.c_void_p(z_dev), C.c_void_p(y_dev), n, dz, dy, k, C.c_void_p(cz_dev),
                             C.c_void_p(cy_dev), C.byref(mi), C.c_void_p(stream)), "edpc_ksg_mi")
    return mi.value


def selftest_wait_timeout(stream: int = 0) -> None:
    """Runs the bounded-wait self-test; raises EdpcError with code 6
    (EDPC_ETIMEOUT) when the wait expired as designed."""
    check(load().edpc_selftest_wait_timeout(C.c_void_p(stream)), "edpc_selftest_wait_timeout")


def compress_independent(files, cfg: Cfg, stream_len: int = 65536, concurrency: int = 8) -> bytes:
    """Archive of independent per-file models: file f gets its own model over
    max(1, ceil(n_f / stream_len)) streams. BF16: all files' models run as one
    batch (members are header variant 2 containers); otherwise one session per
    file, ``concurrency`` at a time."""
    lib = load()
    keep, ptrs, lens = _files(files)
    out = C.c_void_p()
    n = C.c_size_t()
    check(lib.edpc_compress_independent(ptrs, lens, len(keep), C.byref(cfg), int(stream_len), int(concurrency),
                                        C.byref(out), C.byref(n)), "edpc_compress_independent")
    try:
        return C.string_at(out, n.value)
    finally:
        lib.edpc_free(out)


def independent_info(bits) -> list[int]:
    """File sizes of an archive of independent models."""
    lib = load()
    a = _buf(bits)
    nf = C.c_uint64()
    check(lib.edpc_independent_info(_ptr(a), a.size, C.byref(nf), C.c_void_p(0)), "edpc_independent_info")
    sizes = np.zeros(max(1, nf.value), np.uint64)
    check(lib.edpc_independent_info(_ptr(a), a.size, C.byref(nf), _ptr(sizes)), "edpc_independent_info")
    return [int(x) for x in sizes[:nf.value]]


def decompress_member(bits, index: int) -> np.ndarray:
    """File ``index`` of an archive of independent models, decoded alone."""
    lib = load()
    a = _buf(bits)
    out = C.c_void_p()
    n = C.c_size_t()
    check(lib.edpc_decompress_member(_ptr(a), a.size, int(index), C.byref(out), C.byref(n)), "edpc_decompress_member")
    try:
        return np.frombuffer(C.string_at(out, n.value), np.uint8).copy() if n.value else np.zeros(0, np.uint8)
    finally:
        lib.edpc_free(out)


def decompress_independent(bits, concurrency: int = 8) -> list[np.ndarray]:
    """Every file of an archive of independent models."""
    lib = load()
    a = _buf(bits)
    outs = C.c_void_p()
    lens = C.c_void_p()
    nf = C.c_size_t()
    check(lib.edpc_decompress_independent(_ptr(a), a.size, int(concurrency), C.byref(outs), C.byref(lens),
                                          C.byref(nf)), "edpc_decompress_independent")
    try:
        ptrs = C.cast(outs, C.POINTER(C.c_void_p))
        ls = C.cast(lens, C.POINTER(C.c_size_t))
        return [np.frombuffer(C.string_at(ptrs[i], ls[i]), np.uint8).copy() if ls[i] else np.zeros(0, np.uint8)
                for i in range(nf.value)]
    finally:
        lib.edpc_free(outs)
        lib.edpc_free(lens)


class _Session:
    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def run(self, max_steps: int, sync: bool = True) -> int:
        done = C.c_uint64()
        check(load().edpc_session_run(self._h, max_steps, int(sync), C.byref(done)), "edpc_session_run")
        return done.value

    def remaining(self) -> int:
        n = C.c_uint64()
        check(load().edpc_session_remaining(self._h, C.byref(n)), "edpc_session_remaining")
        return n.value

    def profile(self, on: bool = True) -> None:
        check(load().edpc_session_profile(self._h, int(on)), "edpc_session_profile")

    def stats(self) -> Stats:
        s = Stats()
        check(load().edpc_session_stats(self._h, C.byref(s)), "edpc_session_stats")
        return s

    def close(self) -> None:
        if self._h:
            load().edpc_session_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Encoder(_Session):
    """Encoder session. ``data``: host bytes / uint8 array, or ``device_ptr`` + ``length``;
    or ``files`` (host buffers) / ``device_files`` (list of (device pointer, size)) for a file set."""

    def __init__(self, cfg: Cfg, data=None, device_ptr: int | None = None, length: int | None = None,
                 stream: int | None = None, files=None, device_files=None):
        lib = load()
        h = C.c_void_p()
        if files is not None or device_files is not None:
            if device_files is not None:
                keep = None
                n = len(device_files)
                ptrs = (C.c_void_p * max(1, n))(*[int(p) for p, _ in device_files])
                lens = (C.c_size_t * max(1, n))(*[int(x) for _, x in device_files])
                on_dev = 1
            else:
                keep, ptrs, lens = _files(files)
                n, on_dev = len(keep), 0
            check(lib.edpc_encoder_open_many(C.byref(cfg), ptrs, lens, n, on_dev, C.c_void_p(stream or 0),
                                             C.byref(h)), "edpc_encoder_open_many")
            super().__init__(h, (keep, ptrs, lens))
            return
        if device_ptr is not None:
            keep = None
            check(lib.edpc_encoder_open(C.byref(cfg), C.c_void_p(device_ptr), int(length), 1,
                                        C.c_void_p(stream or 0), C.byref(h)), "edpc_encoder_open")
        else:
            keep = _buf(data)
            check(lib.edpc_encoder_open(C.byref(cfg), _ptr(keep), keep.size, 0, C.c_void_p(stream or 0),
                                        C.byref(h)), "edpc_encoder_open")
        super().__init__(h, keep)

    def finish(self) -> bytes:
        lib = load()
        out = C.c_void_p()
        n = C.c_size_t()
        check(lib.edpc_encoder_finish(self._h, C.byref(out), C.byref(n)), "edpc_encoder_finish")
        try:
            return C.string_at(out, n.value)
        finally:
            lib.edpc_free(out)


class Decoder(_Session):
    def __init__(self, bits, out_device_ptr: int | None = None, stream: int | None = None):
        lib = load()
        keep = _buf(bits)
        h = C.c_void_p()
        check(lib.edpc_decoder_open(_ptr(keep), keep.size, C.c_void_p(out_device_ptr or 0), C.c_void_p(stream or 0),
                                    C.byref(h)), "edpc_decoder_open")
        self.n = peek(keep)[1]
        super().__init__(h, keep)

    def finish(self, to_host: bool = True):
        out = np.empty(self.n, dtype=np.uint8) if to_host else None
        check(load().edpc_decoder_finish(self._h, _ptr(out) if to_host else C.c_void_p(0)), "edpc_decoder_finish")
        return out


class Model:
    """One model step at a given state (gradient and parity checks)."""

    def __init__(self, cfg: Cfg, streams: int):
        self.cfg = cfg
        self.b = streams
        self.np = param_count(cfg)
        fp = cfg.latent if cfg.latent else cfg.context * cfg.embed_dim  # latent 0: no LTE, F x F FDMs
        self.fdm = streams * fp * fp
        h = C.c_void_p()
        check(load().edpc_model_create(C.byref(cfg), streams, C.byref(h)), "edpc_model_create")
        self._h = h

    def close(self):
        if self._h:
            load().edpc_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_state(self, which=("P", "U", "M", "V", "Um", "Uv")):
        """Host copies of the state arrays named in ``which`` (the others are
        None): P shared parameters, U per-stream FDMs, M/V and Um/Uv their Adam
        moments; ``t`` is the Adam step count."""
        out = {}
        for k in ("P", "U", "M", "V", "Um", "Uv"):
            n = self.np if k in ("P", "M", "V") else self.fdm
            out[k] = np.empty(n, np.float32) if k in which else None
        t = C.c_uint32()
        ptrs = [C.c_void_p(0) if out[k] is None else _ptr(out[k]) for k in ("P", "U", "M", "V", "Um", "Uv")]
        check(load().edpc_model_get_state(self._h, *ptrs, C.byref(t)), "edpc_model_get_state")
        out["t"] = t.value
        return out

    def set_state(self, P=None, U=None, M=None, V=None, Um=None, Uv=None, t=0):
        arrs = [None if x is None else np.ascontiguousarray(x, dtype=np.float32) for x in (P, U, M, V, Um, Uv)]
        ptrs = [C.c_void_p(0) if a is None else _ptr(a) for a in arrs]
        check(load().edpc_model_set_state(self._h, *ptrs, t), "edpc_model_set_state")

    def forward(self, ctx):
        ctx = np.ascontiguousarray(ctx, dtype=np.uint8)
        z = np.empty((self.b, 256), np.float32)
        p = np.empty((self.b, 256), np.float32)
        check(load().edpc_model_forward(self._h, _ptr(ctx), _ptr(z), _ptr(p)), "edpc_model_forward")
        return z, p

    def backward(self, ctx, targets, active):
        ctx = np.ascontiguousarray(ctx, dtype=np.uint8)
        tg = np.ascontiguousarray(targets, dtype=np.uint8)
        ac = np.ascontiguousarray(active, dtype=np.uint8)
        g = np.empty(self.np, np.float32)
        gu = np.empty(self.fdm, np.float32)
        check(load().edpc_model_backward(self._h, _ptr(ctx), _ptr(tg), _ptr(ac), _ptr(g), _ptr(gu)),
              "edpc_model_backward")
        return g, gu

    def set_tiles(self, codes) -> None:
        """GEMM tile codes per site: 0 heuristic, w = 1/2/4/8 for an N tile of 32*w (capped
        per site), w + 16 for the persistent kernel; BF16 and FP8 only."""
        a = np.ascontiguousarray(codes, dtype=np.uint8)
        check(load().edpc_model_set_tiles(self._h, _ptr(a), a.size), "edpc_model_set_tiles")

    def tune_tiles(self) -> np.ndarray:
        """Times every GEMM site's N tiles and keeps the fastest; returns the codes."""
        n = C.c_uint32()
        codes = np.zeros(512, np.uint8)
        check(load().edpc_model_tune_tiles(self._h, _ptr(codes), codes.size, C.byref(n)), "edpc_model_tune_tiles")
        return codes[:n.value].copy()

    def time_gemms(self, reps: int = 8):
        """Per tcgen05 GEMM site: (mean ms per launch, FLOP per launch, compulsory bytes per
        launch); unused sites are 0."""
        n = C.c_uint32()
        ms = np.zeros(512, np.float64)
        fl = np.zeros(512, np.float64)
        by = np.zeros(512, np.float64)
        check(load().edpc_model_time_gemms(self._h, reps, _ptr(ms), _ptr(fl), _ptr(by), ms.size, C.byref(n)),
              "edpc_model_time_gemms")
        k = n.value
        return ms[:k].copy(), fl[:k].copy(), by[:k].copy()

    def block_io(self, block: int):
        """(S, S + X^(k)) of MBRB ``block`` from the last forward: (streams, F) FP32 arrays."""
        F = self.cfg.context * self.cfg.embed_dim
        a = np.empty((self.b, F), np.float32)
        o = np.empty((self.b, F), np.float32)
        check(load().edpc_model_block_io(self._h, int(block), _ptr(a), _ptr(o)), "edpc_model_block_io")
        return a, o

    def train_step(self, ctx, targets, active):
        ctx = np.ascontiguousarray(ctx, dtype=np.uint8)
        tg = np.ascontiguousarray(targets, dtype=np.uint8)
        ac = np.ascontiguousarray(active, dtype=np.uint8)
        check(load().edpc_model_train_step(self._h, _ptr(ctx), _ptr(tg), _ptr(ac)), "edpc_model_train_step")


def cdf_quantize(p_dev: int, rows: int, freq_dev: int, cum_dev: int, stream: int = 0) -> None:
    """Device pointers: p (rows x 256 f32) -> freq (rows x 256 u32), cum (rows x 257 u32)."""
    check(load().edpc_cdf_quantize(C.c_void_p(p_dev), rows, C.c_void_p(freq_dev), C.c_void_p(cum_dev),
                                   C.c_void_p(stream)), "edpc_cdf_quantize")


def range_encode(sym_dev: int, nsym: int, streams: int, out_dev: int, cap: int, out_len_dev: int,
                 stream: int = 0) -> None:
    """Device pointers: sym (nsym x streams u32) -> out (streams x cap bytes), out_len (streams u32)."""
    check(load().edpc_range_encode(C.c_void_p(sym_dev), nsym, streams, C.c_void_p(out_dev), cap,
                                   C.c_void_p(out_len_dev), C.c_void_p(stream)), "edpc_range_encode")


NOALLOC_MAX_STREAMS = 4096


def range_encode_noalloc(sym_dev: int, nsym: int, streams: int, out_dev: int, cap: int, out_len_dev: int,
                         stream: int = 0) -> None:
    """As range_encode, with the library's fixed scratch instead of per-call
    device allocations (streams <= NOALLOC_MAX_STREAMS)."""
    check(load().edpc_range_encode_noalloc(C.c_void_p(sym_dev), nsym, streams, C.c_void_p(out_dev), cap,
                                           C.c_void_p(out_len_dev), C.c_void_p(stream)),
          "edpc_range_encode_noalloc")
