"""ctypes binding of libedpc.so (argument marshalling only).

Every call goes to the C ABI declared in include/edpc.h; nothing here
computes any part of the method. A missing library raises at load time:
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libedpc.so")

EDPC_ABI_VERSION = 1
EDPC_FORMAT_VERSION = 1  # container format (include/edpc.h)
EDPC_FP32 = 0
EDPC_BF16 = 1
EDPC_FP8E4M3 = 2
EDPC_FLAG_NO_PIPELINE = 1
EDPC_FLAG_NO_GRAPH = 2
EDPC_FLAG_TUNE_TILES = 4
EDPC_FLAG_OVERLAP_FDM = 8
EDPC_FLAG_DELAYED_UPDATE = 16

STATUS = {0: "EDPC_OK", 1: "EDPC_EINVAL", 2: "EDPC_ENOMEM", 3: "EDPC_ECORRUPT", 4: "EDPC_EVERSION",
          5: "EDPC_ECUDA", 6: "EDPC_ETIMEOUT", 7: "EDPC_EARCH"}


class Cfg(C.Structure):
    _fields_ = [
        ("version", C.c_uint32),
        ("streams", C.c_uint32),
        ("context", C.c_uint32),
        ("embed_dim", C.c_uint32),
        ("latent", C.c_uint32),
        ("hidden", C.c_uint32),
        ("blocks", C.c_uint32),
        ("branches", C.c_uint32),
        ("lr", C.c_float),
        ("precision", C.c_uint32),
        ("seed", C.c_uint64),
        ("flags", C.c_uint32),
        ("reserved", C.c_uint32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps_run", C.c_uint64),
        ("steps_total", C.c_uint64),
        ("streams", C.c_uint32),
        ("launches_per_step", C.c_uint32),
        ("fdm_fwd_ms", C.c_double),
        ("fdm_bwd_ms", C.c_double),
        ("fdm_samples", C.c_uint64),
        ("coded_bytes", C.c_uint64),
        ("fdm_adam_ms", C.c_double),
    ]


class SplitPlan(C.Structure):
    _fields_ = [
        ("stream_len", C.c_uint64),
        ("streams", C.c_uint32),
        ("reserved", C.c_uint32),
        ("est_seconds", C.c_double),
        ("step_ms_t0", C.c_double),
        ("step_ms_per_stream", C.c_double),
    ]


P = C.c_void_p
U8P = C.POINTER(C.c_uint8)
FP = C.POINTER(C.c_float)

# name -> (restype, argtypes); the order follows include/edpc.h
PROTOS = {
    "edpc_default_cfg": (None, [C.POINTER(Cfg)]),
    "edpc_strerror": (C.c_char_p, [C.c_int]),
    "edpc_last_error": (C.c_char_p, []),
    "edpc_param_count": (C.c_uint64, [C.POINTER(Cfg)]),
    "edpc_free": (None, [P]),
    "edpc_compress": (C.c_int, [P, C.c_size_t, C.POINTER(Cfg), C.POINTER(P), C.POINTER(C.c_size_t)]),
    "edpc_decompress": (C.c_int, [P, C.c_size_t, C.POINTER(P), C.POINTER(C.c_size_t)]),
    "edpc_peek": (C.c_int, [P, C.c_size_t, C.POINTER(Cfg), C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
    "edpc_encoder_open": (C.c_int, [C.POINTER(Cfg), P, C.c_size_t, C.c_int, P, C.POINTER(P)]),
    "edpc_session_run": (C.c_int, [P, C.c_uint64, C.c_int, C.POINTER(C.c_uint64)]),
    "edpc_session_remaining": (C.c_int, [P, C.POINTER(C.c_uint64)]),
    "edpc_encoder_finish": (C.c_int, [P, C.POINTER(P), C.POINTER(C.c_size_t)]),
    "edpc_decoder_open": (C.c_int, [P, C.c_size_t, P, P, C.POINTER(P)]),
    "edpc_decoder_finish": (C.c_int, [P, P]),
    "edpc_session_stats": (C.c_int, [P, C.POINTER(Stats)]),
    "edpc_session_profile": (C.c_int, [P, C.c_int]),
    "edpc_session_close": (None, [P]),
    "edpc_archive_plan": (C.c_int, [P, C.c_size_t, C.POINTER(Cfg), C.POINTER(SplitPlan)]),
    "edpc_compress_many": (C.c_int, [P, P, C.c_size_t, C.POINTER(Cfg), C.POINTER(P), C.POINTER(C.c_size_t)]),
    "edpc_encoder_open_many": (C.c_int, [C.POINTER(Cfg), P, P, C.c_size_t, C.c_int, P, C.POINTER(P)]),
    "edpc_archive_info": (C.c_int, [P, C.c_size_t, C.POINTER(C.c_uint64), P]),
    "edpc_decompress_many": (C.c_int, [P, C.c_size_t, C.POINTER(P), C.POINTER(P), C.POINTER(C.c_size_t)]),
    "edpc_cdf_quantize": (C.c_int, [P, C.c_uint32, P, P, P]),
    "edpc_range_encode": (C.c_int, [P, C.c_uint32, C.c_uint32, P, C.c_uint32, P, P]),
    "edpc_range_encode_noalloc": (C.c_int, [P, C.c_uint32, C.c_uint32, P, C.c_uint32, P, P]),
    "edpc_model_create": (C.c_int, [C.POINTER(Cfg), C.c_uint32, C.POINTER(P)]),
    "edpc_model_destroy": (None, [P]),
    "edpc_model_get_state": (C.c_int, [P, P, P, P, P, P, P, C.POINTER(C.c_uint32)]),
    "edpc_model_set_state": (C.c_int, [P, P, P, P, P, P, P, C.c_uint32]),
    "edpc_model_forward": (C.c_int, [P, P, P, P]),
    "edpc_model_backward": (C.c_int, [P, P, P, P, P, P]),
    "edpc_model_train_step": (C.c_int, [P, P, P, P]),
    "edpc_model_set_tiles": (C.c_int, [P, P, C.c_uint32]),
    "edpc_model_tune_tiles": (C.c_int, [P, P, C.c_uint32, C.POINTER(C.c_uint32)]),
    "edpc_model_time_gemms": (C.c_int, [P, C.c_uint32, P, P, P, C.c_uint32, C.POINTER(C.c_uint32)]),
    "edpc_model_block_io": (C.c_int, [P, C.c_uint32, P, P]),
    "edpc_ksg_mi": (C.c_int, [P, P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P, P, C.POINTER(C.c_double), P]),
    "edpc_selftest_wait_timeout": (C.c_int, [P]),
    "edpc_compress_independent": (C.c_int, [P, P, C.c_size_t, P, C.c_uint64, C.c_uint32, C.POINTER(C.c_void_p),
                                            C.POINTER(C.c_size_t)]),
    "edpc_independent_info": (C.c_int, [P, C.c_size_t, C.POINTER(C.c_uint64), P]),
    "edpc_decompress_member": (C.c_int, [P, C.c_size_t, C.c_uint64, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]),
    "edpc_decompress_independent": (C.c_int, [P, C.c_size_t, C.c_uint32, C.POINTER(C.c_void_p),
                                              C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]),
}

_LIB = None


def load(path: str | None = None):
    """Loads libedpc.so and sets every prototype. Raises if it is missing."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_2507_18969_gb300._build`")
    lib = C.CDLL(p)
    for name, (res, args) in PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


class EdpcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({detail})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != 0:
        lib = load()
        raise EdpcError(code, where, (lib.edpc_last_error() or b"").decode())
