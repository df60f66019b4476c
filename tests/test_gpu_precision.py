"""Bits/byte of each GEMM precision against the FP64 oracle (needs a GPU).

Input: the first K + 192 bytes of each of the 512 streams of the 64 MiB
multimedia mix, with the 64 MiB workload's model (K = 32, F' = 256, 4 MBRBs of
256); the oracle's code length is stored in tests/golden/oracle_mix_prefix.json
(written by gen_oracle_mix_prefix.py from oracle/ only). The GPU and the
oracle follow different FP trajectories, so the comparison is statistical:
FP32 and BF16 within 0.5 % of the oracle's code length, FP8 e4m3 within 3 %.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_mix_prefix.json")


def _prefix(g):
    x = synth.multimedia_mix(g["total"], g["data_seed"])
    q = x.size // g["streams"]
    per = g["cfg"]["context"] + g["steps"]
    return np.ascontiguousarray(x[: q * g["streams"]].reshape(g["streams"], q)[:, :per]).reshape(-1)


@pytest.fixture(scope="module")
def golden():
    g = json.load(open(GOLDEN))
    xp = _prefix(g)
    assert bytes(xp[:64]).hex() == g["input_sha_prefix"] and xp.size == g["n"]
    return g, xp


@pytest.mark.parametrize("prec,tol", [(edpc.EDPC_FP32, 0.005), (edpc.EDPC_BF16, 0.005), (edpc.EDPC_FP8E4M3, 0.03)],
                         ids=["fp32", "bf16", "fp8"])
def test_code_length_per_precision(golden, prec, tol):
    g, xp = golden
    c = edpc.make_cfg(streams=g["streams"], precision=prec, **g["cfg"])
    bits = edpc.compress(xp, c)
    assert np.array_equal(edpc.decompress(bits), xp)
    _, n, b = edpc.peek(bits)
    code = len(bits) - (88 + 4 * b + 4)
    delta = code / g["code_bytes"] - 1
    print("precision %d: %.4f bits/byte (oracle %.4f), delta %+.3f %%" %
          (prec, 8 * code / n, g["bits_per_byte"], 100 * delta))
    assert abs(delta) <= tol
