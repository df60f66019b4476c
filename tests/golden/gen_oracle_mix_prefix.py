"""Writes oracle_mix_prefix.json: the FP64 oracle's code length on a prefix of
the 64 MiB multimedia mix, the reference for the per-precision bits/byte
delta (FP32, BF16, FP8 e4m3) of the GPU path.

Input: the 64 MiB mix (images / 16-bit PCM / order-3 text in equal thirds,
data seed 20250719) split into 512 contiguous streams; the first K + 192
bytes of each stream (192 model steps after the uniform prefix), i.e. an
input of 512 * 224 bytes whose balanced 512-stream split is exactly those
prefixes. Model: K = 32, D = 16, F' = 256, 4 MBRBs of hidden 256, 2
branches, Adam lr 1e-3, seed 1.

With --delayed the oracle runs the delayed-update schedule and writes
oracle_mix_prefix_delayed.json.

Every stored value comes from ``oracle/`` and ``synth/`` only. Run from the
repository root:  python tests/golden/gen_oracle_mix_prefix.py [--delayed]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle.compress import oracle_compress  # noqa: E402
from oracle.model import Config  # noqa: E402

DATA_SEED = 20250719
TOTAL = 64 << 20
STREAMS = 512
STEPS = 192
CFG = Config(context=32, embed_dim=16, latent=256, hidden=256, blocks=4, branches=2, lr=1e-3, seed=1)


def prefix_input():
    x = synth.multimedia_mix(TOTAL, DATA_SEED)
    q = x.size // STREAMS
    per = CFG.context + STEPS
    return np.ascontiguousarray(x[: q * STREAMS].reshape(STREAMS, q)[:, :per]).reshape(-1)


def main(delayed=False):
    xp = prefix_input()
    t0 = time.time()
    r = oracle_compress(xp, CFG, STREAMS, delayed=delayed)
    t1 = time.time()
    sizes = [len(s) for s in r["streams"]]
    out = dict(
        workload="64 MiB multimedia mix, first K + 192 bytes of each of 512 streams",
        data_seed=DATA_SEED, total=TOTAL, streams=STREAMS, steps=STEPS, n=int(xp.size),
        cfg=dict(context=CFG.context, embed_dim=CFG.embed_dim, latent=CFG.latent, hidden=CFG.hidden,
                 blocks=CFG.blocks, branches=CFG.branches, lr=CFG.lr, seed=CFG.seed),
        code_bytes=int(sum(sizes)),
        bits_per_byte=8.0 * sum(sizes) / xp.size,
        ideal_bits=float(np.sum(r["ideal_bits"])),
        input_sha_prefix=bytes(xp[:64]).hex(),
        oracle_seconds=round(t1 - t0, 1),
    )
    if delayed:
        out["schedule"] = "delayed update (gradient of step i applied after step i + 1)"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_mix_prefix_delayed.json" if delayed else "oracle_mix_prefix.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("bits_per_byte", "code_bytes", "oracle_seconds")}))


if __name__ == "__main__":
    main(delayed="--delayed" in sys.argv[1:])
