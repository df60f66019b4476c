"""Writes oracle_c0.json: the FP64 oracle's result on the small FP32 workload.

Workload: 64 KiB from a seeded order-2 Markov source over 256 symbols (each
transition row Dirichlet(0.1)); 4 streams; K = 16 context bytes, D = 16,
LTE latent 128, 2 MBRB blocks of hidden 128; Adam lr 1e-3; T = 2^16;
32-bit range coder.

With --delayed the oracle runs the delayed-update schedule and writes
oracle_c0_delayed.json.

Every stored value comes from ``oracle/`` and ``synth/`` only. Run from the
repository root:  python tests/golden/gen_oracle_c0.py [--delayed]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle.compress import oracle_compress, oracle_decompress  # noqa: E402
from oracle.model import Config  # noqa: E402

DATA_SEED = 20250718
MODEL_SEED = 1
N = 65536
STREAMS = 4
CFG = Config(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2,
             lr=1e-3, seed=MODEL_SEED)


def main(delayed=False):
    table = synth.markov_table(2, 0.1, DATA_SEED)
    x = synth.markov_bytes(N, 2, 0.1, DATA_SEED, table=table)
    H = synth.markov_entropy_rate(table, 2)
    t0 = time.time()
    r = oracle_compress(x, CFG, STREAMS, delayed=delayed)
    t1 = time.time()
    y = oracle_decompress(r["streams"], N, CFG, STREAMS, delayed=delayed)
    assert np.array_equal(x, y), "oracle round trip failed"
    sizes = [len(s) for s in r["streams"]]
    out = dict(
        workload="order-2 Markov 64 KiB, Dirichlet(0.1) rows",
        data_seed=DATA_SEED, n=N, streams=STREAMS,
        cfg=dict(context=CFG.context, embed_dim=CFG.embed_dim, latent=CFG.latent,
                 hidden=CFG.hidden, blocks=CFG.blocks, branches=CFG.branches,
                 lr=CFG.lr, seed=CFG.seed),
        stream_bytes=sizes,
        bits_per_byte=8.0 * sum(sizes) / N,
        ideal_bits=[float(v) for v in r["ideal_bits"]],
        trunc_bits=[float(v) for v in r["trunc_bits"]],
        entropy_rate_bits=H,
        input_sha_prefix=bytes(x[:64]).hex(),
        oracle_seconds=round(t1 - t0, 1),
    )
    if delayed:
        out["schedule"] = "delayed update (gradient of step i applied after step i + 1)"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c0_delayed.json" if delayed else "oracle_c0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("bits_per_byte", "entropy_rate_bits", "oracle_seconds")}))


if __name__ == "__main__":
    main(delayed="--delayed" in sys.argv[1:])
