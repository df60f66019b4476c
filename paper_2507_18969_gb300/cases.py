"""Named timing cases of the library (for step timing and kernel profiles).

  python -m paper_2507_18969_gb300.cases steps CASE [CHUNKS [delayed]]
      An encoder session on CASE's model and stream count over random bytes
      already on the device (the kernels' work does not depend on the byte
      values): one warm-up chunk of 64 model steps, then CHUNKS timed chunks;
      prints milliseconds per model step (CUDA events). "delayed" selects the
      delayed-update schedule (EDPC_FLAG_DELAYED_UPDATE).
  python -m paper_2507_18969_gb300.cases gemm CASE CODE
      Every tcgen05 GEMM site of CASE's model with every tile code set to CODE,
      each launched alone (Model.time_gemms): ms, GFLOP and TFLOP/s per site.

  python -m paper_2507_18969_gb300.cases ifr [STEPS]
      Sec. 3.1.1's Information Flow Refinement on the 64 MiB mix: models with
      1, 2 and 3 MBRB branches (c1's dims) each take STEPS online steps on
      the first bytes of its 512 streams; then, on the next contexts, every
      block's skip input S and fused output S + X^(k) give I^(k) (Kraskov,
      3 neighbours, on the GPU), and IFR_{k1->k2} = I^(k1) / I^(k2).

Cases: c1 (K=32, F'=256, 4 MBRBs of 256; 512 streams, the 64 MiB workload's
model), c1_32k (the same model, 32768 streams), c4 (K=64, F'=512, 6 MBRBs of
512; 4096 streams, the 1 GiB workload's model) and c4_gemm (c4's F, H and
stream count with F'=16 and 2 blocks: c4's GEMM shapes in well under 1 GB).
"""
from __future__ import annotations

import json
import sys

import numpy as np

CASES = {
    "c1": dict(b=512, K=32, Fp=256, H=256, n=4),
    "c1_32k": dict(b=32768, K=32, Fp=256, H=256, n=4),
    "c4": dict(b=4096, K=64, Fp=512, H=512, n=6),
    "c4_gemm": dict(b=4096, K=64, Fp=16, H=512, n=2),
}


def _cfg(c, edpc, **kw):
    return edpc.make_cfg(streams=c["b"], context=c["K"], embed_dim=16, latent=c["Fp"], hidden=c["H"], blocks=c["n"],
                         branches=2, lr=1e-3, seed=1, precision=edpc.EDPC_BF16, **kw)


def steps(name: str, chunks: int = 2, delayed: bool = False) -> dict:
    import torch
    import paper_2507_18969_gb300 as edpc
    from paper_2507_18969_gb300 import Encoder
    c = CASES[name]
    n = c["b"] * (c["K"] + (chunks + 2) * 64 + 8)
    x = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    flags = edpc.EDPC_FLAG_DELAYED_UPDATE if delayed else 0
    enc = Encoder(_cfg(c, edpc, flags=flags), device_ptr=x.data_ptr(), length=n, stream=st.cuda_stream)
    enc.run(64)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    done = enc.run(64 * chunks)
    e1.record(st)
    torch.cuda.synchronize()
    enc.close()
    ms = e0.elapsed_time(e1) / done
    return dict(case=name, streams=c["b"], delayed=delayed, ms_per_model_step=ms, mbs=c["b"] / ms / 1e3)


def gemm(name: str, code: int) -> list[dict]:
    import paper_2507_18969_gb300 as edpc
    c = CASES[name]
    m = edpc.Model(_cfg(c, edpc), c["b"])
    m.set_tiles(np.full(200, code, np.uint8))
    ms, fl, _ = m.time_gemms(1)
    m.close()
    return [dict(site=int(i), gflop=fl[i] / 1e9, us=ms[i] * 1e3, tflops=fl[i] / ms[i] / 1e9) for i in np.nonzero(fl)[0]]


def ifr(steps: int = 256) -> dict:
    import torch
    import paper_2507_18969_gb300 as edpc
    import synth
    c = CASES["c1"]
    b, K = c["b"], c["K"]
    x = synth.multimedia_mix(64 << 20, 20250719)
    q = x.size // b
    xs = x[: q * b].reshape(b, q)
    res = {"steps": steps, "streams": b, "neighbours": 3, "mi_nats": {}, "ifr": {}}
    for k in (1, 2, 3):
        cfg = edpc.make_cfg(streams=b, context=K, embed_dim=16, latent=c["Fp"], hidden=c["H"], blocks=c["n"],
                            branches=k, lr=1e-3, seed=1, precision=edpc.EDPC_BF16)
        m = edpc.Model(cfg, b)
        ones = np.ones(b, np.uint8)
        for i in range(K, K + steps):
            m.train_step(xs[:, i - K:i], xs[:, i], ones)
        m.forward(np.ascontiguousarray(xs[:, steps + 1:steps + 1 + K]))
        mis = []
        for blk in range(c["n"]):
            s, so = m.block_io(blk)
            zs = torch.from_numpy(s).cuda()
            ys = torch.from_numpy(so).cuda()
            cz = torch.zeros(b, dtype=torch.int32, device="cuda")
            cy = torch.zeros(b, dtype=torch.int32, device="cuda")
            mis.append(edpc.ksg_mi(zs.data_ptr(), ys.data_ptr(), b, s.shape[1], so.shape[1], 3, cz.data_ptr(),
                                   cy.data_ptr()))
        m.close()
        res["mi_nats"][str(k)] = mis
    for k1, k2 in ((1, 2), (1, 3), (2, 3)):
        res["ifr"][f"{k1}->{k2}"] = [a / bb for a, bb in zip(res["mi_nats"][str(k1)], res["mi_nats"][str(k2)])]
    return res


def main(argv) -> int:
    if argv and argv[0] == "ifr":
        print(json.dumps(ifr(int(argv[1]) if len(argv) > 1 else 256)), flush=True)
        return 0
    if len(argv) < 2 or argv[0] not in ("steps", "gemm") or argv[1] not in CASES:
        print(__doc__)
        return 2
    if argv[0] == "steps":
        print(json.dumps(steps(argv[1], int(argv[2]) if len(argv) > 2 else 2,
                               len(argv) > 3 and argv[3] == "delayed")), flush=True)
    else:
        for r in gemm(argv[1], int(argv[2]) if len(argv) > 2 else 0):
            print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
