"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks (no GPU).

The path does not shard within one input, so N GPUs run N replicas; the only
collectives are the barrier and the aggregation of the timing: the value is
all ranks' bytes over the slowest rank's time. Checked here with two gloo
processes, and, for the reference arm, that under a 2-rank launch only rank 0
prints its line while every rank exits 0.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(world, backend="gloo")
    try:
        d.barrier()
        # rank r moved (r + 1) MB in (1 + r) s
        value, t = bench.aggregate((rank + 1) * 1e6, 1.0 + rank, d)
        d.barrier()
        q.put((rank, value, t))
    finally:
        d.close()


def test_replica_aggregation_over_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for _, value, t in res:
        assert t == 2.0                      # the slowest rank's time
        assert abs(value - 1.5) < 1e-12      # (1 + 2) MB / 2 s


def test_reference_arm_prints_once_under_two_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
