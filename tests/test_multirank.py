"""The N > 1 path of bench.py on CPU, with the gloo backend and two ranks.

The sampler's path does not shard within one problem without an exchange of
the ensemble sums every iteration, so `bench.py --gpus N` runs N replicas:
every rank times its own run, the job's time is the slowest rank's (a MAX
reduction), the value counts every rank's work, and rank 0 alone prints.  The
reference arm (the oracle, host cores only) runs on rank 0 alone and the other
ranks exit at once.  No GPU is used here.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench._rank_env()
        # each rank reports a different time; every rank gets the largest
        got = bench._max_over_ranks(10.0 + 5.0 * rank)
        out.put((rank, r, w, lr, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r[0], r[1], r[2], r[3]) for r in res] == [(0, 0, 2, 0), (1, 1, 2, 1)]
    assert all(r[4] == 15.0 for r in res)


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5) == 3.5


def test_reference_arm_two_ranks_prints_once():
    """torchrun with two ranks: one JSON line, from rank 0, exit status 0."""
    import oracle
    oracle.lib()  # the oracle's library is built here, before the ranks start
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
