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
import types

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


# ----------------------------------------------------------------- chain-sharded ensemble
def _shard_worker(rank, world, port, M, n_iter, out):
    """Rank `rank` of a chain-sharded LAPS ensemble, composed on the oracle's
    maps: it advances chains [m0, m1) of the M-chain ensemble (the Philox
    counters carry the global chain index), reduces them to its totals of the
    per-coordinate sums of y, y^2, g, y g and the per-chain sums of the energy
    error (the 4d + 3 numbers a rank contributes), gathers every rank's totals,
    adds them in rank order and runs the unadjusted finalise of Alg. 1 (Sec. 3.1
    steps 2-5, Eq. "L", Sec. 4's window) on the sum; it reports its trace of
    eps, L and max delta."""
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2601_16696_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.set_threads(1)
        pr = W.banana(d=10, M=M, n_steps=100)
        ot = oracle.OracleTarget(pr.kind, pr.d, banana_sb=pr.banana_sb)
        start = oracle.OracleLAPS(ot, pr.x0, seed=3, n_total_steps=pr.n_steps)
        cfg = oracle.default_config()
        y0, u0, g0, lp0 = start.state()
        m0, m1 = rank * M // world, (rank + 1) * M // world
        Y, U, G, LP = (a[m0:m1].copy() for a in (y0, u0, g0, lp0))
        d = pr.d
        eps, L = start.trace[0]["eps"], start.trace[0]["L"]
        T = start.window_T
        window, rows = [], []
        for it in range(n_iter):
            deltas = np.empty(m1 - m0)
            for k, m in enumerate(range(m0, m1)):
                z = oracle.normals(3, m, 1, it, oracle.TAG_O1, 0, d)[0] / np.sqrt(d)
                oracle.O(0.5 * eps, L, z, U[k])
                deltas[k], LP[k] = oracle.Phi(ot, oracle.LF, eps, Y[k], U[k], G[k], LP[k])
                z = oracle.normals(3, m, 1, it, oracle.TAG_O2, 0, d)[0] / np.sqrt(d)
                oracle.O(0.5 * eps, L, z, U[k])
            mine = np.concatenate([Y.sum(0), (Y * Y).sum(0), G.sum(0), (Y * G).sum(0),
                                   [deltas.sum(), (deltas * deltas).sum(), float(m1 - m0)]])
            parts = [torch.zeros(mine.size, dtype=torch.float64) for _ in range(world)]
            dist.all_gather(parts, torch.from_numpy(mine))
            tot = parts[0].numpy().copy()
            for p in parts[1:]:
                tot = tot + p.numpy()  # rank order
            Sy, Syy, Sg, Syg = (tot[q * d:(q + 1) * d] for q in range(4))
            SD, SDD, n = tot[4 * d:]
            var = Syy / M - (Sy / M) ** 2
            V = -(Syg / M - (Sy / M) * (Sg / M))
            D = float(np.mean((1.0 - V) ** 2))
            eevpd = (SDD / n - (SD / n) ** 2) / d
            eps = eps * (oracle.F(cfg.C * D) / eevpd) ** (1.0 / 6.0)
            L = cfg.alpha * np.sqrt(var.sum())
            window.append(Syy / M)
            md = float("nan")
            if len(window) >= T:
                h = np.array(window[-T:])
                md = max(oracle.rel_fluct(h[:, i]) for i in range(d))
            rows.append((eps, L, md))
        out.put((rank, rows))
    finally:
        dist.destroy_process_group()


def test_chain_sharded_ensemble_composes_like_one_rank():
    """Two gloo ranks each advance half of a 63-chain banana ensemble and
    exchange only their totals; every iteration's step size, L and window
    statistic equal the single-rank oracle's to round-off, on both ranks."""
    import numpy as np
    import oracle
    from paper_2601_16696_gb300 import workloads as W
    oracle.lib()
    M, n_iter = 63, 30
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_worker, args=(k, 2, port, M, n_iter, q)) for k in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    pr = W.banana(d=10, M=M, n_steps=100)
    ref = oracle.OracleLAPS(oracle.OracleTarget(pr.kind, pr.d, banana_sb=pr.banana_sb), pr.x0,
                            seed=3, n_total_steps=pr.n_steps)
    ref.iterate(n_iter)
    np.testing.assert_array_equal(np.array(res[0]), np.array(res[1]))  # the same on every rank
    for it, (eps, L, md) in enumerate(res[0]):
        r = ref.trace[it + 1]
        assert eps == pytest.approx(r["eps"], rel=1e-9), it
        assert L == pytest.approx(r["L"], rel=1e-9), it
        if np.isnan(r["max_delta"]):
            assert np.isnan(md)
        else:
            assert md == pytest.approx(r["max_delta"], rel=1e-9), it
    assert sum(not np.isnan(x[2]) for x in res[0]) == n_iter - ref.window_T + 1


# ---- the batch split over ranks by problems (laps_batch_partition, host only)

def _partition_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2601_16696_gb300 import laps, workloads
    laps.lib()  # host-only call: no GPU
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # batch64's shapes (no initial positions drawn): 64 small problems, then d = 10^4, M = 16384
        probs = [types.SimpleNamespace(d=d, M=M) for d, _, M in workloads.batch64_shapes()]
        probs.append(types.SimpleNamespace(d=10000, M=16384))
        mine = laps.partition_problems(probs, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_partition_two_ranks_agree_and_cover_the_batch():
    """Each of two gloo ranks computes its own share of the 65-problem batch;
    the shares are disjoint, cover every problem once, and every rank sees
    the same split."""
    from paper_2601_16696_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_partition_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, g0), (_, g1) = res
    assert g0 == g1
    shares = g0
    assert sorted(shares[0] + shares[1]) == list(range(65))
    assert not set(shares[0]) & set(shares[1])
    # the d = 10^4 problem (index 64, 70% of the coordinates) alone on one rank
    big = [r for r in range(2) if 64 in shares[r]][0]
    assert shares[big] == [64]
