"""GPU parity of the batched path (many diagonal-Gaussian problems of uneven
d and M in one persistent launch) against per-problem FP64 oracle runs.

Problem k of a batch draws from the Philox stream of the batch seed with
problem id k, so the oracle run with pid = k consumes the same noise.  The
batched kernel sums the ensemble in another order than the oracle (and than
the single-problem kernel), so comparisons use the parity bars: per-chain
positions within 1e-5 relative over the first steps at a fixed step size, and
the final b^2 within 10% (tail means, as for single problems).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_16696_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16696_gb300 import build, laps
    build.build()
    laps.lib()
    return laps


def _probs(spec, n_steps, x0_scale=1.0, var=(0.1, 10.0)):
    return [W.gauss_diag(d=d, M=M, n_steps=n_steps, x0_scale=x0_scale, var_lo=var[0],
                         var_hi=var[1], seed=100 + k) for k, (d, M) in enumerate(spec)]


def _ora(ora, pr, seed, pid, **cfg):
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec)
    return ora.OracleLAPS(ot, pr.x0, seed=seed, pid=pid, truth=(pr.Ex2, pr.Varx2),
                          n_total_steps=pr.n_steps, **cfg)


def _rel(xg, xr):
    return (np.linalg.norm(xg - xr, axis=1) / np.linalg.norm(xr, axis=1)).max()


SPEC = [(7, 33), (64, 100), (300, 257), (1500, 64), (3000, 40)]


def test_batch_first_steps_fixed_step(L, ora):
    probs = _probs(SPEC, 50)
    b = L.Batch(probs, n_total_steps=50, fixed_eps=0.05)
    b.init(seed=11)
    refs = [_ora(ora, pr, 11, k, fixed_eps=0.05) for k, pr in enumerate(probs)]
    for k, pr in enumerate(probs):
        np.testing.assert_array_equal(b.sample(k).double().cpu().numpy(), pr.x0)
    for step in range(5):
        b.step(1)
        for k, r in enumerate(refs):
            r.iterate(1)
            rel = _rel(b.sample(k).double().cpu().numpy(), r.x())
            assert rel <= 1e-5, (k, step + 1, rel)
    for k, r in enumerate(refs):
        for a, c in zip(b.trace(k)[:6], r.trace[:6]):
            assert a["L"] == pytest.approx(c["L"], rel=1e-5)


@pytest.mark.parametrize("cpl", [8, 12, 16, 20])
@pytest.mark.parametrize("widen", [0, 1])
def test_batch_every_shape(L, ora, cpl, widen):
    spec = [(d, M) for d, M in SPEC if d <= 512 * cpl // (2 ** widen)]
    probs = _probs(spec, 40)
    b = L.Batch(probs, n_total_steps=40, fixed_eps=0.05)
    b.set_shape(cpl, widen, 32)
    assert b.shape()["coords_per_lane"] == cpl
    b.init(seed=3)
    b.step(3)
    for k, pr in enumerate(probs):
        r = _ora(ora, pr, 3, k, fixed_eps=0.05)
        r.iterate(3)
        assert _rel(b.sample(k).double().cpu().numpy(), r.x()) <= 1e-5, (k, cpl, widen)


def _tail(trace, key, frac=0.5):
    rows = [r for r in trace[1:] if r["phase"] == trace[-1]["phase"]]
    n = max(1, int(len(rows) * frac))
    return float(np.mean([r[key] for r in rows[-n:]]))


def test_batch_whole_run_matches_oracle(L, ora):
    spec = [(20, 1024), (150, 512), (700, 256), (2500, 256)]
    probs = _probs(spec, 600, x0_scale=2.0)
    cfg = dict(force_switch_at=200)
    b = L.Batch(probs, n_total_steps=600, **cfg)
    for k, pr in enumerate(probs):
        b.set_truth(k, pr.Ex2, pr.Varx2)
    b.init(seed=0)
    b.run(iters_per_launch=50)
    for k, pr in enumerate(probs):
        st = b.stats(k)
        r = _ora(ora, pr, 0, k, **cfg)
        r.run()
        assert st["t"] == r.t and st["phase"] == r.phase == 1, k
        assert st["t_switch"] == r.t_switch == 200 and st["integrator"] == r.integrator, k
        bg, bo = _tail(b.trace(k), "b2_avg"), _tail(r.trace, "b2_avg")
        assert abs(bg - bo) <= 0.10 * bo, (k, bg, bo)


def test_batch_graph_replay_equals_steps(L):
    probs = _probs([(33, 300), (400, 200), (1200, 100)], 300)
    outs = []
    for mode in ("graph", "steps"):
        b = L.Batch(probs, n_total_steps=300, force_switch_at=100)
        b.init(seed=5)
        if mode == "graph":
            b.run(iters_per_launch=16)
        else:
            for _ in range(400):
                b.step(1)
        outs.append([b.sample(k).cpu().numpy() for k in range(len(probs))]
                    + [[r["eps"] for r in b.trace(k)] for k in range(len(probs))])
    for a, c in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(c))


def test_batch_d10000_in_the_tuned_shape(L, ora):
    """The batch's d = 10^4 problem in the shape the autotuner picks for the
    whole batch (20 coordinates per lane, so one chain spans a 16-warp group),
    beside a small problem: first steps at a fixed step size within 1e-5."""
    probs = [W.gauss_diag(d=10000, M=256, n_steps=50, x0_scale=1.0, var_lo=1e-2, var_hi=1e2, seed=999),
             W.gauss_diag(d=37, M=1000, n_steps=50, x0_scale=1.0, seed=5)]
    b = L.Batch(probs, n_total_steps=50, fixed_eps=0.02)
    b.set_shape(20, 0, 128)
    assert b.shape()["coords_per_lane"] == 20 and b.shape()["threads"] == 512
    b.init(seed=13)
    refs = [_ora(ora, pr, 13, k, fixed_eps=0.02) for k, pr in enumerate(probs)]
    for step in range(5):
        b.step(1)
        for k, r in enumerate(refs):
            r.iterate(1)
            rel = _rel(b.sample(k).double().cpu().numpy(), r.x())
            assert rel <= 1e-5, (k, step + 1, rel)


def test_batch_autotuner_keeps_parity(L, ora):
    probs = _probs(SPEC, 40)
    b = L.Batch(probs, n_total_steps=40, fixed_eps=0.05)
    b.init(seed=7)
    b.tune()
    sh = b.shape()
    assert sh["tuned"] == 1 and sh["coords_per_lane"] in (8, 12, 16, 20)
    b.step(4)
    for k, pr in enumerate(probs):
        r = _ora(ora, pr, 7, k, fixed_eps=0.05)
        r.iterate(4)
        assert _rel(b.sample(k).double().cpu().numpy(), r.x()) <= 1e-5, k


def test_batch_switch_at_the_end_samples_in_x(L, ora):
    # a switch that leaves no room for a proposal ends the run with the
    # preconditioner set and y still in the target's coordinates
    probs = _probs([(40, 200), (90, 64)], 110)
    b = L.Batch(probs, n_total_steps=110, force_switch_at=100)
    b.init(seed=2)
    b.run(iters_per_launch=32)
    for k, pr in enumerate(probs):
        st = b.stats(k)
        r = _ora(ora, pr, 2, k, force_switch_at=100)
        r.run()
        assert st["phase"] == r.phase == 1 and st["done"] == 1 and st["t"] == r.t
        xg = b.sample(k).double().cpu().numpy()
        assert np.isfinite(xg).all()
        # same ensemble scale as the oracle's final ensemble (x, not y)
        assert np.allclose(np.sqrt((xg ** 2).mean()), np.sqrt((r.x() ** 2).mean()), rtol=0.05)


def test_batch_barrier_timeout_reported(L):
    probs = _probs([(16, 64), (32, 64)], 20)
    b = L.Batch(probs, n_total_steps=20, barrier_timeout_ns=20_000_000, barrier_extra_arrivals=1)
    with pytest.raises(L.LapsError) as e:
        b.init(seed=1)
        b.stats(0)
    assert e.value.status == 4


def test_batch_rejects_bad_problems(L):
    pr = W.gauss_diag(d=20000, M=4, n_steps=5)
    with pytest.raises(L.LapsError) as e:
        L.Batch([pr], n_total_steps=5)
    assert e.value.status == 1


def test_batch_extreme_shapes(L, ora):
    """The largest dimension the batch serves (d = 10240) beside the smallest
    (d = 2), with 2 and 3 chains: first steps within 1e-5 of the oracle."""
    probs = [W.gauss_diag(d=10240, M=3, n_steps=20, x0_scale=1.0, var_lo=0.1, var_hi=10.0, seed=21),
             W.gauss_diag(d=2, M=2, n_steps=20, x0_scale=1.0, var_lo=0.5, var_hi=2.0, seed=22)]
    b = L.Batch(probs, n_total_steps=20, fixed_eps=0.05)
    b.init(seed=17)
    b.step(3)
    for k, pr in enumerate(probs):
        r = _ora(ora, pr, 17, k, fixed_eps=0.05)
        r.iterate(3)
        assert _rel(b.sample(k).double().cpu().numpy(), r.x()) <= 1e-5, k


def test_empty_calls_are_no_ops(L):
    """M = 0 points and n = 0 counters: nothing to do, status OK."""
    pr = W.gauss_diag(d=5, M=2, n_steps=5)
    tg = L.Target.from_problem(pr)
    lp, g = tg.logp_grad(torch.empty(0, 5, dtype=torch.float32, device="cuda"))
    assert lp.numel() == 0 and g.numel() == 0
    out = L.philox(torch.empty(0, 4, dtype=torch.int32, device="cuda"), 1)
    assert out.numel() == 0


def test_batch_partitioned_by_problems(L, ora):
    """A batch split over two ranks by laps_batch_partition (the ranks emulated
    one after the other on this GPU; the sub-batches exchange nothing): each
    sub-batch carries its problems' ids of the whole batch, so every problem
    follows the oracle run with pid = its index in the whole batch (first
    steps at a fixed step size) and the whole batch's run of it."""
    probs = _probs(SPEC, 40)
    shares = L.partition_problems(probs, 2)
    assert sorted(shares[0] + shares[1]) == list(range(len(probs))) and all(shares)
    whole = L.Batch(probs, n_total_steps=40, fixed_eps=0.05)
    whole.init(seed=21)
    whole.step(4)
    for share in shares:
        sub = L.Batch([probs[k] for k in share], n_total_steps=40, fixed_eps=0.05, ids=share)
        sub.init(seed=21)
        sub.step(4)
        for j, k in enumerate(share):
            r = _ora(ora, probs[k], 21, k, fixed_eps=0.05)
            r.iterate(4)
            xs = sub.sample(j).double().cpu().numpy()
            assert _rel(xs, r.x()) <= 1e-5, (k, share)
            assert _rel(xs, whole.sample(k).double().cpu().numpy()) <= 1e-5, (k, share)
    with pytest.raises(L.LapsError):
        L.Batch(probs[:2], n_total_steps=40, ids=[3, 3])
    with pytest.raises(L.LapsError):
        L.Batch(probs[:1], n_total_steps=40, ids=[1 << 24])
