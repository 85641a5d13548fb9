"""The chain-sharded ensemble (laps_create_sharded) on one GPU.

Chains are independent between the ensemble reductions (Sec. 2, Eq. "ECA"),
so an ensemble can be split over ranks that exchange only their totals of the
sums the finalise needs, once per Alg. 1 iteration.  Here:
- one rank: the results equal the unsharded sampler's bit for bit (the rank's
  totals are formed in the finalise's own order and grouping);
- two ranks emulated in one process: two host threads drive one sampler each
  (half of the chains) on their own streams; the exchange is a host barrier
  plus device copies, and no kernel waits on another.  The union of the two
  halves follows the unsharded run (only the association of the ensemble
  sums differs) and the FP64 oracle, and both ranks hold the same step size,
  L and phase machine.
"""
import threading

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


def _rel(xg, xr):
    return (np.linalg.norm(xg - xr, axis=1) / np.linalg.norm(xr, axis=1)).max()


class _Exchange:
    """All-gather between sampler threads of one process: each rank's totals
    are copied into every rank's receive buffer in rank order."""

    def __init__(self, L, n):
        self.L, self.n = L, n
        self.barrier = threading.Barrier(n, timeout=120)
        self.send = [None] * n

    def fn(self, rank):
        def gather(send, recv, nbytes, stream):
            st = torch.cuda.ExternalStream(stream)
            st.synchronize()  # this rank's totals are written
            self.send[rank] = send
            self.barrier.wait()
            with torch.cuda.stream(st):
                for q in range(self.n):
                    self.L.device_bytes(recv + q * nbytes, nbytes).copy_(self.L.device_bytes(self.send[q], nbytes))
            st.synchronize()
            self.barrier.wait()  # no rank reuses its send buffer before every copy ended
        return gather


def _run_ranks(L, pr, n, seed, steps, **cfg):
    """n sampler threads over the chains of pr; returns the samplers after
    `steps` (None: the whole run)."""
    tg = L.Target.from_problem(pr)
    ex = _Exchange(L, n)
    bounds = [k * pr.M // n for k in range(n + 1)]
    samplers = [L.Sampler(tg, bounds[k + 1] - bounds[k], n_total_steps=pr.n_steps,
                          shard=(pr.M, bounds[k], k, n, ex.fn(k)), **cfg) for k in range(n)]
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    errors = []

    def work(k):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                samplers[k].init(x0[bounds[k]:bounds[k + 1]].contiguous(), seed=seed)
                if steps is None:
                    samplers[k].run()
                else:
                    samplers[k].step(steps)
            st.synchronize()
        except Exception as e:  # noqa: BLE001
            errors.append(e)
            ex.barrier.abort()

    ts = [threading.Thread(target=work, args=(k,)) for k in range(n)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=600)
    assert not errors, errors
    torch.cuda.synchronize()
    return samplers, tg


def _union(samplers):
    return np.concatenate([s.sample().double().cpu().numpy() for s in samplers])


def test_one_rank_equals_unsharded(L):
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=100)
    tg = L.Target.from_problem(pr)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    a = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
    a.init(x0, seed=2)
    a.run()
    b = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, shard=(pr.M, 0, 0, 1, None), **cfg)
    b.init(x0, seed=2)
    b.run()
    np.testing.assert_array_equal(a.sample().cpu().numpy(), b.sample().cpu().numpy())
    ta, tb = a.trace(), b.trace()
    assert [r["eps"] for r in ta] == [r["eps"] for r in tb]
    assert a.stats()["t_switch"] == b.stats()["t_switch"] == 100


@pytest.mark.parametrize("n", [2, 3])
def test_two_ranks_first_steps_match_oracle(L, ora, n):
    """Fixed step size: per-chain positions of the union within 1e-5 of the
    unsharded run and of the oracle over 10 steps; every rank's L equal (two
    ranks of 150 and 151 chains, three of 100, 100 and 101)."""
    pr = W.logreg(n_data=1000, M=301, n_steps=200)
    cfg = dict(fixed_eps=0.01)
    ranks, tg = _run_ranks(L, pr, n, 3, 10, **cfg)
    one = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
    one.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=3)
    one.step(10)
    xu = _union(ranks)
    assert _rel(xu, one.sample().double().cpu().numpy()) <= 1e-5
    ot = ora.OracleTarget(pr.kind, pr.d, X=pr.X, y=pr.y, prior_var=pr.prior_var)
    r = ora.OracleLAPS(ot, pr.x0, seed=3, n_total_steps=pr.n_steps, **cfg)
    r.iterate(10)
    assert _rel(xu, r.x()) <= 1e-5
    la = [q["L"] for q in ranks[0].trace()]
    for k in range(1, n):
        assert [q["L"] for q in ranks[k].trace()] == la
    for a, b in zip(la, r.trace):
        assert a == pytest.approx(b["L"], rel=1e-5)


def test_two_ranks_whole_run(L, ora):
    """The controller on, the switch forced at step 100, MAMS to step 400: both
    ranks hold the same phase machine; the union's final second moments
    against the oracle's final ensemble below 10/M, as for one rank."""
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=100)
    ranks, _ = _run_ranks(L, pr, 2, 0, None, **cfg)
    s0, s1 = ranks[0].stats(), ranks[1].stats()
    for k in ("t", "t_switch", "phase", "eps", "L", "integrator", "acc"):
        assert s0[k] == s1[k], k
    r = ora.OracleLAPS(ora.OracleTarget(pr.kind, pr.d, X=pr.X, y=pr.y, prior_var=pr.prior_var), pr.x0,
                       seed=0, n_total_steps=pr.n_steps, **cfg)
    r.run()
    assert s0["t"] == r.t and s0["t_switch"] == r.t_switch == 100
    xu, xr = _union(ranks), r.x()
    b2 = float(np.mean(((xu ** 2).mean(0) - (xr ** 2).mean(0)) ** 2 / (xr ** 2).var(0)))
    print("two-rank logistic-regression run: b^2 against the oracle's final ensemble %.2e (bar %.2e)"
          % (b2, 10.0 / pr.M))
    assert b2 < 10.0 / pr.M


def test_two_ranks_dense_gaussian_first_steps(L, ora):
    pr = W.icg(d=40, M=257, n_steps=100)
    cfg = dict(fixed_eps=0.002, dense_streamed=1)
    ranks, _ = _run_ranks(L, pr, 2, 4, 5, **cfg)
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec)
    r = ora.OracleLAPS(ot, pr.x0, seed=4, n_total_steps=pr.n_steps, fixed_eps=0.002)
    r.iterate(5)
    assert _rel(_union(ranks), r.x()) <= 1e-5


def test_sharded_rejections(L):
    pr = W.banana(d=10, M=8, n_steps=10)
    tg = L.Target.from_problem(pr)
    with pytest.raises(L.LapsError) as e:
        L.Sampler(tg, 8, n_total_steps=10, shard=(8, 0, 0, 1, None))  # register-resident target
    assert e.value.status == 6
    lr = W.logreg(n_data=100, n_feat=5, M=8, n_steps=10)
    ltg = L.Target.from_problem(lr)
    with pytest.raises(L.LapsError) as e:
        L.Sampler(ltg, 8, n_total_steps=10, shard=(12, 6, 0, 2, None))  # chains past M_total, no callback
    assert e.value.status == 1
    with pytest.raises(L.LapsError) as e:
        L.Sampler(ltg, 8, n_total_steps=10, shard=(16, 0, 0, 1, None))  # one rank short of its ensemble
    assert e.value.status == 1
