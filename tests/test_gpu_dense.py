"""GPU parity of the dense-precision Gaussian (the randomly oriented
ill-conditioned Gaussian of the paper's Sec. 6), sampled in the register-resident
kernel (P in shared memory, one matrix-vector product per chain) for d <= 128
and on the streamed path (its gradient -P x one chains-by-coordinates
contraction) beyond, both against the FP64 oracle on the same binary32-rounded
precision matrix; the run-level tests cover both paths.

The target is ill-conditioned (condition number 1.1e5), so -P x cancels and a
binary32 dot product is off by ~1e-4 of max|g|; the kernel accumulates the
products exactly in float-float (a compensated dot product), so gradients are
held to 1e-6 of max|g| per point and log p to 1e-6 relative.  Per-chain
positions within 1e-5 over the first 10 steps; final b^2 within 10% (a run
switched into MAMS is held to its path-independent quantities, see below).
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


def _gpu(L, pr, seed=0, **cfg):
    tg = L.Target.from_problem(pr)
    s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
    s.set_truth(pr.Ex2, pr.Varx2)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=seed)
    s._tg = tg
    return s


def _ora(ora, pr, seed=0, **cfg):
    ot = ora.OracleTarget(ora.GAUSS_DENSE, pr.d, prec=pr.prec)
    return ora.OracleLAPS(ot, pr.x0, seed=seed, truth=(pr.Ex2, pr.Varx2), n_total_steps=pr.n_steps,
                          **cfg)


def _rel(a, b):
    return float((np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max())


@pytest.mark.parametrize("d,M", [(100, 1000), (7, 33), (37, 65), (300, 100), (512, 40)])
def test_dense_logp_grad(L, ora, d, M):
    """Points from N(0, I) (far from the target's typical set: gradients up to
    ~1e4 with cancellation) and from the target itself; ragged M and d."""
    pr = W.icg(d=d, M=M, seed=1)
    rng = np.random.default_rng(5)
    lc = np.linalg.cholesky(pr.extra["cov"])
    for X in (rng.standard_normal((M, d)), rng.standard_normal((M, d)) @ lc.T):
        X = X.astype(np.float32).astype(np.float64)
        lp, g = L.Target.from_problem(pr).logp_grad(torch.tensor(X, dtype=torch.float32, device="cuda"))
        lp_o, g_o = ora.OracleTarget(ora.GAUSS_DENSE, d, prec=pr.prec).logp_grad(X)
        g = g.double().cpu().numpy()
        err = np.abs(g - g_o).max(axis=1) / np.abs(g_o).max(axis=1)
        assert err.max() <= 1e-6, err.max()
        np.testing.assert_allclose(lp.double().cpu().numpy(), lp_o, rtol=1e-6)


PATHS = [pytest.param(0, id="resident"), pytest.param(1, id="streamed")]


@pytest.mark.parametrize("streamed", PATHS)
def test_dense_first_ten_steps_fixed_step(L, ora, streamed):
    """Full size (d = 100, M = 4096, condition number 1.1e5), step size held fixed."""
    pr = W.icg()
    s = _gpu(L, pr, seed=3, fixed_eps=0.002, dense_streamed=streamed)
    assert s.launch_info()["resident"] == 1 - streamed
    r = _ora(ora, pr, seed=3, fixed_eps=0.002)
    np.testing.assert_array_equal(s.sample().double().cpu().numpy(), pr.x0)
    for k in range(10):
        s.step(1)
        r.iterate(1)
        rel = _rel(s.sample().double().cpu().numpy(), r.x())
        assert rel <= 1e-5, (k + 1, rel)
    for a, b in zip(s.trace()[1:11], r.trace[1:11]):
        assert a["dtilde"] == pytest.approx(b["dtilde"], rel=1e-4)
        assert a["L"] == pytest.approx(b["L"], rel=1e-5)


@pytest.mark.parametrize("streamed", PATHS)
def test_dense_first_ten_steps_adaptive(L, ora, streamed):
    """Paper defaults: the bar is 3x the oracle's own divergence from its run
    with a binary32 state (see tests/test_gpu_parity.py), never below 1e-5."""
    pr = W.icg(M=1024)
    s = _gpu(L, pr, seed=3, dense_streamed=streamed)
    r = _ora(ora, pr, seed=3)
    r32 = _ora(ora, pr, seed=3, round_state_f32=1)
    rows = []
    for k in range(10):
        s.step(1)
        r.iterate(1)
        r32.iterate(1)
        bar = max(1e-5, 3.0 * _rel(r32.x(), r.x()))
        rel = _rel(s.sample().double().cpu().numpy(), r.x())
        rows.append("%d: %.1e / %.1e" % (k + 1, rel, bar))
        assert rel <= bar, (k + 1, rel, bar)
    print("icg (%s) adaptive first steps, error / bar: %s"
          % ("streamed" if streamed else "resident", ", ".join(rows)))
    assert s.trace()[1]["eps_used"] == pytest.approx(r.trace[1]["eps_used"], rel=1e-6)


def _tail(trace, key, phase):
    rows = [x for x in trace[1:] if x["phase"] == phase]
    return float(np.mean([x[key] for x in rows[len(rows) // 2:]]))


@pytest.mark.parametrize("streamed", PATHS)
def test_dense_final_b2_within_10_percent(L, ora, streamed):
    """Whole unswitched run, M = 1024, 2000 steps (oracle seed-to-seed spread of
    the b^2_avg tail mean 2%); b^2_max falls below 0.01 after ~630 gradients."""
    pr = W.icg(M=1024, n_steps=2000)
    s = _gpu(L, pr, seed=0, dense_streamed=streamed)
    s.run()
    st = s.stats()
    r = _ora(ora, pr, seed=0)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase == 0
    bg, bo = _tail(s.trace(), "b2_avg", 0), _tail(r.trace, "b2_avg", 0)
    assert abs(bg - bo) <= 0.10 * bo, (bg, bo)


_SWITCHED_SEEDS = (0, 1, 2, 3, 4)
_switched_oracle = {}


def _switched_oracle_runs(ora, pr, cfg):
    """The oracle's switched runs, seeds 0..4 (computed once for both paths)."""
    if not _switched_oracle:
        for sd in _SWITCHED_SEEDS:
            r = _ora(ora, pr, seed=sd, **cfg)
            r.run()
            _switched_oracle[sd] = (r.t, r.phase, r.t_switch, r.trace)
    return _switched_oracle


@pytest.mark.parametrize("streamed", PATHS)
def test_dense_switched_run(L, ora, streamed):
    """Switch forced at step 400: the diagonal preconditioner cannot undo the
    rotation, so MAMS is still removing bias at the end and one run's b^2
    depends on its path (oracle seed spread of the b^2_avg tail mean 17%,
    0.0044-0.0062).  The 10% bar on b^2 is therefore applied to means over
    five seeds of the b^2_avg tail means.  The step size the bisection freezes at (0.239-0.245 over the seeds;
    set at the first proposal within 0.03 of the target acceptance, so it
    moves in steps of a few percent between paths) and the acceptance
    (0.72-0.74) are held to 6% and 0.06 on seed 0."""
    pr = W.icg(M=1024, n_steps=2000)
    cfg = {"force_switch_at": 400}
    ref = _switched_oracle_runs(ora, pr, cfg)
    bgs, bos = [], []
    for sd in _SWITCHED_SEEDS:
        s = _gpu(L, pr, seed=sd, dense_streamed=streamed, **cfg)
        s.run()
        st = s.stats()
        rt, rphase, rsw, rtrace = ref[sd]
        assert st["t"] == rt and st["phase"] == rphase == 1 and st["t_switch"] == rsw == 400
        tg = s.trace()
        if sd == 0:
            assert tg[-1]["eps"] == pytest.approx(rtrace[-1]["eps"], rel=0.06)
            ag = np.mean([x["acc"] for x in tg[-20:]])
            ao = np.mean([x["acc"] for x in rtrace[-20:]])
            assert abs(ag - ao) <= 0.06, (ag, ao)
        bgs.append(_tail(tg, "b2_avg", 1))
        bos.append(_tail(rtrace, "b2_avg", 1))
    bg, bo = float(np.mean(bgs)), float(np.mean(bos))
    print("dense switched run (%s): b^2_avg tail, 5-seed mean: GPU %.4g, oracle %.4g"
          % ("streamed" if streamed else "resident", bg, bo))
    assert abs(bg - bo) <= 0.10 * bo, (bgs, bos)


@pytest.mark.parametrize("streamed", PATHS)
def test_dense_determinism_and_checkpoint(L, streamed):
    pr = W.icg(d=40, M=200, n_steps=300)
    a = _gpu(L, pr, seed=4, force_switch_at=100, dense_streamed=streamed)
    a.step(150)
    b = _gpu(L, pr, seed=4, force_switch_at=100, dense_streamed=streamed)
    b.step(90)
    blob = b.checkpoint()
    c = _gpu(L, pr, seed=99, force_switch_at=100, dense_streamed=streamed)
    c.restore(blob)
    c.step(60)
    np.testing.assert_array_equal(a.sample().cpu().numpy(), c.sample().cpu().numpy())
    assert a.stats()["eps"] == c.stats()["eps"]


def test_dense_path_by_dimension(L, ora):
    """d <= 128 runs in the register-resident kernel, larger d on the streamed
    path; the larger case's first steps against the oracle."""
    pr = W.icg(d=150, M=256, n_steps=50)
    s = _gpu(L, pr, seed=2, fixed_eps=0.002)
    assert s.launch_info()["resident"] == 0
    r = _ora(ora, pr, seed=2, fixed_eps=0.002)
    s.step(5)
    r.iterate(5)
    assert _rel(s.sample().double().cpu().numpy(), r.x()) <= 1e-5
    small = W.icg(d=37, M=65, n_steps=50)
    s = _gpu(L, small, seed=2, fixed_eps=0.002)
    assert s.launch_info()["resident"] == 1
    r = _ora(ora, small, seed=2, fixed_eps=0.002)
    s.step(5)
    r.iterate(5)
    assert _rel(s.sample().double().cpu().numpy(), r.x()) <= 1e-5


def test_dense_rejected_where_not_built(L):
    pr = W.icg(d=16, M=32, n_steps=10)
    tg = L.Target.from_problem(pr)
    with pytest.raises(L.LapsError):
        L.Sampler(tg, pr.M, n_total_steps=10, dtilde_K=10)     # full-rank proxy: resident only
    with pytest.raises(L.LapsError):
        L.Sampler(tg, pr.M, n_total_steps=10, precision=1)     # mixed precision: LOGREG only
    big = W.icg(d=520, M=4, n_steps=10)
    with pytest.raises(L.LapsError):
        L.Target.from_problem(big)                             # d > 512
