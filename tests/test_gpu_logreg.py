"""GPU parity of the logistic-regression target and the streamed LAPS path
(state in global memory, gradient by the ensemble contraction kernel) against
the FP64 oracle.

Data sets are reduced (n = 77 .. 3000 rows) so that the oracle finishes in
seconds; shapes are chosen to be ragged against the kernels' tiles (64 chains,
64 data rows, feature padding to a multiple of 64).  The posterior moments of
this target have no closed form: whole runs are compared with the oracle run
on the same data, seed and Philox streams.
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


def _ot(ora, pr):
    return ora.OracleTarget(pr.kind, pr.d, X=pr.X, y=pr.y, prior_var=pr.prior_var)


def _gpu(L, pr, seed=0, **cfg):
    tg = L.Target.from_problem(pr)
    s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=seed)
    s._tg = tg
    return s


def _ora(ora, pr, seed=0, **cfg):
    return ora.OracleLAPS(_ot(ora, pr), pr.x0, seed=seed, n_total_steps=pr.n_steps, **cfg)


def _rel(xg, xr):
    return (np.linalg.norm(xg - xr, axis=1) / np.linalg.norm(xr, axis=1)).max()


# ------------------------------------------------------------------ the target
@pytest.mark.parametrize("n,nf,M", [(1000, 100, 300), (77, 5, 65), (3000, 250, 130),
                                    (500, 60, 64), (64, 63, 2)])
def test_logreg_logp_grad(L, ora, n, nf, M):
    pr = W.logreg(n_data=n, n_feat=nf, M=M, n_steps=10)
    rng = np.random.default_rng(3)
    x = (0.3 * rng.standard_normal((M, pr.d))).astype(np.float32)
    tg = L.Target.from_problem(pr)
    lp, g = tg.logp_grad(torch.from_numpy(x).cuda())
    lpr, gr = _ot(ora, pr).logp_grad(x.astype(np.float64))
    g = g.double().cpu().numpy()
    scale = np.abs(gr).max(axis=1, keepdims=True)
    assert np.max(np.abs(g - gr) / scale) < 1e-5
    # FP32 sums of n terms of size ~1: |error| ~ 1e-7 sqrt(n) per term scale
    np.testing.assert_allclose(lp.double().cpu().numpy(), lpr, rtol=2e-6, atol=1e-3)


def test_logreg_autograd_vs_finite_differences(L, ora):
    from paper_2601_16696_gb300.autograd import target_logp
    pr = W.logreg(n_data=400, n_feat=20, M=16, n_steps=10)
    rng = np.random.default_rng(5)
    x = torch.from_numpy((0.3 * rng.standard_normal((16, pr.d))).astype(np.float32)).cuda()
    x.requires_grad_(True)
    tg = L.Target.from_problem(pr)
    w = torch.linspace(0.5, 1.5, 16, device="cuda")
    (target_logp(x, tg) * w).sum().backward()
    ot = _ot(ora, pr)
    xd = x.detach().double().cpu().numpy()
    h = 1e-4
    fd = np.zeros_like(xd)
    for i in range(pr.d):  # central differences of the FP64 oracle, h = 1e-4
        e = np.zeros(pr.d)
        e[i] = h
        fd[:, i] = (ot.logp_grad(xd + e)[0] - ot.logp_grad(xd - e)[0]) / (2 * h)
    want = fd * w.double().cpu().numpy()[:, None]
    got = x.grad.double().cpu().numpy()
    scale = np.abs(want).max(axis=1, keepdims=True)
    assert np.max(np.abs(got - want) / scale) < 1e-5


# ------------------------------------------------------------------ the sampler
@pytest.mark.parametrize("n,nf,M", [(1000, 100, 512), (300, 30, 77), (400, 150, 130),
                                    (200, 240, 33)])
def test_logreg_first_ten_steps_fixed_step(L, ora, n, nf, M):
    pr = W.logreg(n_data=n, n_feat=nf, M=M, n_steps=200)
    s = _gpu(L, pr, seed=3, fixed_eps=0.01)
    assert s.launch_info()["resident"] == 0
    r = _ora(ora, pr, seed=3, fixed_eps=0.01)
    np.testing.assert_array_equal(s.sample().double().cpu().numpy(), pr.x0)
    for k in range(10):
        s.step(1)
        r.iterate(1)
        rel = _rel(s.sample().double().cpu().numpy(), r.x())
        assert rel <= 1e-5, (k + 1, rel)
    for a, b in zip(s.trace()[:11], r.trace[:11]):
        assert a["L"] == pytest.approx(b["L"], rel=1e-5)
        assert a["t"] == b["t"]


def test_logreg_first_ten_steps_adaptive(L, ora):
    pr = W.logreg(n_data=1000, M=512, n_steps=200)
    s = _gpu(L, pr, seed=3)
    r = _ora(ora, pr, seed=3)
    r32 = _ora(ora, pr, seed=3, round_state_f32=1)
    rows = []
    for k in range(10):
        s.step(1)
        r.iterate(1)
        r32.iterate(1)
        xr = r.x()
        bar = max(1e-5, 3.0 * _rel(r32.x(), xr))
        rel = _rel(s.sample().double().cpu().numpy(), xr)
        rows.append("%d: %.1e / %.1e" % (k + 1, rel, bar))
        assert rel <= bar, (k + 1, rel, bar)
    print("logreg adaptive first steps, error / bar: %s" % ", ".join(rows))


def test_logreg_adjusted_proposals_match(L, ora):
    """The first MAMS proposals after a forced switch, step size held by the
    oracle's own bisection: same accept decisions on almost every chain."""
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=60)
    s = _gpu(L, pr, seed=1, **cfg)
    r = _ora(ora, pr, seed=1, **cfg)
    s.step(60)
    r.iterate(60)
    assert s.stats()["phase"] == 1 == r.phase
    assert s.stats()["integrator"] == r.integrator == 1
    for _ in range(3):
        s.step(1)
        r.iterate(1)
        tg, tr = s.trace()[-1], r.trace[-1]
        assert tg["t"] == tr["t"]
        assert tg["acc"] == pytest.approx(tr["acc"], abs=0.02)
        assert tg["eps"] == pytest.approx(tr["eps"], rel=1e-3)


def test_logreg_whole_run_matches_oracle(L, ora):
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=100)
    s = _gpu(L, pr, seed=0, **cfg)
    s.run()
    st = s.stats()
    r = _ora(ora, pr, seed=0, **cfg)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase == 1
    assert st["t_switch"] == r.t_switch and st["integrator"] == r.integrator
    xg = s.sample().double().cpu().numpy()
    xr = r.x()
    # second moments of the two final ensembles: the oracle's as the reference
    m2g, m2r = (xg ** 2).mean(0), (xr ** 2).mean(0)
    v2r = (xr ** 2).var(0)
    b2 = float(np.mean((m2g - m2r) ** 2 / v2r))
    assert b2 < 10.0 / pr.M, b2  # two independent ensembles give ~2/M
    frozen = [row["acc"] for row in s.trace() if row["phase"] == 1 and not row["adapting"]]
    assert not frozen or abs(np.mean(frozen) - 0.7) < 0.1


# ------------------------------------------------------------------ mixed precision
# The unadjusted phase of the mixed form evaluates the target on BF16-rounded
# data with the tensor cores: points as two BF16 terms (about 16 significant
# bits), residuals y - sigmoid(z) as one BF16 term, FP32 accumulation.  Its
# reference is the FP64 oracle on the BF16-rounded data; the error bars below
# are the arithmetic's, stated with the result.

def _bf16_round(X):
    return torch.from_numpy(np.asarray(X, dtype=np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("n,nf,M", [(1000, 100, 300), (77, 5, 129), (3000, 120, 8192),
                                    (64, 63, 2), (10000, 100, 256)])
def test_mixed_gradient_vs_oracle_on_bf16_data(L, ora, n, nf, M):
    pr = W.logreg(n_data=n, n_feat=nf, M=M, n_steps=10)
    s = _gpu(L, pr, seed=0, precision=1)
    _, _, g, lp, _ = s.state()
    ot = ora.OracleTarget(pr.kind, pr.d, X=_bf16_round(pr.X), y=pr.y, prior_var=pr.prior_var)
    lpr, gr = ot.logp_grad(pr.x0.astype(np.float64))
    g = g.double().cpu().numpy()
    scale = np.abs(gr).max(axis=1, keepdims=True)
    err_g = np.max(np.abs(g - gr) / scale)
    # one BF16 rounding of each residual (relative 2^-9), averaged over the rows
    assert err_g < 4e-3, err_g
    err_lp = np.max(np.abs(lp.cpu().numpy() - lpr) / (np.abs(lpr) + 1.0))
    assert err_lp < 2e-5, err_lp


@pytest.mark.parametrize("n,nf,M", [(1000, 100, 300), (129, 40, 1000)])
def test_mixed_target_call_vs_oracle_on_bf16_data(L, ora, n, nf, M):
    pr = W.logreg(n_data=n, n_feat=nf, M=M, n_steps=10)
    rng = np.random.default_rng(9)
    x = (0.3 * rng.standard_normal((M, pr.d))).astype(np.float32)
    tg = L.Target.from_problem(pr)
    lp, g = tg.logp_grad(torch.from_numpy(x).cuda(), precision=1)
    tg.check()  # no bounded wait expired
    ot = ora.OracleTarget(pr.kind, pr.d, X=_bf16_round(pr.X), y=pr.y, prior_var=pr.prior_var)
    lpr, gr = ot.logp_grad(x.astype(np.float64))
    g = g.double().cpu().numpy()
    assert np.max(np.abs(g - gr) / np.abs(gr).max(axis=1, keepdims=True)) < 4e-3
    assert np.max(np.abs(lp.double().cpu().numpy() - lpr) / (np.abs(lpr) + 1.0)) < 2e-5


def test_mixed_first_steps_error_stated(L, ora):
    pr = W.logreg(n_data=1000, M=512, n_steps=200)
    s = _gpu(L, pr, seed=3, fixed_eps=0.01, precision=1)
    ot = ora.OracleTarget(pr.kind, pr.d, X=_bf16_round(pr.X), y=pr.y, prior_var=pr.prior_var)
    r = ora.OracleLAPS(ot, pr.x0, seed=3, n_total_steps=pr.n_steps, fixed_eps=0.01)
    errs = []
    for _ in range(10):
        s.step(1)
        r.iterate(1)
        errs.append(_rel(s.sample().double().cpu().numpy(), r.x()))
    assert max(errs) < 1e-4, errs


def test_mixed_whole_run_matches_oracle(L, ora):
    """A whole mixed-precision run (BF16 tensor-core contraction while
    unadjusted, FP32 once adjusted) against the FP64 oracle on the FP32 data:
    the adjusted phase's Metropolis test targets the FP32 posterior, so the
    final ensemble is held to the FP32 form's bar, b^2 of its second moments
    against the oracle's final ensemble below 10/M (two independent ensembles
    of the same posterior give ~2/M)."""
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=100)
    a = _gpu(L, pr, seed=0, precision=1, **cfg)
    a.run()
    r = _ora(ora, pr, seed=0, **cfg)
    r.run()
    sa = a.stats()
    assert sa["t"] == r.t and sa["t_switch"] == r.t_switch == 100 and sa["integrator"] == r.integrator
    xa, xr = a.sample().double().cpu().numpy(), r.x()
    m2a, m2r, v2r = (xa ** 2).mean(0), (xr ** 2).mean(0), (xr ** 2).var(0)
    b2 = float(np.mean((m2a - m2r) ** 2 / v2r))
    print("mixed whole run: b^2 of the final second moments against the oracle's %.2e (bar %.2e)"
          % (b2, 10.0 / pr.M))
    assert b2 < 10.0 / pr.M, b2
    # the adjusted phase tests log p of one arithmetic: acceptance is sane from the first proposal
    rows = [r for r in a.trace() if r["phase"] == 1 and r["acc"] == r["acc"]]
    assert rows[0]["acc"] > 0.5, rows[0]
    frozen = [r["acc"] for r in rows if not r["adapting"]]
    assert not frozen or abs(np.mean(frozen) - 0.7) < 0.1


def test_mixed_rejects_unbuilt_shapes(L):
    pr = W.logreg(n_data=200, n_feat=150, M=64, n_steps=10)  # d = 151 -> kp = 192
    tg = L.Target.from_problem(pr)
    with pytest.raises(L.LapsError) as e:
        L.Sampler(tg, pr.M, n_total_steps=10, precision=1)
    assert e.value.status == 6


def test_logreg_determinism_and_checkpoint(L):
    pr = W.logreg(n_data=500, n_feat=30, M=200, n_steps=200)
    outs = []
    for _ in range(2):
        s = _gpu(L, pr, seed=9, force_switch_at=50)
        s.run()
        outs.append(s.sample().cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    a = _gpu(L, pr, seed=4, force_switch_at=50)
    a.step(40)
    blob = a.checkpoint()
    a.step(40)
    b = _gpu(L, pr, seed=7, force_switch_at=50)
    b.restore(blob)
    b.step(40)
    np.testing.assert_array_equal(a.sample().cpu().numpy(), b.sample().cpu().numpy())
