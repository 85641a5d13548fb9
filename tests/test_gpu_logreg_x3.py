"""GPU parity of the logistic-regression gradient on the tensor cores at FP32
accuracy (precision LAPS_BF16X3: points, data and residuals each split into
three BF16 terms, the six cross products of order >= 2^-16, FP32 accumulation)
and of the sampler forms that use it (LAPS_BF16X3 in both phases,
LAPS_MIXED_BF16X3 once adjusted), against the FP64 oracle on the unrounded
data.

The bars are those of the FP32 form (test_gpu_logreg.py): this arithmetic
claims FP32 accuracy, so it is held to the FP32 form's tolerances, and its
gradient error is compared with the FP32 form's own on the same points.
Shapes are ragged against the kernel's tiles (128 chains, 64 data rows,
feature padding to 64 or 128).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2601_16696_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

BF16X3, MIXED_BF16X3 = 2, 3


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


def _errs(g, lp, gr, lpr):
    g = g.double().cpu().numpy()
    scale = np.abs(gr).max(axis=1, keepdims=True)
    eg = float(np.max(np.abs(g - gr) / scale))
    el = float(np.max(np.abs(lp.double().cpu().numpy() - lpr) / (np.abs(lpr) + 1.0)))
    return eg, el


# ------------------------------------------------------------------ the target
@pytest.mark.parametrize("n,nf,M", [(1000, 100, 300), (77, 5, 65), (500, 60, 64), (64, 63, 2),
                                    (3000, 127, 130), (129, 40, 1000)])
def test_x3_logp_grad(L, ora, n, nf, M):
    pr = W.logreg(n_data=n, n_feat=nf, M=M, n_steps=10)
    rng = np.random.default_rng(3)
    x = (0.3 * rng.standard_normal((M, pr.d))).astype(np.float32)
    tg = L.Target.from_problem(pr)
    xd = torch.from_numpy(x).cuda()
    lp, g = tg.logp_grad(xd, precision=BF16X3)
    tg.check()  # no bounded wait expired
    lpr, gr = _ot(ora, pr).logp_grad(x.astype(np.float64))
    eg, el = _errs(g, lp, gr, lpr)
    assert eg < 1e-5, eg
    np.testing.assert_allclose(lp.double().cpu().numpy(), lpr, rtol=2e-6, atol=1e-3)
    # FP32 accuracy: not far from the FP32 form's own error on the same points
    lp32, g32 = tg.logp_grad(xd, precision=0)
    eg32, el32 = _errs(g32, lp32, gr, lpr)
    assert eg <= max(4.0 * eg32, 2e-6), (eg, eg32)
    assert el <= max(4.0 * el32, 1e-7), (el, el32)


def test_x3_logp_grad_full_size_sampled(L, ora):
    """The bench's logistic regression (n = 10^4, d = 101, M = 8192), one launch
    over every chain; 64 sampled chains against the oracle.  The split form's
    gradient stays under the FP32 bar (1e-5 of max|g|), which the BF16 form
    misses by far, so the bar tells the two classes apart.  At this size the
    FP32 form adds its rows in seven ranges of ~1430 (the wave-filling split),
    the split form in two ranges of 5000 in tensor memory, so here the FP32
    form is the more accurate of the two (printed)."""
    pr = W.logreg(n_steps=10)
    assert pr.M == 8192 and pr.d == 101
    rng = np.random.default_rng(8)
    x = (0.2 * rng.standard_normal((pr.M, pr.d))).astype(np.float32)
    tg = L.Target.from_problem(pr)
    xd = torch.from_numpy(x).cuda()
    lp, g = tg.logp_grad(xd, precision=BF16X3)
    tg.check()
    idx = np.sort(rng.choice(pr.M, 64, replace=False))
    lpr, gr = _ot(ora, pr).logp_grad(x[idx].astype(np.float64))
    eg, el = _errs(g[idx], lp[idx], gr, lpr)
    lp32, g32 = tg.logp_grad(xd, precision=0)
    eg32, el32 = _errs(g32[idx], lp32[idx], gr, lpr)
    lp16, g16 = tg.logp_grad(xd, precision=1)
    eg16, _ = _errs(g16[idx], lp16[idx], gr, lpr)
    print("full-size gradient error / max|g|: split form %.2e, FP32 form %.2e, BF16 form %.2e" % (eg, eg32, eg16))
    assert eg < 1e-5, (eg, eg32)
    assert eg32 < 1e-5, eg32
    assert eg16 > 1e-5, eg16
    assert el < 2e-6, (el, el32)
    assert torch.isfinite(g).all() and torch.isfinite(lp).all()


def test_x3_rejects_unbuilt_shapes(L):
    pr = W.logreg(n_data=200, n_feat=150, M=64, n_steps=10)  # d = 151 -> kp = 192
    tg = L.Target.from_problem(pr)
    for p in (BF16X3, MIXED_BF16X3):
        with pytest.raises(L.LapsError) as e:
            L.Sampler(tg, pr.M, n_total_steps=10, precision=p)
        assert e.value.status == 6
    with pytest.raises(L.LapsError):
        tg.logp_grad(torch.zeros(4, pr.d, device="cuda"), precision=BF16X3)


# ------------------------------------------------------------------ the sampler
@pytest.mark.parametrize("n,nf,M", [(1000, 100, 512), (300, 30, 77), (200, 127, 33)])
def test_x3_first_ten_steps_fixed_step(L, ora, n, nf, M):
    pr = W.logreg(n_data=n, n_feat=nf, M=M, n_steps=200)
    s = _gpu(L, pr, seed=3, fixed_eps=0.01, precision=BF16X3)
    r = _ora(ora, pr, seed=3, fixed_eps=0.01)
    for k in range(10):
        s.step(1)
        r.iterate(1)
        rel = _rel(s.sample().double().cpu().numpy(), r.x())
        assert rel <= 1e-5, (k + 1, rel)
    for a, b in zip(s.trace()[:11], r.trace[:11]):
        assert a["L"] == pytest.approx(b["L"], rel=1e-5)


def test_x3_first_ten_steps_adaptive(L, ora):
    pr = W.logreg(n_data=1000, M=512, n_steps=200)
    s = _gpu(L, pr, seed=3, precision=BF16X3)
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
    print("logreg bf16x3 adaptive first steps, error / bar: %s" % ", ".join(rows))


@pytest.mark.parametrize("precision", [BF16X3, MIXED_BF16X3])
def test_x3_adjusted_proposals_match(L, ora, precision):
    """The first MAMS proposals after a forced switch: acceptance and the
    bisected step size as the oracle's (the mixed form reaches the switch on
    the BF16 data, so its state there differs slightly)."""
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=60)
    s = _gpu(L, pr, seed=1, precision=precision, **cfg)
    r = _ora(ora, pr, seed=1, **cfg)
    s.step(60)
    r.iterate(60)
    assert s.stats()["phase"] == 1 == r.phase
    tol_acc, tol_eps = (0.02, 1e-3) if precision == BF16X3 else (0.05, 0.02)
    for _ in range(3):
        s.step(1)
        r.iterate(1)
        tg, tr = s.trace()[-1], r.trace[-1]
        assert tg["t"] == tr["t"]
        assert tg["acc"] == pytest.approx(tr["acc"], abs=tol_acc)
        assert tg["eps"] == pytest.approx(tr["eps"], rel=tol_eps)
    s._tg.check()


@pytest.mark.parametrize("precision", [BF16X3, MIXED_BF16X3])
def test_x3_whole_run_matches_oracle(L, ora, precision):
    pr = W.logreg(n_data=1000, M=512, n_steps=400)
    cfg = dict(force_switch_at=100)
    s = _gpu(L, pr, seed=0, precision=precision, **cfg)
    s.run()
    st = s.stats()
    r = _ora(ora, pr, seed=0, **cfg)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase == 1
    assert st["t_switch"] == r.t_switch
    xg = s.sample().double().cpu().numpy()
    xr = r.x()
    m2g, m2r = (xg ** 2).mean(0), (xr ** 2).mean(0)
    v2r = (xr ** 2).var(0)
    b2 = float(np.mean((m2g - m2r) ** 2 / v2r))
    assert b2 < 10.0 / pr.M, b2  # two independent ensembles give ~2/M
    rows = [row for row in s.trace() if row["phase"] == 1 and row["acc"] == row["acc"]]
    assert rows[0]["acc"] > 0.5, rows[0]  # one arithmetic in every Metropolis test
    frozen = [row["acc"] for row in rows if not row["adapting"]]
    assert not frozen or abs(np.mean(frozen) - 0.7) < 0.1


def test_x3_determinism_and_checkpoint(L):
    pr = W.logreg(n_data=500, n_feat=30, M=200, n_steps=200)
    outs = []
    for _ in range(2):
        s = _gpu(L, pr, seed=9, force_switch_at=50, precision=BF16X3)
        s.run()
        outs.append(s.sample().cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    a = _gpu(L, pr, seed=4, force_switch_at=50, precision=MIXED_BF16X3)
    a.step(40)
    blob = a.checkpoint()
    a.step(40)
    b = _gpu(L, pr, seed=7, force_switch_at=50, precision=MIXED_BF16X3)
    b.restore(blob)
    b.step(40)
    np.testing.assert_array_equal(a.sample().cpu().numpy(), b.sample().cpu().numpy())


def test_precision_values_checked(L):
    pr = W.logreg(n_data=200, n_feat=20, M=64, n_steps=10)
    tg = L.Target.from_problem(pr)
    with pytest.raises(L.LapsError) as e:
        L.Sampler(tg, pr.M, n_total_steps=10, precision=7)
    assert e.value.status == 1  # LAPS_ERR_INVALID_ARG
    g = W.gauss_diag(d=10, M=64, n_steps=10)
    gt = L.Target.from_problem(g)
    for p in (BF16X3, MIXED_BF16X3):
        with pytest.raises(L.LapsError) as e:
            L.Sampler(gt, g.M, n_total_steps=10, precision=p)
        assert e.value.status == 6  # LAPS_ERR_UNSUPPORTED: the split forms are LOGREG's


def test_long_run_against_reference_moments(L):
    """A run at full size (n = 10^4 rows, d = 101) with M = 16384 chains, the
    switch forced at step 200 and MAMS at FP32 accuracy on the tensor cores
    to step 1200, against the stored reference moments of this posterior
    (importance sampling in FP64, independent of the sampler): over the last
    half of the adjusted phase b^2 stays at the finite-M floor of exact
    samples (E b^2_avg = 1/M; b^2_max about the largest of 101 chi^2_1 draws
    over M, ~10/M)."""
    ref = W.logreg_reference_moments()
    if ref is None:
        pytest.skip("reference moments not generated")
    pr = W.logreg(M=16384, n_steps=1200)
    s = _gpu(L, pr, seed=5, precision=BF16X3, force_switch_at=200)
    s.set_truth(*ref)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=5)
    s.run()
    st = s.stats()
    assert st["phase"] == 1 and st["t_switch"] == 200
    rows = [r for r in s.trace() if r["phase"] == 1 and r["t"] > 200]
    tail = rows[len(rows) // 2:]
    b2a = float(np.mean([r["b2_avg"] for r in tail]))
    b2m = float(np.mean([r["b2_max"] for r in tail]))
    acc = float(np.mean([r["acc"] for r in tail]))
    print("long logreg run, M = %d: tail b^2_avg %.2e (%.2f/M), b^2_max %.2e (%.1f/M), acceptance %.3f"
          % (pr.M, b2a, b2a * pr.M, b2m, b2m * pr.M, acc))
    assert b2a < 3.0 / pr.M and b2m < 25.0 / pr.M, (b2a, b2m)
    assert abs(acc - 0.7) < 0.1
