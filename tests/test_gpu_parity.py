"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Same seeded inputs (workloads), same Philox streams.  Bars: the random
stream bit-exact; target log p / gradients at FP32 accuracy; per-chain
positions within 1e-5 relative over the first 10 steps; final b^2 of the
second moments within 10% of the oracle's.

The 1e-5 position bar is applied with the step size held fixed (the paper's
fixed-step comparison).  With the adaptive controller the first update of
eps divides the wanted EEVPD by a measured EEVPD that is ~1e-8 (u0 is
parallel to g0), so the binary32 rounding of the chain state alone moves the
run by ~1e-4 within a few steps; there the bar is three times the divergence
between the oracle and the oracle run with its state rounded to binary32
(computed from the oracle alone, in the test), and never below 1e-5.
"""
import math

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
    if pr.Ex2 is not None:
        s.set_truth(pr.Ex2, pr.Varx2)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=seed)
    s._tg = tg
    return s


def _ora(ora, pr, seed=0, **cfg):
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb,
                          funnel_sv=pr.funnel_sv)
    truth = (pr.Ex2, pr.Varx2) if pr.Ex2 is not None else None
    return ora.OracleLAPS(ot, pr.x0, seed=seed, truth=truth, n_total_steps=pr.n_steps, **cfg)


# ------------------------------------------------------------------ random stream
def test_philox_bit_exact(L, ora):
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x0123456789ABCDEF
    out = L.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), seed).cpu().numpy()
    ref = ora.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    np.testing.assert_array_equal(out.view(np.uint32), ref)


def test_normals_match_oracle(L, ora):
    for (m0, nm, t, tag, d) in [(0, 300, 5, 1, 101), (17, 64, 0xFFFFFFFF, 1, 7), (3, 50, 9, 3, 64)]:
        g = L.normals(11, m0, nm, t, tag, 2, d).double().cpu().numpy()
        r = ora.normals(11, m0, nm, t, tag, 2, d)
        np.testing.assert_allclose(g, r, rtol=0, atol=3e-6 * max(1.0, np.abs(r).max()))


# ------------------------------------------------------------------ targets
def _points(pr, M, scale, seed):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((M, pr.d))).astype(np.float32)


@pytest.mark.parametrize("name", ["gauss_d100", "banana_d100", "funnel_d101"])
def test_target_logp_grad(L, ora, name):
    pr = W.by_name(name, M=4)
    x = _points(pr, 1000, 0.8, 1)
    tg = L.Target.from_problem(pr)
    lp, g = tg.logp_grad(torch.from_numpy(x).cuda())
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb,
                          funnel_sv=pr.funnel_sv)
    lpr, gr = ot.logp_grad(x.astype(np.float64))
    g = g.double().cpu().numpy()
    scale = np.abs(gr).max(axis=1, keepdims=True)
    # FP32 arithmetic: the funnel's g_v adds terms of size (d-1)/2 that cancel
    assert np.max(np.abs(g - gr) / scale) < 1e-5
    np.testing.assert_allclose(lp.double().cpu().numpy(), lpr, rtol=2e-6, atol=1e-5)


@pytest.mark.parametrize("name", ["gauss_d100", "banana_d100", "funnel_d101"])
def test_autograd_backward_vs_finite_differences(L, ora, name):
    from paper_2601_16696_gb300.autograd import target_logp
    pr = W.by_name(name, M=4)
    x = torch.from_numpy(_points(pr, 64, 0.6, 2)).cuda().requires_grad_(True)
    tg = L.Target.from_problem(pr)
    lp = target_logp(x, tg)
    w = torch.linspace(0.5, 1.5, 64, device="cuda")
    (lp * w).sum().backward()
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb,
                          funnel_sv=pr.funnel_sv)
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


# ------------------------------------------------------------------ first steps
FIXED = {"gauss_d100": 0.05, "banana_d100": 0.1, "funnel_d101": 0.1}


def _rel(xg, xr):
    return (np.linalg.norm(xg - xr, axis=1) / np.linalg.norm(xr, axis=1)).max()


@pytest.mark.parametrize("name", ["gauss_d100", "banana_d100", "funnel_d101"])
def test_first_ten_steps_fixed_step(L, ora, name):
    """Full-size ensembles, step size held fixed: per-chain positions <= 1e-5."""
    pr = W.by_name(name)
    s = _gpu(L, pr, seed=3, fixed_eps=FIXED[name])
    r = _ora(ora, pr, seed=3, fixed_eps=FIXED[name])
    np.testing.assert_array_equal(s.sample().double().cpu().numpy(), pr.x0)
    for k in range(10):
        s.step(1)
        r.iterate(1)
        rel = _rel(s.sample().double().cpu().numpy(), r.x())
        assert rel <= 1e-5, (k + 1, rel)
    for a, b in zip(s.trace()[:11], r.trace[:11]):
        assert a["L"] == pytest.approx(b["L"], rel=1e-5)


@pytest.mark.parametrize("name", ["gauss_d100", "banana_d100", "funnel_d101"])
def test_first_ten_steps_adaptive(L, ora, name):
    """Paper defaults: the bar is set by the oracle's own sensitivity to a
    binary32 state (see the module docstring)."""
    pr = W.by_name(name)
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
    print("%s adaptive first steps, error / bar: %s" % (name, ", ".join(rows)))
    # step 1 uses eps0 and L0 only: it meets the plain bar
    tg = s.trace()
    assert tg[1]["eps_used"] == pytest.approx(r.trace[1]["eps_used"], rel=1e-6)


# ------------------------------------------------------------------ whole runs
def _final_b2(trace, key, frac=0.5):
    """b^2 of the final ensembles: the mean over the last half of the
    iterations of the final phase.  One ensemble's b^2 is dominated by its
    finite-M noise (a chi^2-like draw: ~14% spread for b^2_avg at d = 100,
    ~50% for b^2_max), and the GPU and oracle runs decorrelate after a few
    tens of steps, so single final values differ by that noise; the tail mean
    averages many decorrelated ensembles (oracle seed-to-seed spread 1-5% for
    b^2_avg, ~10% for b^2_max)."""
    rows = [r for r in trace[1:] if r["phase"] == trace[-1]["phase"]]
    n = max(1, int(len(rows) * frac))
    return float(np.mean([r[key] for r in rows[-n:]]))


@pytest.mark.parametrize("name,kw,cfg,key", [
    ("gauss_d100", {}, {}, "b2_avg"),
    ("gauss_d100", {}, {"force_switch_at": 400}, "b2_avg"),
    ("banana_d100", {"M": 4096, "n_steps": 2000}, {"force_switch_at": 400}, "b2_max"),
])
def test_final_b2_within_10_percent(L, ora, name, kw, cfg, key):
    pr = W.by_name(name, **kw)
    s = _gpu(L, pr, seed=0, **cfg)
    s.run()
    st = s.stats()
    r = _ora(ora, pr, seed=0, **cfg)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase
    bg, bo = _final_b2(s.trace(), key), _final_b2(r.trace, key)
    assert abs(bg - bo) <= 0.10 * bo, (bg, bo)
    if cfg.get("force_switch_at"):
        assert st["t_switch"] == r.t_switch and st["integrator"] == r.integrator


def test_funnel_whole_run_statistics(L, ora):
    """The funnel (d = 101, M = 4096, 2000 steps, switch forced at step 400).
    Its b^2 is not a usable bar: Var[x_i^2] is astronomically large, so b^2
    is ~5e-5 and spreads by 20% (b^2_avg) to 5x (b^2_max) between oracle seeds.
    The GPU run is held to what four oracle seeds agree on: the phase machine
    exactly; the frozen acceptance (0.70 .. 0.72); the bisected step size
    (1.85 .. 2.13); E[v^2] of the final ensemble (8.0 .. 8.6, the neck still
    under-sampled against the true 9, with a sampling sd of 0.18)."""
    pr = W.by_name("funnel_d101", n_steps=2000)
    cfg = {"force_switch_at": 400}
    s = _gpu(L, pr, seed=0, **cfg)
    s.run()
    st = s.stats()
    r = _ora(ora, pr, seed=0, **cfg)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase == 1
    assert st["t_switch"] == r.t_switch and st["integrator"] == r.integrator

    def tail(trace):
        rows = [q for q in trace if q["phase"] == 1 and not q["adapting"]]
        return float(np.mean([q["acc"] for q in rows])), rows[-1]["eps_used"]

    (ag, eg), (ao, eo) = tail(s.trace()), tail(r.trace)
    assert abs(ag - ao) <= 0.03, (ag, ao)
    assert abs(eg - eo) <= 0.2 * eo, (eg, eo)
    vg = float((s.sample()[:, 0].double() ** 2).mean())
    vo = float((r.x()[:, 0] ** 2).mean())
    assert abs(vg - vo) <= 1.0 and 7.0 <= vg <= 10.0, (vg, vo)
    assert _final_b2(s.trace(), "b2_avg") < 1e-3


def test_mn4_path_runs_and_matches(L, ora):
    pr = W.gauss_diag(d=250, M=256, n_steps=1500, var_lo=0.1, var_hi=10.0, x0_scale=1.0)
    s = _gpu(L, pr, seed=0, force_switch_at=600)
    s.run()
    st = s.stats()
    r = _ora(ora, pr, seed=0, force_switch_at=600)
    r.run()
    assert st["integrator"] == 2 == r.integrator
    bg, bo = _final_b2(s.trace(), "b2_avg"), _final_b2(r.trace, "b2_avg")
    assert abs(bg - bo) <= 0.10 * bo, (bg, bo)
    tr = s.trace()
    frozen = [row for row in tr if row["phase"] == 1 and not row["adapting"]]
    assert frozen and abs(np.mean([row["acc"] for row in frozen]) - 0.9) < 0.06


# ------------------------------------------------------------------ shapes / edges
@pytest.mark.parametrize("d,M", [(2, 2), (7, 33), (13, 1000), (64, 257), (101, 300), (300, 100)])
def test_ragged_shapes_first_steps(L, ora, d, M):
    pr = W.gauss_diag(d=d, M=M, n_steps=50, x0_scale=1.0)
    s = _gpu(L, pr, seed=5, fixed_eps=0.05)
    r = _ora(ora, pr, seed=5, fixed_eps=0.05)
    s.step(5)
    r.iterate(5)
    xg = s.sample().double().cpu().numpy()
    xr = r.x()
    rel = np.linalg.norm(xg - xr, axis=1) / np.linalg.norm(xr, axis=1)
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("lpc,cpl", [(4, 4), (8, 4), (8, 8), (16, 4), (16, 8), (32, 4), (32, 8)])
def test_every_launch_shape(L, ora, lpc, cpl):
    d = min(lpc * cpl, 101)
    pr = W.funnel(d=d, M=200, n_steps=40)
    s = _gpu(L, pr, seed=1, lanes_per_chain=lpc, coords_per_lane=cpl, fixed_eps=0.1)
    info = s.launch_info()
    assert info["lanes_per_chain"] == lpc and info["coords_per_lane"] == cpl
    r = _ora(ora, pr, seed=1, fixed_eps=0.1)
    s.step(5)
    r.iterate(5)
    xg = s.sample().double().cpu().numpy()
    rel = np.linalg.norm(xg - r.x(), axis=1) / np.linalg.norm(r.x(), axis=1)
    assert rel.max() <= 1e-5, rel.max()


def test_determinism(L):
    pr = W.banana(d=20, M=1000, n_steps=300)
    outs = []
    for _ in range(2):
        s = _gpu(L, pr, seed=9, force_switch_at=100)
        s.run()
        outs.append((s.sample().cpu().numpy(), [r["eps"] for r in s.trace()]))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_checkpoint_resume_bit_exact(L):
    pr = W.gauss_diag(d=50, M=300, n_steps=400)
    a = _gpu(L, pr, seed=4, force_switch_at=120)
    a.step(60)
    a.step(60)
    b = _gpu(L, pr, seed=4, force_switch_at=120)
    b.step(60)
    blob = b.checkpoint()
    c = _gpu(L, pr, seed=99, force_switch_at=120)  # different seed: the blob carries it
    c.restore(blob)
    c.step(60)
    np.testing.assert_array_equal(a.sample().cpu().numpy(), c.sample().cpu().numpy())
    assert a.stats()["eps"] == c.stats()["eps"]


def test_philox_initial_positions(L, ora):
    pr = W.gauss_diag(d=9, M=40, n_steps=10)
    tg = L.Target.from_problem(pr)
    s = L.Sampler(tg, pr.M, n_total_steps=10)
    s.init(None, x0_scale=2.5, seed=21)
    x = s.sample().double().cpu().numpy()
    ref = 2.5 * ora.normals(21, 0, 40, 0, ora.TAG_X0, 0, 9)
    np.testing.assert_allclose(x, ref, atol=2e-5)


def test_barrier_timeout_is_reported_and_context_recovers(L):
    pr = W.gauss_diag(d=16, M=64, n_steps=20)
    s = _gpu(L, pr, seed=0, barrier_extra_arrivals=1, barrier_timeout_ns=20_000_000)
    st, _ = s.stats_status()
    assert st == 4  # LAPS_ERR_TIMEOUT from the bounded grid barrier
    ok = _gpu(L, pr, seed=0)
    ok.step(3)
    assert ok.stats()["t"] == 3


def test_nonfinite_start_is_reported(L):
    """A NaN initial position would poison every ensemble mean: init reports it."""
    pr = W.gauss_diag(d=10, M=64, n_steps=20)
    x0 = pr.x0.copy()
    x0[5, 3] = np.nan
    pr.x0 = x0
    s = _gpu(L, pr, seed=0)
    st, _ = s.stats_status()
    assert st == 5  # LAPS_ERR_NONFINITE


def test_nonfinite_step_is_reverted(L, ora):
    """A step that overflows (binary32 on the GPU, cosh in the oracle) leaves
    every chain where it was and halves eps."""
    pr = W.gauss_diag(d=10, M=64, n_steps=20)
    s = _gpu(L, pr, seed=0, eps0_coef=1e30)
    x0 = s.sample().cpu().numpy()
    s.step(1)
    st = s.stats()
    assert st["nonfinite_total"] == 64
    np.testing.assert_array_equal(s.sample().cpu().numpy(), x0)
    r = _ora(ora, pr, seed=0, eps0_coef=1e30)
    r.iterate(1)
    assert st["eps"] == pytest.approx(r.trace[1]["eps"], rel=1e-6)


def test_invalid_arguments(L):
    pr = W.banana(d=10, M=8)
    with pytest.raises(L.LapsError):
        L.Target(L.BANANA, 7)          # odd d
    tg = L.Target.from_problem(pr)
    with pytest.raises(L.LapsError):
        L.Sampler(tg, 1)               # M < 2
    s = L.Sampler(tg, 8, n_total_steps=10)
    with pytest.raises(L.LapsError):
        s.step(1)                      # before init
