"""GPU parity of the paper's own switch rule (Sec. 4, Eq. "relative
fluctuations"; the exit test of Alg. 1's unadjusted loop) firing by itself.

The window statistic delta_i = sqrt(Var_window[E x_i^2]) / mean_window[E x_i^2]
over the last T = ceil(0.2 n_total_steps) steps, and the switch at the first
full-window step where max_i delta_i < switch_tol, are computed by the device
window ring and slice owners (register-resident, batched and streamed paths);
the oracle recomputes them from its stored window every step.  Both runs start from the same ensemble and draw the same
Philox stream, and no run here forces the switch.

- With the step size held fixed (the fixed-step comparison of App. A), the
  chains of a Gaussian target stay coupled to the oracle's for the whole
  unadjusted phase (the common noise contracts them), so max_i delta_i is
  compared row by row at 1e-4 relative and the switch step must be equal.
- With the paper's step-size controller, binary32 rounding of the state moves
  the first controller updates by ~1e-4 relative (u0 is parallel to g0, so the
  first measured EEVPD is ~1e-8), and the window's early rows inherit that;
  the per-row bar is three times the divergence between the oracle and the
  oracle with its state rounded to binary32 (computed here from the oracle
  alone; its largest size within ten rows), never below 1e-4.  The switch
  step must still be equal.
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


class _BatchRun:
    """One problem in the batched path (problem id 0), with the single-problem
    sampler's run / stats / trace calls."""

    def __init__(self, L, pr, seed, **cfg):
        self.b = L.Batch([pr], n_total_steps=pr.n_steps, **cfg)
        self.b.set_truth(0, pr.Ex2, pr.Varx2)
        self.b.init(seed=seed)

    def run(self):
        self.b.run(iters_per_launch=64)

    def stats(self):
        return self.b.stats(0)

    def trace(self):
        return self.b.trace(0)


def _dense(pr):
    """The same Gaussian given by its precision matrix (the streamed path's
    dense-precision target, GAUSS_DENSE with dense_streamed)."""
    pr.kind = W.GAUSS_DENSE
    pr.prec = np.diag(pr.prec)
    return pr


def _pair(L, ora, pr, seed, path="resident", **cfg):
    if path == "streamed":
        pr = _dense(pr)
        cfg = dict(cfg, dense_streamed=1)
    if path == "batch":
        s = _BatchRun(L, pr, seed, **cfg)
    else:
        tg = L.Target.from_problem(pr)
        s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
        s.set_truth(pr.Ex2, pr.Varx2)
        s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=seed)
        s._tg = tg
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec)
    cfg.pop("dense_streamed", None)
    r = ora.OracleLAPS(ot, pr.x0, seed=seed, truth=(pr.Ex2, pr.Varx2), n_total_steps=pr.n_steps,
                       **cfg)
    return s, r


def _window_rows(trace, T, t_switch):
    """max_i delta_i of every unadjusted iteration with a full window, keyed by
    t (the GPU labels the row of the switching iteration with the new phase,
    the oracle with the old one; both record that iteration's delta there)."""
    return {q["t"]: q["max_delta"] for q in trace if T <= q["t"] <= t_switch}


def _tail_b2(trace, key):
    rows = [q for q in trace[1:] if q["phase"] == trace[-1]["phase"]]
    n = max(1, len(rows) // 2)
    return float(np.mean([q[key] for q in rows[-n:]]))


D10 = dict(d=10, n_steps=1000, x0_scale=1.0, var_lo=0.1, var_hi=10.0)
# (path, problem, seed, config).  The register-resident kernel holds at most
# ~19k chains of d = 10 at once, where the statistic's finite-M floor
# sqrt(2/M) ~ 0.011 lies above the paper's 0.01: it runs d = 10, M = 16384 at
# threshold 0.02, and d = 100, M = 4096 (variances 1e-2 .. 1e2, floor ~ 0.02)
# at 0.05.  The batched path holds any M: d = 10, M = 65536 at the paper's 0.01
# (floor ~ 0.0055).
FIXED = {
    "resident_d10_M16384": ("resident", dict(M=16384, **D10), 0, dict(fixed_eps=0.6, switch_tol=0.02)),
    "resident_d100_M4096": ("resident", dict(d=100, M=4096, n_steps=2000), 0,
                            dict(fixed_eps=0.3, switch_tol=0.05)),
    "batch_d10_M65536": ("batch", dict(M=65536, **D10), 0, dict(fixed_eps=0.6)),
    # the streamed path's finalise kernel (the same Gaussian as a dense precision matrix)
    "streamed_d10_M65536": ("streamed", dict(M=65536, **D10), 0, dict(fixed_eps=0.6)),
}
# adaptive runs: seeds whose switch step the oracle and its binary32 variant
# agree on, with max delta more than 1% away from the threshold on both sides.
# After the switch the adaptive runs decorrelate from the oracle's; their final
# b^2 (~1/M) then differs by finite-M noise: at M = 16384 the tail b^2 is
# compared as a mean over five seeds (the seed spread there is ~15%).
ADAPTIVE = {
    "resident_d10_M16384": ("resident", dict(M=16384, **D10), 1, dict(switch_tol=0.02), (1, 2, 3, 4, 5)),
    "batch_d10_M65536": ("batch", dict(M=65536, **D10), 0, {}, (0,)),
}


@pytest.mark.parametrize("name", sorted(FIXED))
def test_switch_rule_fires_fixed_step(L, ora, name):
    path, kw, seed, cfg = FIXED[name]
    pr = W.gauss_diag(**kw)
    s, r = _pair(L, ora, pr, seed, path, **cfg)
    s.run()
    r.run()
    st = s.stats()
    T = r.window_T
    tol = cfg.get("switch_tol", 0.01)
    assert r.t_switch > T and r.phase == 1  # the rule fired, after the window filled
    assert st["t_switch"] == r.t_switch, (st["t_switch"], r.t_switch)
    assert st["t"] == r.t and st["phase"] == 1 and st["integrator"] == r.integrator
    rg, ro = _window_rows(s.trace(), T, r.t_switch), _window_rows(r.trace, T, r.t_switch)
    assert sorted(rg) == sorted(ro) and len(ro) == r.t_switch - T + 1
    worst = max(abs(rg[t] - ro[t]) / ro[t] for t in ro)
    print("%s: %d window rows, max_delta worst rel %.2e, t_switch %d" % (name, len(ro), worst, r.t_switch))
    assert worst <= 1e-4, worst
    # the last row is the one that fired, the one before it did not
    assert ro[r.t_switch] < tol <= ro[r.t_switch - 1]
    assert rg[r.t_switch] < tol <= rg[r.t_switch - 1]
    bg, bo = _tail_b2(s.trace(), "b2_avg"), _tail_b2(r.trace, "b2_avg")
    assert abs(bg - bo) <= 0.10 * bo, (bg, bo)


@pytest.mark.parametrize("name", sorted(ADAPTIVE))
def test_switch_rule_fires_adaptive(L, ora, name):
    """The step-size controller on (Sec. 3.1)."""
    path, kw, seed, cfg, b2_seeds = ADAPTIVE[name]
    pr = W.gauss_diag(**kw)
    s, r = _pair(L, ora, pr, seed, path, **cfg)
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec)
    r32 = ora.OracleLAPS(ot, pr.x0, seed=seed, truth=(pr.Ex2, pr.Varx2), n_total_steps=pr.n_steps,
                         round_state_f32=1, **cfg)
    s.run()
    r.run()
    r32.iterate(r.t_switch)
    st = s.stats()
    T = r.window_T
    assert r.t_switch > T and r.phase == 1
    assert st["t_switch"] == r.t_switch, (st["t_switch"], r.t_switch)
    rg, ro = _window_rows(s.trace(), T, r.t_switch), _window_rows(r.trace, T, r.t_switch)
    r3 = _window_rows(r32.trace, T, r.t_switch)
    assert sorted(rg) == sorted(ro) == sorted(r3)
    # the binary32 divergence changes sign along the window rows; the bar takes
    # its largest size within ten rows of t
    div = {t: abs(r3[t] - ro[t]) / ro[t] for t in ro}
    worst_ratio, worst = 0.0, 0.0
    for t in ro:
        near = max(div[q] for q in range(t - 10, t + 11) if q in div)
        bar = max(1e-4, 3.0 * near)
        rel = abs(rg[t] - ro[t]) / ro[t]
        worst, worst_ratio = max(worst, rel), max(worst_ratio, rel / bar)
        assert rel <= bar, (t, rel, bar)
    print("%s adaptive: %d window rows, max_delta worst rel %.2e, worst rel/bar %.2f, t_switch %d"
          % (name, len(ro), worst, worst_ratio, r.t_switch))
    assert st["t"] == r.t and st["phase"] == 1 and st["integrator"] == r.integrator
    bgs, bos = [], []
    for sd in b2_seeds:
        if sd != seed:
            s, r = _pair(L, ora, pr, sd, path, **cfg)
            s.run()
            r.run()
        bgs.append(_tail_b2(s.trace(), "b2_avg"))
        bos.append(_tail_b2(r.trace, "b2_avg"))
    bg, bo = float(np.mean(bgs)), float(np.mean(bos))
    print("%s adaptive: tail b^2_avg over %d seed(s): GPU %.4g, oracle %.4g" % (name, len(bgs), bg, bo))
    assert abs(bg - bo) <= 0.10 * bo, (bgs, bos)
