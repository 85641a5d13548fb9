"""GPU parity of the paper's ablation settings (Table "mams", Fig. "stepsize",
Fig. "chains"): whole runs in the configurations bench.py --ablations times,
against the FP64 oracle.  Bar: the b^2 tail mean of the final phase within 10%
(oracle seed-to-seed spread of these means <= 5%), equal switch step.

- MAMS only: the switch forced after the first step, so the adjusted phase
  runs alone from a preconditioner of the first ensemble;
- a fixed step size throughout the unadjusted phase;
- a small ensemble (M = 64), below the paper's working range.
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


def _tail(trace, key):
    rows = [r for r in trace[1:] if r["phase"] == trace[-1]["phase"]]
    return float(np.mean([r[key] for r in rows[len(rows) // 2:]]))


@pytest.mark.parametrize("name,pr_fn,key,cfg", [
    ("mams_only_gauss", lambda: W.gauss_diag(), "b2_avg", {"force_switch_at": 1}),
    ("mams_only_banana", lambda: W.banana(M=1024, n_steps=1500), "b2_max", {"force_switch_at": 1}),
    ("small_M", lambda: W.gauss_diag(M=64), "b2_avg", {}),
    ("fixed_step", lambda: W.gauss_diag(), "b2_avg", {"fixed_eps": 0.3, "adjusted": 0}),
])
def test_ablation_run_matches_oracle(L, ora, name, pr_fn, key, cfg):
    pr = pr_fn()
    tg = L.Target.from_problem(pr)
    s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, **cfg)
    s.set_truth(pr.Ex2, pr.Varx2)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=0)
    s.run()
    st = s.stats()
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb, funnel_sv=pr.funnel_sv)
    r = ora.OracleLAPS(ot, pr.x0, seed=0, truth=(pr.Ex2, pr.Varx2), n_total_steps=pr.n_steps, **cfg)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase and st["t_switch"] == r.t_switch
    bg, bo = _tail(s.trace(), key), _tail(r.trace, key)
    assert abs(bg - bo) <= 0.10 * bo, (name, bg, bo)
    if cfg.get("force_switch_at"):
        ag = np.mean([x["acc"] for x in s.trace()[-50:]])
        ao = np.mean([x["acc"] for x in r.trace[-50:]])
        assert abs(ag - ao) <= 0.1, (ag, ao)
