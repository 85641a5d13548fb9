"""User-supplied targets (LAPS_USER): the caller's log-density and gradient,
written here with torch operations, called by the sampler once per gradient
evaluation of the ensemble on its stream.  The same targets as the built-in
ones, so the oracle's closed forms check the whole path: per-chain positions
within 1e-5 over the first 10 fixed-step steps, final b^2 within 10%.
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


def _gauss_fn(prec):
    p = torch.tensor(prec, dtype=torch.float32, device="cuda")

    def fn(x, logp, grad):
        g = -p * x
        grad.copy_(g)
        logp.copy_(0.5 * (g * x).double().sum(dim=1).float())
    return fn


def _banana_fn(sb):
    inv = 1.0 / (sb * sb)

    def fn(x, logp, grad):
        a, b = x[:, 0::2], x[:, 1::2]
        r = b - a * a
        grad[:, 0::2] = -a + 2.0 * a * r * inv
        grad[:, 1::2] = -r * inv
        logp.copy_((-0.5 * a * a - 0.5 * r * r * inv).double().sum(dim=1).float())
    return fn


def _rel(a, b):
    return float((np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max())


@pytest.mark.parametrize("pr_fn,eps", [
    (lambda: W.gauss_diag(d=100, M=512, n_steps=50), 0.05),
    (lambda: W.banana(d=100, M=1024, n_steps=50), 0.01),
    (lambda: W.gauss_diag(d=37, M=65, n_steps=50, x0_scale=1.0), 0.05),
])
def test_user_target_first_ten_steps(L, ora, pr_fn, eps):
    pr = pr_fn()
    fn = _gauss_fn(pr.prec) if pr.kind == W.GAUSS_DIAG else _banana_fn(pr.banana_sb)
    tg = L.Target.from_callable(pr.d, fn)
    x0 = torch.tensor(pr.x0, dtype=torch.float32, device="cuda")
    lp, g = tg.logp_grad(x0)
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec, banana_sb=pr.banana_sb)
    lp_o, g_o = ot.logp_grad(pr.x0)
    np.testing.assert_allclose(g.double().cpu().numpy(), g_o, rtol=1e-6, atol=1e-6 * np.abs(g_o).max())
    np.testing.assert_allclose(lp.double().cpu().numpy(), lp_o, rtol=1e-5)
    s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, fixed_eps=eps)
    s.init(x0, seed=3)
    r = ora.OracleLAPS(ot, pr.x0, seed=3, n_total_steps=pr.n_steps, fixed_eps=eps)
    for k in range(10):
        s.step(1)
        r.iterate(1)
        rel = _rel(s.sample().double().cpu().numpy(), r.x())
        assert rel <= 1e-5, (k + 1, rel)


def test_user_target_whole_run(L, ora):
    """The Gaussian of the headline's first configuration through the switch and
    the adjusted phase (MN2 proposals: the callback runs twice per step)."""
    pr = W.gauss_diag()
    tg = L.Target.from_callable(pr.d, _gauss_fn(pr.prec))
    s = L.Sampler(tg, pr.M, n_total_steps=pr.n_steps, force_switch_at=400)
    s.set_truth(pr.Ex2, pr.Varx2)
    s.init(torch.tensor(pr.x0, dtype=torch.float32, device="cuda"), seed=0)
    s.run()
    st = s.stats()
    ot = ora.OracleTarget(pr.kind, pr.d, prec=pr.prec)
    r = ora.OracleLAPS(ot, pr.x0, seed=0, truth=(pr.Ex2, pr.Varx2), n_total_steps=pr.n_steps,
                       force_switch_at=400)
    r.run()
    assert st["t"] == r.t and st["phase"] == r.phase == 1 and st["t_switch"] == r.t_switch
    tail = lambda tr: float(np.mean([x["b2_avg"] for x in
                                     [y for y in tr[1:] if y["phase"] == 1][-300:]]))
    bg, bo = tail(s.trace()), tail(r.trace)
    assert abs(bg - bo) <= 0.10 * bo, (bg, bo)


def test_user_target_error_is_reported(L):
    def bad(x, logp, grad):
        raise ValueError("no density here")

    tg = L.Target.from_callable(8, bad)
    with pytest.raises(L.LapsError, match="user_fn"):
        tg.logp_grad(torch.zeros(4, 8, device="cuda"))
    s = L.Sampler(tg, 16, n_total_steps=10)
    with pytest.raises(L.LapsError, match="user_fn"):
        s.init(torch.zeros(16, 8, device="cuda"), seed=0)
    assert tg._errors and isinstance(tg._errors[0], ValueError)
