"""The seeded workloads: shapes, determinism, and the reference moments they
attach (closed forms for the Gaussian, banana and funnel targets; the Laplace
approximation for logistic regression, pinned here by brute-force integration
of a two-dimensional posterior)."""
import numpy as np
import pytest

from paper_2601_16696_gb300 import workloads as W


def test_workloads_deterministic_and_binary32():
    a, b = W.banana(d=20, M=50), W.banana(d=20, M=50)
    np.testing.assert_array_equal(a.x0, b.x0)
    assert np.array_equal(a.x0, a.x0.astype(np.float32).astype(np.float64))
    g = W.gauss_diag(d=10, M=4)
    np.testing.assert_allclose(g.Ex2, 1.0 / g.prec)


def test_batch64_shapes():
    probs = W.batch64(with_big=True)
    assert len(probs) == 65
    d = np.array([p.d for p in probs[:-1]])
    M = np.array([p.M for p in probs[:-1]])
    assert d.min() >= 10 and d.max() <= 2000
    assert set(M) <= {512, 1024, 2048, 4096}
    assert probs[-1].d == 10000 and probs[-1].M == 16384


def _grid_moments(ora, pr, half_width=8.0, n=241):
    """E[w_i^2], Var[w_i^2] of the exact 2-D posterior on a grid around the mode."""
    mu_sq, var_sq = W.logreg_laplace_moments(pr.X, pr.y, pr.prior_var)
    ot = ora.OracleTarget(pr.kind, pr.d, X=pr.X, y=pr.y, prior_var=pr.prior_var)
    # centre and scale from a short Newton solve (the grid must contain the mass)
    w = np.zeros(2)
    for _ in range(30):
        lp, g = ot.logp_grad(w)
        h = 1e-5
        H = np.zeros((2, 2))
        for i in range(2):
            e = np.zeros(2)
            e[i] = h
            H[:, i] = (ot.logp_grad(w + e)[1] - ot.logp_grad(w - e)[1]) / (2 * h)
        w = w - np.linalg.solve(H, g)
    sd = np.sqrt(np.diag(np.linalg.inv(-H)))
    axes = [w[i] + sd[i] * np.linspace(-half_width, half_width, n) for i in range(2)]
    G0, G1 = np.meshgrid(axes[0], axes[1], indexing="ij")
    pts = np.stack([G0.ravel(), G1.ravel()], axis=1)
    lp, _ = ot.logp_grad(pts)
    p = np.exp(lp - lp.max())
    p /= p.sum()
    ex2 = np.array([(p * pts[:, i] ** 2).sum() for i in range(2)])
    ex4 = np.array([(p * pts[:, i] ** 4).sum() for i in range(2)])
    return ex2, ex4 - ex2 ** 2, mu_sq, var_sq


@pytest.mark.parametrize("n_data", [500, 4000])
def test_logreg_laplace_moments_against_integration(ora, n_data):
    pr = W.logreg(n_data=n_data, n_feat=1, M=4, n_steps=1, data_seed=3)
    ex2, var2, lap_ex2, lap_var2 = _grid_moments(ora, pr)
    # the Laplace error in E[w^2] shrinks like 1/sqrt(n) relative to sd(w^2)
    err = np.abs(lap_ex2 - ex2) / np.sqrt(var2)
    assert err.max() < 4.0 / np.sqrt(n_data), (err, ex2, lap_ex2)
    np.testing.assert_allclose(lap_var2, var2, rtol=20.0 / np.sqrt(n_data))


def test_logreg_truth_attached_on_request():
    pr = W.logreg(n_data=300, n_feat=5, M=4, n_steps=1, with_truth=True)
    assert pr.Ex2.shape == (6,) and np.all(pr.Varx2 > 0)
    assert W.logreg(n_data=300, n_feat=5, M=4, n_steps=1).Ex2 is None


def _importance():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_logreg_moments.py")
    spec = importlib.util.spec_from_file_location("make_logreg_moments", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("n_data", [500, 4000])
def test_importance_moments_against_integration(ora, n_data):
    """The importance-sampling estimator behind the stored logistic-regression
    moments reproduces the brute-force integral of a 2-D posterior within its
    own standard error."""
    pr = W.logreg(n_data=n_data, n_feat=1, M=4, n_steps=1, data_seed=3)
    ex2, var2, _, _ = _grid_moments(ora, pr)
    iex2, ivar2, se, ess = _importance().importance_moments(pr.X, pr.y, pr.prior_var, 40000)
    assert ess > 30000
    assert np.all(np.abs(iex2 - ex2) < 5.0 * se), ((iex2 - ex2) / se)
    np.testing.assert_allclose(ivar2, var2, rtol=0.05)


def test_logreg_reference_moments_file():
    """The stored reference moments of the full-size workload: the effective
    sample size and Monte Carlo error it states, and its Laplace column equal
    to the workload's own Laplace moments (the same data)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "logreg_d101_n10000_moments.txt")
    import re
    head = " ".join(line for line in open(path) if line.startswith("#"))
    ess = float(re.search(r"effective sample size (\d+)", head).group(1))
    assert ess > 1e5
    a = np.loadtxt(path)
    assert a.shape == (101, 5) and np.array_equal(a[:, 0], np.arange(101))
    ex2, var2, se, lap = a[:, 1], a[:, 2], a[:, 3], a[:, 4]
    assert np.all(var2 > 0) and np.all(se / np.sqrt(var2) < 0.01)
    pr = W.logreg(with_truth=True)
    np.testing.assert_allclose(lap, pr.Ex2, rtol=1e-12)
    truth = W.logreg_reference_moments()
    np.testing.assert_array_equal(truth[0], ex2)
    np.testing.assert_array_equal(truth[1], var2)
