"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than its own
formula: closed forms, exact samples of the target, an independent numerical
ODE solution, convergence orders, reversibility, brute-force histograms.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2601_16696_gb300 import workloads as W


# ----------------------------------------------------------------- random stream
def test_philox_uniform_statistics(ora):
    n = 1 << 18
    ctrs = np.zeros((n, 4), dtype=np.uint32)
    ctrs[:, 0] = np.arange(n)
    ctrs[:, 1] = 7
    ctrs[:, 2] = 3
    ctrs[:, 3] = 1
    out = ora.philox(ctrs, (0x12345678, 0x9ABCDEF0))
    u = ((out.astype(np.float64) // 512) + 0.5) / 8388608.0
    u = u.ravel()
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.002
    assert stats.kstest(u[:200000], "uniform").pvalue > 1e-4
    bits = np.unpackbits(out.view(np.uint8)).reshape(-1, 32 * 4).mean(0)
    assert np.all(np.abs(bits - 0.5) < 6 * 0.5 / math.sqrt(n))
    c = np.corrcoef(out[:, 0].astype(np.float64), out[:, 1].astype(np.float64))[0, 1]
    assert abs(c) < 0.01
    # a bijection on 128-bit counters: no repeated outputs
    assert np.unique(out.view(np.dtype((np.void, 16)))).size == n


def test_philox_known_answers(ora):
    """Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC11, 2011) bit for bit on
    the known-answer vectors its authors publish with the generator: the zero
    counter and key, the all-ones counter and key, and the counter and key made
    of the leading hexadecimal digits of pi.  The statistical pins above pass for
    any good mixer; a wrong multiplier, Weyl constant or round count fails here."""
    cases = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in cases:
        got = ora.philox(np.array([ctr], dtype=np.uint32), np.array(key, dtype=np.uint32))[0]
        assert tuple(int(v) for v in got) == want, ([hex(v) for v in got], ctr, key)


def test_philox_avalanche(ora):
    """Flipping one counter bit flips about half of the 128 output bits."""
    rng = np.random.default_rng(1)
    n = 4096
    base = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = (11, 22)
    o0 = ora.philox(base, key)
    for word in range(4):
        for bit in (0, 13, 31):
            flip = base.copy()
            flip[:, word] ^= np.uint32(1 << bit)
            o1 = ora.philox(flip, key)
            hd = np.unpackbits((o0 ^ o1).view(np.uint8)).reshape(n, -1).sum(1)
            assert abs(hd.mean() - 64) < 0.5, (word, bit, hd.mean())
    # the key matters as well
    o2 = ora.philox(base, (12, 22))
    hd = np.unpackbits((o0 ^ o2).view(np.uint8)).reshape(n, -1).sum(1)
    assert abs(hd.mean() - 64) < 0.5


def test_uniform_mapping_exact(ora):
    assert ora.uniform(0) == 2.0 ** -24
    assert ora.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(2)
    for r in rng.integers(0, 2**32, size=1000):
        v = ora.uniform(int(r))
        assert 0.0 < v < 1.0 and float(np.float32(v)) == v  # exact in binary32


def test_normals_statistics(ora):
    z = ora.normals(seed=5, m0=0, nm=2000, t=17, tag=ora.TAG_O1, pid=0, d=128).ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 0.01
    assert abs(stats.kurtosis(z)) < 0.05
    assert stats.kstest(z[:100000], "norm").pvalue > 1e-4
    # different streams (tag, step, chain) are uncorrelated
    z2 = ora.normals(seed=5, m0=0, nm=2000, t=17, tag=ora.TAG_O2, pid=0, d=128).ravel()
    z3 = ora.normals(seed=5, m0=0, nm=2000, t=18, tag=ora.TAG_O1, pid=0, d=128).ravel()
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01 and abs(np.corrcoef(z, z3)[0, 1]) < 0.01
    # the padding convention: coordinate i takes block i // 4, lane i % 4
    z5 = ora.normals(seed=5, m0=3, nm=1, t=17, tag=1, pid=0, d=5)
    z8 = ora.normals(seed=5, m0=3, nm=1, t=17, tag=1, pid=0, d=8)
    np.testing.assert_array_equal(z5[0], z8[0, :5])


# ----------------------------------------------------------------- targets
def _targets(ora):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((50, 4))
    y = (rng.random(50) < 0.5).astype(float)
    return [
        ora.OracleTarget(ora.GAUSS_DIAG, 7, prec=rng.uniform(0.1, 10, 7)),
        ora.OracleTarget(ora.BANANA, 6, banana_sb=0.1),
        ora.OracleTarget(ora.FUNNEL, 5, funnel_sv=3.0),
        ora.OracleTarget(ora.LOGREG, 4, X=X, y=y, prior_var=1.0),
        ora.OracleTarget(ora.GAUSS_DENSE, 5, prec=_spd(rng, 5)),
    ]


def _spd(rng, d):
    A = rng.standard_normal((d, d))
    return A @ A.T / d + 0.1 * np.eye(d)


def test_gradients_central_differences(ora):
    rng = np.random.default_rng(4)
    for tg in _targets(ora):
        x = rng.standard_normal(tg.d) * 0.7
        lp, g = tg.logp_grad(x)
        h = 1e-5
        fd = np.empty(tg.d)
        for i in range(tg.d):
            e = np.zeros(tg.d)
            e[i] = h
            fd[i] = (tg.logp_grad(x + e)[0] - tg.logp_grad(x - e)[0]) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(g).max()))


def test_logreg_closed_form_at_zero(ora):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((30, 3))
    y = (rng.random(30) < 0.3).astype(float)
    tg = ora.OracleTarget(ora.LOGREG, 3, X=X, y=y)
    lp, g = tg.logp_grad(np.zeros(3))
    assert lp == pytest.approx(-30 * math.log(2.0), rel=1e-14)
    np.testing.assert_allclose(g, X.T @ (y - 0.5), rtol=1e-13, atol=1e-13)


def _score_identities(tg, xs):
    """E_p[grad log p] = 0 and V_ii = -Cov(x_i, d_i log p) = 1 under exact samples."""
    _, g = tg.logp_grad(xs)
    M = xs.shape[0]
    gm = g.mean(0)
    se_g = g.std(0) / math.sqrt(M)
    assert np.all(np.abs(gm) < 5 * se_g + 1e-12), (gm, se_g)
    prod = -(xs - xs.mean(0)) * g
    V = prod.mean(0)
    se_v = prod.std(0) / math.sqrt(M)
    assert np.all(np.abs(V - 1) < 5 * se_v), (V, se_v)


def test_banana_score_identities_exact_samples(ora):
    rng = np.random.default_rng(6)
    M, s = 400000, 0.1
    a = rng.standard_normal(M)
    b = a * a + s * rng.standard_normal(M)
    xs = np.stack([a, b, b * 0 + rng.standard_normal(M), 0 * b], 1)
    xs[:, 3] = xs[:, 2] ** 2 + s * rng.standard_normal(M)
    _score_identities(ora.OracleTarget(ora.BANANA, 4, banana_sb=s), xs)


def test_funnel_score_identities_exact_samples(ora):
    rng = np.random.default_rng(7)
    M, sv = 400000, 3.0
    v = sv * rng.standard_normal(M)
    x = rng.standard_normal((M, 3)) * np.exp(v / 2)[:, None]
    _score_identities(ora.OracleTarget(ora.FUNNEL, 4, funnel_sv=sv), np.column_stack([v, x]))


def test_dense_gauss_score_identities_exact_samples(ora):
    """Exact draws of the rotated ill-conditioned Gaussian (the workload's own
    precision matrix, d = 100): E[grad log p] = 0 and Cov(x, grad log p) = -I,
    the whole matrix (a dropped or misplaced entry of P x shows off the
    diagonal); and log p's value at x = P^-1 b is -1/2 b^T P^-1 b."""
    pr = W.icg(d=100, M=8)
    tg = ora.OracleTarget(ora.GAUSS_DENSE, pr.d, prec=pr.prec)
    rng = np.random.default_rng(7)
    Lc = np.linalg.cholesky(pr.extra["cov"])
    M = 20000
    X = rng.standard_normal((M, pr.d)) @ Lc.T
    _, G = tg.logp_grad(X)
    # normalise each coordinate pair by its natural scale sqrt(E x_i^2 E g_j^2)
    sx = np.sqrt(np.mean(X * X, axis=0))
    sg = np.sqrt(np.mean(G * G, axis=0))
    np.testing.assert_allclose(G.mean(axis=0) / sg, 0.0, atol=5.0 / np.sqrt(M))
    V = (X - X.mean(0)).T @ (G - G.mean(0)) / M
    np.testing.assert_allclose(V / np.outer(sx, sg), -np.eye(pr.d) / np.outer(sx, sg),
                               atol=6.0 / np.sqrt(M))
    b = rng.standard_normal(pr.d)
    x = np.linalg.solve(pr.prec, b)
    lp, g = tg.logp_grad(x)
    np.testing.assert_allclose(g, -b, rtol=1e-8, atol=1e-8)
    assert lp == pytest.approx(-0.5 * b @ x, rel=1e-10)


def test_icg_workload_condition_and_truth():
    """The stand-in for the paper's ill-conditioned Gaussian: d = 100, condition
    number about 1e5, a dense rotation (every precision row has many
    non-negligible entries), and truths from the covariance of the rounded P."""
    pr = W.icg()
    ev = np.linalg.eigvalsh(pr.prec)
    assert 5e4 < ev.max() / ev.min() < 2e5
    off = np.abs(pr.prec - np.diag(np.diag(pr.prec)))
    assert (off > 1e-3 * np.abs(pr.prec).max()).sum(axis=1).min() > 50
    np.testing.assert_allclose(pr.Ex2, np.diag(np.linalg.inv(pr.prec)), rtol=1e-9)
    assert np.array_equal(pr.prec, pr.prec.T)
    assert np.array_equal(pr.prec, pr.prec.astype(np.float32).astype(np.float64))


def test_gauss_truth_moments_match_workload():
    """The closed-form truths of the workloads agree with Monte Carlo draws."""
    rng = np.random.default_rng(8)
    pb = W.banana(d=2, M=4)
    a = rng.standard_normal(2_000_000)
    b = a * a + 0.1 * rng.standard_normal(a.size)
    np.testing.assert_allclose([np.mean(a * a), np.mean(b * b)], pb.Ex2, rtol=0.01)
    np.testing.assert_allclose([np.var(a * a), np.var(b * b)], pb.Varx2, rtol=0.08)
    pf = W.funnel(d=2, M=4, sv=1.0)
    v = rng.standard_normal(2_000_000)
    x = rng.standard_normal(v.size) * np.exp(v / 2)
    np.testing.assert_allclose([np.mean(v * v), np.mean(x * x)], pf.Ex2, rtol=0.01)
    np.testing.assert_allclose([np.var(v * v), np.var(x * x)], pf.Varx2, rtol=0.1)


# ----------------------------------------------------------------- maps
def test_O_update_norm_and_noise_scale(ora):
    rng = np.random.default_rng(9)
    d = 20000
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    z = rng.standard_normal(d) / math.sqrt(d)   # Z ~ N(0, I/d): std 1/sqrt(d)
    L, eps = 1.0, 0.5108                        # c1 = exp(-eps/L) ~ 0.6
    v = u.copy()
    ora.O(eps, L, z, v)
    assert abs(np.linalg.norm(v) - 1) < 1e-14
    assert abs(u @ v - math.exp(-eps / L)) < 0.02
    w = u.copy()
    ora.O(0.0, L, z, w)                          # no refresh at eps = 0
    np.testing.assert_allclose(w, u, atol=1e-15)


def _rk4_velocity(g, u, T, n):
    """du/dt = (I - u u^T) g / (d-1), K' = g . u, by classical RK4."""
    d = g.size

    def f(s):
        uu = s[:d]
        return np.concatenate([(g - uu * (uu @ g)) / (d - 1), [g @ uu]])

    s = np.concatenate([u, [0.0]])
    h = T / n
    for _ in range(n):
        k1 = f(s)
        k2 = f(s + 0.5 * h * k1)
        k3 = f(s + 0.5 * h * k2)
        k4 = f(s + h * k3)
        s = s + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return s[:d], s[d]


@pytest.mark.parametrize("scale", [0.3, 3.0, 30.0])
def test_B_update_matches_riccati_ode(ora, scale):
    rng = np.random.default_rng(10)
    d = 6
    g = scale * rng.standard_normal(d)
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    eps = 0.7
    v = u.copy()
    dk = ora.B(eps, g, v)
    v_ref, k_ref = _rk4_velocity(g, u, eps, 4000)
    np.testing.assert_allclose(v, v_ref, atol=1e-9)
    assert dk == pytest.approx(k_ref, abs=1e-8 * max(1, abs(k_ref)))
    assert abs(np.linalg.norm(v) - 1) < 1e-13


def test_B_update_zero_gradient(ora):
    u = np.array([0.6, 0.8, 0.0])
    v = u.copy()
    assert ora.B(1.0, np.zeros(3), v) == 0.0
    np.testing.assert_array_equal(v, u)


# ----------------------------------------------------------------- integrators
@pytest.mark.parametrize("integ", [0, 1, 2])
def test_integrator_coefficients(ora, integ):
    b, a = ora.coefs(integ)
    assert b.sum() == pytest.approx(1.0, abs=1e-12)
    assert a.sum() == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(b, b[::-1], atol=0)
    np.testing.assert_allclose(a, a[::-1], atol=0)
    assert len(a) == {0: 1, 1: 2, 2: 5}[integ]   # gradients per step, Table "integrators"


def _flow(ora, tg, integ, x0, u0, T, n):
    x, u = x0.copy(), u0.copy()
    lp, g = tg.logp_grad(x)
    dl = 0.0
    for _ in range(n):
        de, lp = ora.Phi(tg, integ, T / n, x, u, g, lp)
        dl += de
    return x, u, dl


@pytest.mark.parametrize("integ,order", [(0, 2), (1, 2), (2, 4)])
def test_integrator_order_and_energy(ora, integ, order):
    tg = ora.OracleTarget(ora.BANANA, 4, banana_sb=0.7)
    rng = np.random.default_rng(11)
    x0 = rng.standard_normal(4) * 0.5
    u0 = rng.standard_normal(4)
    u0 /= np.linalg.norm(u0)
    T = 1.0
    xr, ur, _ = _flow(ora, tg, 2, x0, u0, T, 4000)
    ns = [20, 40, 80] if order == 2 else [10, 20, 40]
    errs, energies = [], []
    for n in ns:
        x, u, dl = _flow(ora, tg, integ, x0, u0, T, n)
        errs.append(np.linalg.norm(x - xr) + np.linalg.norm(u - ur))
        energies.append(abs(dl))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - order) < 0.35), slopes
    # the energy error of the exact flow is zero: Delta vanishes at the same order
    e_slopes = np.log2(np.array(energies[:-1]) / np.array(energies[1:]))
    assert np.all(e_slopes > order - 0.5), e_slopes


@pytest.mark.parametrize("integ", [0, 1, 2])
def test_reversibility(ora, integ):
    tg = ora.OracleTarget(ora.FUNNEL, 5, funnel_sv=3.0)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(5) * 0.8
    u = rng.standard_normal(5)
    u /= np.linalg.norm(u)
    x0, u0 = x.copy(), u.copy()
    lp, g = tg.logp_grad(x)
    d1 = 0.0
    for _ in range(7):
        de, lp = ora.Phi(tg, integ, 0.2, x, u, g, lp)
        d1 += de
    u *= -1
    d2 = 0.0
    for _ in range(7):
        de, lp = ora.Phi(tg, integ, 0.2, x, u, g, lp)
        d2 += de
    np.testing.assert_allclose(x, x0, atol=1e-12)
    np.testing.assert_allclose(-u, u0, atol=1e-12)
    assert d2 == pytest.approx(-d1, abs=1e-11)


# ----------------------------------------------------------------- ensemble estimators
def test_F_closed_form(ora):
    assert ora.F(0.0) == 0.0
    assert ora.F(1.0) == pytest.approx(1.0, rel=1e-15)
    assert ora.F(0.25) == pytest.approx(2.0 / 9.0, rel=1e-15)
    Ds = np.logspace(-8, 3, 200)
    Fs = np.array([ora.F(D) for D in Ds])
    assert np.all(np.diff(Fs) > 0)
    assert ora.F(1e-10) / (4 * 1e-15) == pytest.approx(1.0, rel=1e-4)


def test_dtilde_diag_gaussian_closed_form(ora):
    """App. B.2, Eq. D2: D~_diag(N, N') = (1/d) sum (1 - S'_ii / S_ii)^2."""
    rng = np.random.default_rng(13)
    S = np.array([1.0, 2.0, 0.5, 3.0, 1.0])
    Sp = np.array([1.2, 1.5, 0.5, 4.0, 0.8])
    M = 400000
    X = rng.standard_normal((M, 5)) * np.sqrt(Sp) + 2.5   # a shifted ensemble
    G = -X / S                                             # target N(0, diag S)
    want = np.mean((1 - Sp / S) ** 2)
    got = ora.dtilde_diag(X, G + 0.0)
    # V_ii is centred in x, so only the covariance enters; the shift of the
    # ensemble adds -2.5/S to every gradient but not to V
    G2 = -(X - 2.5) / S
    got2 = ora.dtilde_diag(X, G2)
    assert got2 == pytest.approx(want, abs=0.004)
    assert got == pytest.approx(got2, rel=1e-9)
    # zero exactly when the ensemble is the target (up to sampling error)
    X3 = rng.standard_normal((M, 5)) * np.sqrt(S)
    assert ora.dtilde_diag(X3, -X3 / S) < 2e-4


def test_L_two_chains(ora):
    a = np.array([1.0, -2.0, 0.5])
    b = np.array([3.0, 0.0, 0.5])
    want = 2.0 * math.sqrt(np.sum((a - b) ** 2) / 4)
    assert ora.L_of(np.stack([a, b]), alpha=2.0) == pytest.approx(want, rel=1e-15)


def test_rel_fluct_closed_forms(ora):
    T = 37
    assert ora.rel_fluct(np.full(T, 4.0)) == 0.0
    assert ora.rel_fluct(np.full(T, 4.2)) < 1e-15
    a = 0.3
    alt = 1 + a * (-1.0) ** np.arange(T + 1)[:T]
    mu = alt.mean()
    # mean of an odd-length alternating series is 1 + a/T
    assert mu == pytest.approx(1 + a / T)
    ramp = 5.0 + np.arange(T)
    want = math.sqrt(T * (T + 1) / 12.0) / (5.0 + (T - 1) / 2)
    assert ora.rel_fluct(ramp) == pytest.approx(want, rel=1e-12)
    T2 = 40
    alt2 = 1 + a * (-1.0) ** np.arange(T2)
    assert ora.rel_fluct(alt2) == pytest.approx(a * math.sqrt(T2 / (T2 - 1)), rel=1e-12)


@pytest.mark.parametrize("eps0", [0.01, 50.0])
def test_bisection_brackets_and_converges(ora, eps0):
    root = math.log(2.0)                   # a(eps) = exp(-eps), a* = 1/2
    eps, lo, hi = eps0, 0.0, 0.0
    seen_bracket = False
    for _ in range(60):
        eps, lo, hi = ora.bisect(eps, math.exp(-eps), 0.5, lo, hi)
        if lo > 0 and hi > 0:
            seen_bracket = True
            assert lo <= root <= hi
    assert seen_bracket and abs(eps - root) < 1e-9


# ----------------------------------------------------------------- MAMS exactness
def _banana2(rng, M, s):
    a = rng.standard_normal(M)
    return np.ascontiguousarray(np.stack([a, a * a + s * rng.standard_normal(M)], 1))


def _exactness_stats(before, after):
    """KS of the x1 marginal vs N(0,1) and chi^2 symmetry of the (x1, x1') histogram."""
    ks = stats.kstest(after[:, 0], "norm").pvalue
    edges = np.linspace(-2.5, 2.5, 11)
    H, _, _ = np.histogram2d(before[:, 0], after[:, 0], bins=[edges, edges])
    iu = np.triu_indices(H.shape[0], 1)
    num = (H[iu] - H.T[iu]) ** 2
    den = H[iu] + H.T[iu]
    ok = den > 0
    chi2 = np.sum(num[ok] / den[ok])
    sym = stats.chi2.sf(chi2, ok.sum())
    mb = abs(after[:, 1].mean() - 1.0) / (after[:, 1].std() / math.sqrt(after.shape[0]))
    return ks, sym, mb


def test_mams_detailed_balance_histogram(ora):
    """App. F: the adjusted kernel leaves p invariant and is reversible."""
    s = 0.5
    tg = ora.OracleTarget(ora.BANANA, 2, banana_sb=s)
    rng = np.random.default_rng(14)
    X = _banana2(rng, 200000, s)
    before = X.copy()
    acc_p, acc = ora.mams_batch(tg, ora.MN2, eps=0.35, L=1.25 * 15 * 0.35, n_steps=15, seed=3,
                                X=X)
    assert 0.3 < acc.mean() < 0.9
    ks, sym, mb = _exactness_stats(before, X)
    assert ks > 1e-3 and sym > 1e-3 and mb < 4.5, (ks, sym, mb, acc.mean())
    # the acceptance statistic averages to the accepted fraction
    assert abs(acc_p.mean() - acc.mean()) < 0.01


@pytest.mark.parametrize("mode", [1, 2])
def test_mams_histogram_has_power(ora, mode):
    """Planted mistakes in the acceptance rule (accept all / flipped energy
    sign) must be caught by the same statistics."""
    s = 0.5
    tg = ora.OracleTarget(ora.BANANA, 2, banana_sb=s)
    rng = np.random.default_rng(14)
    X = _banana2(rng, 200000, s)
    before = X.copy()
    ora.mams_batch(tg, ora.MN2, eps=0.35, L=1.25 * 15 * 0.35, n_steps=15, seed=3, X=X,
                   mh_mode=mode)
    ks, sym, mb = _exactness_stats(before, X)
    assert min(ks, sym) < 1e-6 or mb > 8, (ks, sym, mb)


def test_mams_stationarity_gaussian_mn4(ora):
    rng = np.random.default_rng(15)
    d = 8
    var = np.logspace(-1, 1, d)
    tg = ora.OracleTarget(ora.GAUSS_DIAG, d, prec=1 / var)
    M = 100000
    X = np.ascontiguousarray(rng.standard_normal((M, d)) * np.sqrt(var))
    for p in range(3):
        ora.mams_batch(tg, ora.MN4, eps=0.6, L=1.25 * 15 * 0.6, n_steps=15, seed=4, X=X, p=p,
                       t0=15 * p)
    ex2 = (X * X).mean(0)
    se = np.sqrt(2 * var * var / M)
    assert np.all(np.abs(ex2 - var) < 5 * se), (ex2 - var) / se


# ----------------------------------------------------------------- the unadjusted step
def test_unadjusted_step_without_noise_is_leapfrog(ora):
    """With L -> infinity the O maps only renormalise, so one unadjusted
    iteration is one leapfrog step Phi_eps (Eq. "discrete update")."""
    pr = W.gauss_diag(d=6, M=5, n_steps=100)
    tg = ora.OracleTarget(ora.GAUSS_DIAG, 6, prec=pr.prec)
    run = ora.OracleLAPS(tg, pr.x0, seed=1, alpha=1e300)
    y0, u0, g0, lp0 = run.state()
    eps = run.trace[0]["eps"]
    run.iterate(1)
    y1, u1, _, _ = run.state()
    for m in range(5):
        x, u, g = y0[m].copy(), u0[m].copy(), g0[m].copy()
        ora.Phi(tg, ora.LF, eps, x, u, g, lp0[m])
        np.testing.assert_allclose(y1[m], x, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(u1[m], u / np.linalg.norm(u), rtol=1e-12, atol=1e-13)


def test_initialisation(ora):
    """Alg. 1 / App. C: eps0 = 0.01 sqrt(d), L0 = 2 sqrt(sum Var x0), u0 = g0/|g0|."""
    pr = W.gauss_diag(d=10, M=32, n_steps=100)
    tg = ora.OracleTarget(ora.GAUSS_DIAG, 10, prec=pr.prec)
    run = ora.OracleLAPS(tg, pr.x0, seed=1)
    r0 = run.trace[0]
    assert r0["eps"] == pytest.approx(0.01 * math.sqrt(10))
    assert r0["L"] == pytest.approx(2 * math.sqrt(np.var(pr.x0, axis=0).sum()), rel=1e-12)
    _, u, g, _ = run.state()
    np.testing.assert_allclose(u, g / np.linalg.norm(g, axis=1, keepdims=True), rtol=1e-14)


def test_eevpd_scales_like_eps6(ora):
    """Sec. 3.1: EEVPD grows as eps^6 (Gaussian, exact ensemble).  alpha -> 0
    makes the first O a full refresh, so the velocities are uniform on the
    sphere (the initial u0 = g0/|g0| would cancel the leading eps^3 term of
    the energy error and give eps^7 instead)."""
    d, M = 50, 8192
    var = np.logspace(-1, 1, d)
    rng = np.random.default_rng(16)
    x0 = rng.standard_normal((M, d)) * np.sqrt(var)
    tg = ora.OracleTarget(ora.GAUSS_DIAG, d, prec=1 / var)
    ee = []
    for coef in (0.005, 0.01):
        run = ora.OracleLAPS(tg, x0, seed=2, eps0_coef=coef, alpha=1e-9)
        run.iterate(1)
        ee.append(run.trace[1]["eevpd"])
    slope = math.log2(ee[1] / ee[0])
    assert abs(slope - 6.0) < 0.05, slope


# ------------------------------------------------------------------ full-rank D~ (App. B)
def test_rademacher_stream(ora):
    z = np.array([ora.rademacher(5, 0, 7, k, 512) for k in range(8)])
    assert set(np.unique(z)) == {-1.0, 1.0}
    assert abs(z.mean()) < 0.05
    assert not np.array_equal(z[0], z[1])
    assert not np.array_equal(ora.rademacher(5, 0, 7, 0, 64), ora.rademacher(5, 0, 8, 0, 64))
    assert not np.array_equal(ora.rademacher(5, 0, 7, 0, 64), ora.rademacher(5, 1, 7, 0, 64))


def test_dtilde_full_scaled_gaussian(ora):
    """Exact draws of N(0, s^2 Sigma) against the target N(0, Sigma): I - V = (1 - s^2) I,
    so D~ = (1 - s^2)^2 (Rademacher |z|^2 = d: no Hutchinson noise), up to the ensemble's
    off-diagonal noise ~ d / M."""
    rng = np.random.default_rng(1)
    d, M, s = 12, 40000, 1.3
    sig = np.exp(np.linspace(-1.0, 1.0, d))
    X = rng.standard_normal((M, d)) * sig * s
    G = -X / sig ** 2
    want = (1.0 - s * s) ** 2
    got = ora.dtilde_full(X, G, K=50, seed=3)
    # Hutchinson's expectation is the ensemble's own |I - V|_F^2 / d (plain numpy)
    V = -np.cov(X.T, G.T, bias=True)[:d, d:]
    B = np.eye(d) - V
    assert abs(got - np.sum(B * B) / d) < 0.02 * want
    assert abs(got - want) < 0.04 * want + 3.0 * d / M
    assert abs(ora.dtilde_diag(X, G) - want) < 0.04 * want


def test_dtilde_full_correlated_gaussian(ora):
    """Dense precision P, ensemble covariance C != P^-1: D~_full -> |I - C P|_F^2 / d,
    which the diagonal proxy (sum of the diagonal terms only) underestimates."""
    rng = np.random.default_rng(2)
    d, M = 6, 100000
    A = rng.standard_normal((d, d))
    P = A @ A.T / d + np.eye(d)
    Cv = 0.6 * np.linalg.inv(P) + 0.05 * np.outer(np.ones(d), np.ones(d))
    # an off-target ensemble mean: V is a covariance, so a missing centring would show
    X = rng.multivariate_normal(np.full(d, 0.7), Cv, size=M)
    G = -X @ P
    B = np.eye(d) - Cv @ P
    exact_full = np.sum(B * B) / d
    exact_diag = np.sum(np.diag(B) ** 2) / d
    assert exact_full > 1.2 * exact_diag
    got = ora.dtilde_full(X, G, K=400, seed=11)
    assert abs(got - exact_full) < 0.06 * exact_full, (got, exact_full)
    assert abs(ora.dtilde_diag(X, G) - exact_diag) < 0.03 * exact_diag


def test_dtilde_noise_floor_wishart(ora):
    """Both proxies on exact draws of the target itself (N(0, I), g = -x): V is
    the ensemble covariance S (a Wishart matrix over M - 1 degrees of freedom,
    normalised by M), so the finite-M floor of the proxies is fixed by its
    moments, E (S_ij - delta_ij)^2 = ((M - 1)(1 + delta_ij) + delta_ij) / M^2:
      D~_full -> ((M - 1)(d + 1) + 1) / M^2,   D~_diag -> (2 (M - 1) + 1) / M^2.
    The full-rank floor grows with d (every off-diagonal covariance is noise)."""
    rng = np.random.default_rng(0)
    d, M, reps = 20, 200, 60
    full, diag = [], []
    for r in range(reps):
        X = rng.standard_normal((M, d))
        full.append(ora.dtilde_full(X, -X, K=50, seed=r))
        diag.append(ora.dtilde_diag(X, -X))
    want_full = ((M - 1) * (d + 1) + 1) / M ** 2
    want_diag = (2 * (M - 1) + 1) / M ** 2
    for v, want in ((np.array(full), want_full), (np.array(diag), want_diag)):
        se = v.std() / np.sqrt(reps)
        assert abs(v.mean() - want) < 4.0 * se + 1e-3 * want, (v.mean(), want, se)
