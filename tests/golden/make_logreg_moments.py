"""Writes logreg_d101_n10000_moments.txt: reference second moments of the
logistic-regression posterior of the seeded workload (X 10000 x 100
standardised columns plus an intercept, w_true ~ N(0, I/100), prior N(0, I);
the stand-in for the paper's German Credit target of Sec. 6), for the bias
b^2 of Eq. "bias".

The posterior has no closed form.  The moments are estimated by
self-normalised importance sampling in FP64: proposals from the Laplace
Gaussian N(mode, s^2 H^-1) (H the negative Hessian at the mode, s = 1.05 so
that the proposal's tails are slightly heavier than the posterior's), weights
p(w) / q(w) with log p from the oracle's logistic-regression log density.
The file states the effective sample size and, per coordinate, the Monte
Carlo standard error of E[w_i^2] (delta method); with n = 10^4 rows the
posterior is close to Gaussian, the weights vary little and the standard
error is far below sd(w_i^2) / 100.

    python tests/golden/make_logreg_moments.py [n_draws]

Test infrastructure: it calls the oracle only (and numpy for the proposal).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "logreg_d101_n10000_moments.txt")
SCALE = 1.05


def importance_moments(X, y, prior_var, n_draws, seed=0, chunk=8192):
    """E[w_i^2], Var[w_i^2], the standard error of E[w_i^2] and the effective
    sample size, by self-normalised importance sampling from the Laplace
    Gaussian with covariance SCALE^2 H^-1."""
    import oracle
    from paper_2601_16696_gb300 import workloads
    mode, H = workloads.logreg_laplace(X, y, prior_var)
    d = mode.size
    cov = np.linalg.inv(H) * SCALE ** 2
    Lc = np.linalg.cholesky(cov)
    ot = oracle.OracleTarget(oracle.LOGREG, d, X=X, y=y, prior_var=prior_var)
    rng = np.random.default_rng(seed)
    logw, W2 = [], []
    for k0 in range(0, n_draws, chunk):
        n = min(chunk, n_draws - k0)
        z = rng.standard_normal((n, d))
        w = mode + z @ Lc.T
        lp, _ = ot.logp_grad(w)
        # log q up to a constant: -1/2 |L^-1 (w - mode)|^2 = -1/2 |z|^2
        lq = -0.5 * np.einsum("ij,ij->i", z, z)
        logw.append(lp - lq)
        W2.append(w * w)
    logw = np.concatenate(logw)
    W2 = np.concatenate(W2)
    a = np.exp(logw - logw.max())
    a /= a.sum()
    ess = 1.0 / np.sum(a * a)
    ex2 = a @ W2
    ex4 = a @ (W2 * W2)
    var2 = ex4 - ex2 * ex2
    se = np.sqrt(np.sum((a[:, None] * (W2 - ex2)) ** 2, axis=0))
    return ex2, var2, se, ess


def main(n_draws=200000):
    import oracle
    from paper_2601_16696_gb300 import workloads
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    pr = workloads.logreg(with_truth=True)
    t0 = time.time()
    ex2, var2, se, ess = importance_moments(pr.X, pr.y, pr.prior_var, n_draws)
    dt = time.time() - t0
    with open(OUT, "w") as f:
        f.write("# Reference second moments of the logistic-regression posterior (Sec. 6 target stand-in;\n")
        f.write("# b^2 of Eq. \"bias\"): workloads.logreg() defaults, d = %d, n = %d rows, prior N(0, I).\n"
                % (pr.d, pr.X.shape[0]))
        f.write("# Self-normalised importance sampling, %d draws from N(mode, %.2f^2 H^-1), log p from the\n"
                % (n_draws, SCALE))
        f.write("# oracle; effective sample size %.0f; %.0f s.  Written by tests/golden/make_logreg_moments.py.\n"
                % (ess, dt))
        f.write("# columns: i  E[w_i^2]  Var[w_i^2]  standard error of E[w_i^2]  Laplace E[w_i^2]\n")
        for i in range(pr.d):
            f.write("%d %.17g %.17g %.6g %.17g\n" % (i, ex2[i], var2[i], se[i], pr.Ex2[i]))
    print("wrote %s: ESS %.0f of %d draws, max se / sd(w^2) %.2e, max |IS - Laplace| / sd(w^2) %.3f"
          % (OUT, ess, n_draws, np.max(se / np.sqrt(var2)), np.max(np.abs(ex2 - pr.Ex2) / np.sqrt(var2))))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 200000)
