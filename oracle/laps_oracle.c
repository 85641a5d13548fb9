/*
 * laps_oracle.c -- plain FP64 CPU restatement of LAPS.  TEST INFRASTRUCTURE:
 * only tests, the smoke check and the benchmark's cpu_baseline leg load it.
 *
 * Each function follows one passage of the paper (Robnik & Seljak, "Faster
 * parallel MCMC: Metropolis adjustment is best served warm"), cited beside it.
 * Plain definitions are written out directly: two-pass means and variances,
 * the cosh/sinh form of the velocity update, the window statistics recomputed
 * from the stored window every step.  The loop over chains inside one
 * iteration may run on several OpenMP threads; chains are independent there
 * and every cross-chain sum is taken afterwards, serially, in chain order, so
 * the result does not depend on the thread count.
 *
 * Pins (tests/test_oracle_*.py check each against something other than this
 * file): Philox by its statistics, by the generator's published known-answer
 * vectors and, on a GPU, bit equality with cuRAND's device Philox4x32-10 on
 * 2^20 random (counter, key) pairs (tests/test_gpu_philox_curand.py); O/A/B by
 * unit norm, reversibility and an RK4 solution of the
 * velocity ODE; integrators by coefficient identities and their convergence
 * order; Delta by its vanishing at the integrator order; F and D~_diag by
 * closed forms on Gaussians; MAMS by a brute-force transition histogram and
 * stationarity; the full run by exact Gaussian / banana / funnel moments.
 * Logistic regression log p and gradient are pinned by finite differences and
 * by the closed form at w = 0; a whole run on a two-dimensional posterior by
 * the brute-force integral of its second moments (tests/test_oracle_runs.py).
 * The full-size posterior's moments come from importance sampling with this
 * log density, its estimator pinned by the same integral in 2-D.
 */
#include "laps_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.2): ten rounds of
 * two 32x32->64 multiplications whose halves are xor-ed with the other words
 * and the round key; the key is bumped by the Weyl constants between rounds. */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double ora_uniform(uint32_t r) {
    return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); /* 2^-23 */
}

static const double ORA_PI = 3.14159265358979323846;

void ora_normals4(uint64_t seed, uint32_t j, uint32_t m, uint32_t t, uint32_t tag,
                  uint32_t pid, double z[4]) {
    uint32_t ctr[4] = {j, m, t, tag | (pid << 8)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    /* Box-Muller on the pairs (r0, r1) and (r2, r3) */
    for (int h = 0; h < 2; ++h) {
        double u0 = ora_uniform(r[2 * h]), u1 = ora_uniform(r[2 * h + 1]);
        double rad = sqrt(-2.0 * log(u0));
        z[2 * h] = rad * cos(2.0 * ORA_PI * u1);
        z[2 * h + 1] = rad * sin(2.0 * ORA_PI * u1);
    }
}

void ora_normals(uint64_t seed, uint32_t m, uint32_t t, uint32_t tag, uint32_t pid,
                 int64_t d, double* z) {
    for (int64_t j = 0; 4 * j < d; ++j) {
        double q[4];
        ora_normals4(seed, (uint32_t)j, m, t, tag, pid, q);
        for (int k = 0; k < 4 && 4 * j + k < d; ++k) z[4 * j + k] = q[k];
    }
}

/* Diagnostic only (round_state_f32): round a vector to binary32 after a map,
 * and form logistic-regression logits as a binary32 dot product, to measure
 * how much binary32 arithmetic perturbs the run.  Set by ora_iterate for the
 * duration of one iteration. */
static int g_round_f32 = 0;

/* ------------------------------------------------------------------------ */
/* Targets.  log p up to an additive constant, and its gradient. */
static double softplus(double z) { return (z > 0 ? z : 0.0) + log1p(exp(-fabs(z))); }
static double sigmoid(double z) {
    if (z >= 0) return 1.0 / (1.0 + exp(-z));
    double e = exp(z);
    return e / (1.0 + e);
}

double ora_logp_grad(const ora_target* tg, const double* x, double* g) {
    const int64_t d = tg->d;
    double lp = 0.0;
    switch (tg->kind) {
    case ORA_GAUSS_DIAG: /* -1/2 sum prec_i x_i^2 */
        for (int64_t i = 0; i < d; ++i) {
            lp += -0.5 * tg->prec[i] * x[i] * x[i];
            g[i] = -tg->prec[i] * x[i];
        }
        break;
    case ORA_GAUSS_DENSE: /* -1/2 x^T P x, grad -P x (Sec. 6, the rotated ill-conditioned Gaussian) */
        for (int64_t i = 0; i < d; ++i) {
            double r = 0.0;
            for (int64_t j = 0; j < d; ++j) r += tg->prec[i * d + j] * x[j];
            g[i] = -r;
            lp += -0.5 * x[i] * r;
        }
        break;
    case ORA_BANANA: { /* pairs (a, b) = (x_2k, x_2k+1): a ~ N(0,1), b|a ~ N(a^2, s^2) */
        const double s2 = tg->banana_sb * tg->banana_sb;
        for (int64_t k = 0; 2 * k + 1 < d; ++k) {
            double a = x[2 * k], b = x[2 * k + 1];
            double r = b - a * a;
            lp += -0.5 * a * a - 0.5 * r * r / s2;
            g[2 * k] = -a + 2.0 * a * r / s2;
            g[2 * k + 1] = -r / s2;
        }
        break;
    }
    case ORA_FUNNEL: { /* v = x_0 ~ N(0, sv^2); x_i | v ~ N(0, e^v), i = 1..d-1 */
        const double v = x[0], sv2 = tg->funnel_sv * tg->funnel_sv;
        const double n = (double)(d - 1);
        double ss = 0.0;
        for (int64_t i = 1; i < d; ++i) ss += x[i] * x[i];
        const double ev = exp(-v);
        lp = -0.5 * v * v / sv2 - 0.5 * n * v - 0.5 * ev * ss;
        g[0] = -v / sv2 - 0.5 * n + 0.5 * ev * ss;
        for (int64_t i = 1; i < d; ++i) g[i] = -x[i] * ev;
        break;
    }
    case ORA_LOGREG: { /* sum_n [y_n z_n - softplus(z_n)] - |w|^2 / (2 prior_var) */
        for (int64_t i = 0; i < d; ++i) {
            lp += -0.5 * x[i] * x[i] / tg->prior_var;
            g[i] = -x[i] / tg->prior_var;
        }
        for (int64_t n = 0; n < tg->n_data; ++n) {
            const double* xn = tg->X + n * d;
            double z = 0.0;
            if (g_round_f32) { /* diagnostic: a binary32 dot product, in index order */
                float zf = 0.0f;
                for (int64_t i = 0; i < d; ++i) zf = fmaf((float)xn[i], (float)x[i], zf);
                z = zf;
            } else {
                for (int64_t i = 0; i < d; ++i) z += xn[i] * x[i];
            }
            lp += tg->y[n] * z - softplus(z);
            double r = tg->y[n] - sigmoid(z);
            for (int64_t i = 0; i < d; ++i) g[i] += r * xn[i];
        }
        break;
    }
    default:
        lp = NAN;
    }
    return lp;
}

/* evaluation in the sampler's coordinates y, with x = sigma o y (sigma NULL:
 * identity).  The gradient in y is sigma o grad_x; log p is unchanged. */
static double eval_y(const ora_target* tg, const double* sigma, const double* y, double* gy,
                     double* xbuf) {
    if (!sigma) return ora_logp_grad(tg, y, gy);
    const int64_t d = tg->d;
    for (int64_t i = 0; i < d; ++i) xbuf[i] = sigma[i] * y[i];
    double lp = ora_logp_grad(tg, xbuf, gy);
    for (int64_t i = 0; i < d; ++i) gy[i] *= sigma[i];
    return lp;
}

/* ------------------------------------------------------------------------ */
/* App. E, Eq. "O update": partial velocity refresh on the unit sphere. */
void ora_O(int64_t d, double eps, double L, const double* z, double* u) {
    const double c1 = exp(-eps / L);
    const double c2 = sqrt(1.0 - c1 * c1);
    double nrm = 0.0;
    for (int64_t i = 0; i < d; ++i) {
        u[i] = c1 * u[i] + c2 * z[i];
        nrm += u[i] * u[i];
    }
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < d; ++i) u[i] /= nrm;
}

/* App. E, "Position update". */
void ora_A(int64_t d, double eps, const double* u, double* x) {
    for (int64_t i = 0; i < d; ++i) x[i] += eps * u[i];
}

/* App. E, Eq. "B MCHMC" and the kinetic energy change below it. */
double ora_B(int64_t d, double eps, const double* g, double* u) {
    double gn = 0.0;
    for (int64_t i = 0; i < d; ++i) gn += g[i] * g[i];
    gn = sqrt(gn);
    if (gn == 0.0) return 0.0; /* no force: u is unchanged, no energy change */
    double eu = 0.0;
    for (int64_t i = 0; i < d; ++i) eu += (g[i] / gn) * u[i];
    const double delta = eps * gn / (double)(d - 1);
    const double ch = cosh(delta), sh = sinh(delta);
    const double den = ch + eu * sh;
    const double coef = sh + eu * (ch - 1.0);
    for (int64_t i = 0; i < d; ++i) u[i] = (u[i] + coef * (g[i] / gn)) / den;
    return (double)(d - 1) * log(den);
}

/* Table "integrators": b_1 ... b_K (velocity stages), a_1 ... a_{K-1}
 * (position stages); the omitted ones follow from the symmetry
 * a_k = a_{K-k}, b_k = b_{K+1-k} and the normalisation sum b = sum a = 1. */
int ora_integrator_coefs(int integ, double* b, double* a) {
    switch (integ) {
    case ORA_LF:
        b[0] = 0.5; b[1] = 0.5;
        a[0] = 1.0;
        return 2;
    case ORA_MN2: {
        const double b1 = 0.1931833275;
        b[0] = b1; b[1] = 1.0 - 2.0 * b1; b[2] = b1;
        a[0] = 0.5; a[1] = 0.5;
        return 3;
    }
    case ORA_MN4: {
        const double b1 = 0.0839831526, b2 = 0.6822365335;
        const double a1 = 0.2539785108, a2 = -0.032302867;
        const double b3 = 0.5 - b1 - b2;           /* sum b = 1 */
        const double a3 = 1.0 - 2.0 * (a1 + a2);   /* sum a = 1 */
        b[0] = b1; b[1] = b2; b[2] = b3; b[3] = b3; b[4] = b2; b[5] = b1;
        a[0] = a1; a[1] = a2; a[2] = a3; a[3] = a2; a[4] = a1;
        return 6;
    }
    }
    return 0;
}

static void round_f32(int64_t d, double* v) {
    if (!g_round_f32) return;
    for (int64_t i = 0; i < d; ++i) v[i] = (double)(float)v[i];
}

/* Eq. "integrator": Phi = B_{b1 eps} A_{a1 eps} B_{b2 eps} ... B_{bK eps}.
 * Energy error: each A adds -log p(x') + log p(x), each B its kinetic term. */
static double phi_y(const ora_target* tg, const double* sigma, int integ, double eps,
                    double* y, double* u, double* g, double* logp, double* xbuf) {
    double b[8], a[8];
    const int K = ora_integrator_coefs(integ, b, a);
    const int64_t d = tg->d;
    double delta = 0.0;
    for (int k = 0; k < K; ++k) {
        delta += ora_B(d, b[k] * eps, g, u);
        round_f32(d, u);
        if (k < K - 1) {
            ora_A(d, a[k] * eps, u, y);
            round_f32(d, y);
            double lp_new = eval_y(tg, sigma, y, g, xbuf);
            round_f32(d, g);
            delta += -lp_new + *logp;
            *logp = lp_new;
        }
    }
    return delta;
}

double ora_Phi(const ora_target* tg, int integ, double eps, double* x, double* u, double* g,
               double* logp) {
    return phi_y(tg, NULL, integ, eps, x, u, g, logp, NULL);
}

static int grads_per_step(int integ) { return integ == ORA_LF ? 1 : (integ == ORA_MN2 ? 2 : 5); }

/* ------------------------------------------------------------------------ */
/* Eq. "bias bound": F(D) = 4 D^{3/2} / (1 + D^{1/2})^2. */
double ora_F(double D) {
    const double s = sqrt(D);
    return 4.0 * D * s / ((1.0 + s) * (1.0 + s));
}

/* App. B, "Diagonal": D~_diag = (1/d) sum_i (1 - V_ii)^2 with
 * V_ii = E_rho[-(x_i - E_rho x_i) d_i log p]  (Eq. ECA for the expectations). */
double ora_dtilde_diag(int64_t M, int64_t d, const double* X, const double* G) {
    double acc = 0.0;
    for (int64_t i = 0; i < d; ++i) {
        double mx = 0.0;
        for (int64_t m = 0; m < M; ++m) mx += X[m * d + i];
        mx /= (double)M;
        double v = 0.0;
        for (int64_t m = 0; m < M; ++m) v += -(X[m * d + i] - mx) * G[m * d + i];
        v /= (double)M;
        acc += (1.0 - v) * (1.0 - v);
    }
    return acc / (double)d;
}

/* Rademacher entry z_k,i = +1 if bit (i mod 32) of word (i / 32 mod 4) of
 * Philox(counter (i / 128, k, t, 5 | pid << 8)) is set, else -1. */
double ora_rademacher(uint64_t seed, uint32_t pid, uint32_t t, uint32_t k, int64_t i) {
    uint32_t ctr[4] = {(uint32_t)(i / 128), k, t, 5u | (pid << 8)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    ora_philox4x32_10(ctr, key, out);
    return ((out[(i / 32) % 4] >> (i % 32)) & 1u) ? 1.0 : -1.0;
}

/* App. B, "Full rank": D~ = |I - V|_F^2 / d with V_ij = -Cov_rho(x_i, d_j log p),
 * by Hutchinson's trace estimator over K Rademacher vectors z_k (drawn for
 * step t):  (I - V) z = z + Cov_rho(x, g.z), so
 *   D~_full = (1/(d K)) sum_k | z_k + (1/M) sum_m (x^m - xbar)(s_mk - sbar_k) |^2,
 * s_mk = g^m . z_k  (Eq. ECA for the ensemble expectations). */
double ora_dtilde_full(int64_t M, int64_t d, const double* X, const double* G, int K, uint64_t seed,
                       uint32_t pid, uint32_t t) {
    double* z = (double*)malloc((size_t)d * sizeof(double));
    double* sm = (double*)malloc((size_t)M * sizeof(double));
    double* xbar = (double*)malloc((size_t)d * sizeof(double));
    for (int64_t i = 0; i < d; ++i) {
        double a = 0.0;
        for (int64_t m = 0; m < M; ++m) a += X[m * d + i];
        xbar[i] = a / (double)M;
    }
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        for (int64_t i = 0; i < d; ++i) z[i] = ora_rademacher(seed, pid, t, (uint32_t)k, i);
        double sbar = 0.0;
        for (int64_t m = 0; m < M; ++m) {
            double a = 0.0;
            for (int64_t i = 0; i < d; ++i) a += G[m * d + i] * z[i];
            sm[m] = a;
            sbar += a;
        }
        sbar /= (double)M;
        for (int64_t i = 0; i < d; ++i) {
            double c = 0.0;
            for (int64_t m = 0; m < M; ++m) c += (X[m * d + i] - xbar[i]) * (sm[m] - sbar);
            c /= (double)M;
            acc += (z[i] + c) * (z[i] + c);
        }
    }
    free(z);
    free(sm);
    free(xbar);
    return acc / ((double)d * (double)K);
}

static double var_col(int64_t M, int64_t d, const double* X, int64_t i) {
    double mx = 0.0;
    for (int64_t m = 0; m < M; ++m) mx += X[m * d + i];
    mx /= (double)M;
    double v = 0.0;
    for (int64_t m = 0; m < M; ++m) v += (X[m * d + i] - mx) * (X[m * d + i] - mx);
    return v / (double)M;
}

/* Eq. "L": L = alpha (sum_i Var_rho[x_i])^{1/2}. */
double ora_L_of(int64_t M, int64_t d, const double* X, double alpha) {
    double s = 0.0;
    for (int64_t i = 0; i < d; ++i) s += var_col(M, d, X, i);
    return alpha * sqrt(s);
}

/* Eq. "relative fluctuations": delta = sigma / mu over a window of T values,
 * sigma^2 with the 1/(T-1) normalisation. */
double ora_rel_fluct(int64_t T, const double* hist) {
    double mu = 0.0;
    for (int64_t s = 0; s < T; ++s) mu += hist[s];
    mu /= (double)T;
    double v = 0.0;
    for (int64_t s = 0; s < T; ++s) v += (hist[s] - mu) * (hist[s] - mu);
    v /= (double)(T - 1);
    return sqrt(v) / mu;
}

/* Sec. 5.1: double (halve) until the root of a(eps) - a* is bracketed, then
 * bisect the bracket. */
double ora_bisect(double eps, double a, double a_target, double* lo, double* hi) {
    if (a > a_target) { /* steps too small */
        *lo = eps;
        return (*hi > 0) ? 0.5 * (*lo + *hi) : 2.0 * eps;
    }
    *hi = eps;
    return (*lo > 0) ? 0.5 * (*lo + *hi) : 0.5 * eps;
}

/* ------------------------------------------------------------------------ */
void ora_config_default(ora_config* c) {
    c->C = 0.025;
    c->alpha = 2.0;
    c->switch_tol = 0.01;
    c->window_frac = 0.2;
    c->acc_tol = 0.03;
    c->adj_L_factor = 1.25;
    c->eps0_coef = 0.01;
    c->a_target_mn2 = 0.7;
    c->a_target_mn4 = 0.9;
    c->n_total_steps = 2000;
    c->steps_per_proposal = 15;
    c->mn4_min_dim = 200;
    c->eevpd_centered = 1;
    c->adjusted = 1;
    c->force_switch_at = 0;
    c->fixed_eps = 0.0;
    c->round_state_f32 = 0;
    c->dtilde_K = 0;
}

struct ora_state {
    ora_target tg;
    ora_config cfg;
    int64_t M, d;
    uint64_t seed;
    uint32_t pid;
    double *y, *u, *g, *logp;          /* sampler coordinates */
    double *y0, *u0, *g0, *logp0;      /* per-chain copies (revert / reject) */
    double* sigma;                     /* preconditioner (NULL before the switch) */
    double* xbuf;                      /* per-chain scratch for x = sigma o y */
    double* delta;                     /* per-chain energy error of the iteration */
    double* acc;                       /* per-chain acceptance probability */
    int* bad;                          /* per-chain non-finite flag */
    double* window;                    /* [T][d] ring of E[x_i^2] */
    int64_t T, win_n;
    double *Ex2, *Varx2;               /* truth for b^2 (optional) */
    double eps, L;
    int phase, t, t_switch, integ, adapting, p, done;
    double lo, hi, a_target;
    long long grads;
};

static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

static void state_stats(const ora_state* s, ora_trace_row* row);

ora_state* ora_create(const ora_target* tg, const ora_config* cfg, int64_t M, const double* x0,
                      uint64_t seed, uint32_t pid) {
    ora_state* s = (ora_state*)xcalloc(1, sizeof(ora_state));
    s->tg = *tg;
    s->cfg = *cfg;
    s->M = M;
    s->d = tg->d;
    s->seed = seed;
    s->pid = pid;
    const int64_t Md = M * s->d;
    s->y = (double*)xcalloc(Md, sizeof(double));
    s->u = (double*)xcalloc(Md, sizeof(double));
    s->g = (double*)xcalloc(Md, sizeof(double));
    s->logp = (double*)xcalloc(M, sizeof(double));
    s->y0 = (double*)xcalloc(Md, sizeof(double));
    s->u0 = (double*)xcalloc(Md, sizeof(double));
    s->g0 = (double*)xcalloc(Md, sizeof(double));
    s->logp0 = (double*)xcalloc(M, sizeof(double));
    s->xbuf = (double*)xcalloc(Md, sizeof(double));
    s->delta = (double*)xcalloc(M, sizeof(double));
    s->acc = (double*)xcalloc(M, sizeof(double));
    s->bad = (int*)xcalloc(M, sizeof(int));
    s->T = (int64_t)ceil(cfg->window_frac * (double)cfg->n_total_steps);
    if (s->T < 2) s->T = 2;
    s->window = (double*)xcalloc(s->T * s->d, sizeof(double));
    memcpy(s->y, x0, (size_t)Md * sizeof(double));

    const int64_t d = s->d;
    /* Alg. 1 / App. C "Initialization": gradient at x0, velocity along it */
    for (int64_t m = 0; m < M; ++m) {
        double* ym = s->y + m * d;
        double* um = s->u + m * d;
        double* gm = s->g + m * d;
        s->logp[m] = ora_logp_grad(tg, ym, gm);
        double gn = 0.0;
        for (int64_t i = 0; i < d; ++i) gn += gm[i] * gm[i];
        gn = sqrt(gn);
        if (gn > 0.0) {
            for (int64_t i = 0; i < d; ++i) um[i] = gm[i] / gn;
        } else { /* no gradient: a uniformly random direction */
            ora_normals(seed, (uint32_t)m, 0xFFFFFFFFu, ORA_TAG_O1, pid, d, um);
            double n2 = 0.0;
            for (int64_t i = 0; i < d; ++i) n2 += um[i] * um[i];
            n2 = sqrt(n2);
            for (int64_t i = 0; i < d; ++i) um[i] /= n2;
        }
    }
    s->eps = cfg->fixed_eps > 0 ? cfg->fixed_eps : cfg->eps0_coef * sqrt((double)d);
    s->L = ora_L_of(M, d, s->y, cfg->alpha);
    s->phase = 0;
    s->t = 0;
    s->t_switch = -1;
    s->integ = ORA_LF;
    s->grads = 1;
    return s;
}

void ora_destroy(ora_state* s) {
    if (!s) return;
    free(s->y); free(s->u); free(s->g); free(s->logp);
    free(s->y0); free(s->u0); free(s->g0); free(s->logp0);
    free(s->sigma); free(s->xbuf); free(s->delta); free(s->acc); free(s->bad);
    free(s->window); free(s->Ex2); free(s->Varx2);
    free(s);
}

void ora_set_truth(ora_state* s, const double* Ex2, const double* Varx2) {
    free(s->Ex2); free(s->Varx2);
    s->Ex2 = (double*)xcalloc(s->d, sizeof(double));
    s->Varx2 = (double*)xcalloc(s->d, sizeof(double));
    memcpy(s->Ex2, Ex2, (size_t)s->d * sizeof(double));
    memcpy(s->Varx2, Varx2, (size_t)s->d * sizeof(double));
}

void ora_get_x(const ora_state* s, double* x) {
    for (int64_t m = 0; m < s->M; ++m)
        for (int64_t i = 0; i < s->d; ++i)
            x[m * s->d + i] = (s->sigma ? s->sigma[i] : 1.0) * s->y[m * s->d + i];
}

void ora_get_state(const ora_state* s, double* y, double* u, double* g, double* logp) {
    const size_t Md = (size_t)(s->M * s->d);
    if (y) memcpy(y, s->y, Md * sizeof(double));
    if (u) memcpy(u, s->u, Md * sizeof(double));
    if (g) memcpy(g, s->g, Md * sizeof(double));
    if (logp) memcpy(logp, s->logp, (size_t)s->M * sizeof(double));
}

void ora_get_sigma(const ora_state* s, double* sigma) {
    for (int64_t i = 0; i < s->d; ++i) sigma[i] = s->sigma ? s->sigma[i] : 1.0;
}
int ora_phase(const ora_state* s) { return s->phase; }
int ora_t(const ora_state* s) { return s->t; }
int ora_t_switch(const ora_state* s) { return s->t_switch; }
int ora_window_T(const ora_state* s) { return (int)s->T; }
int ora_integrator(const ora_state* s) { return s->integ; }

/* moments of the ensemble in x space that every trace row reports */
static void state_stats(const ora_state* s, ora_trace_row* row) {
    const int64_t M = s->M, d = s->d;
    double sum_var = 0.0, b2max = 0.0, b2sum = 0.0;
    for (int64_t i = 0; i < d; ++i) {
        const double sg = s->sigma ? s->sigma[i] : 1.0;
        double mx = 0.0, mxx = 0.0;
        for (int64_t m = 0; m < M; ++m) {
            double x = sg * s->y[m * d + i];
            mx += x;
            mxx += x * x;
        }
        mx /= (double)M;
        mxx /= (double)M;
        double v = 0.0;
        for (int64_t m = 0; m < M; ++m) {
            double x = sg * s->y[m * d + i];
            v += (x - mx) * (x - mx);
        }
        sum_var += v / (double)M;
        if (s->Ex2) {
            double b2 = (mxx - s->Ex2[i]) * (mxx - s->Ex2[i]) / s->Varx2[i];
            b2sum += b2;
            if (b2 > b2max) b2max = b2;
        }
    }
    row->sum_var = sum_var;
    row->b2_max = s->Ex2 ? b2max : NAN;
    row->b2_avg = s->Ex2 ? b2sum / (double)d : NAN;
}

void ora_row0(const ora_state* s, ora_trace_row* row) {
    memset(row, 0, sizeof(*row));
    row->phase = 0;
    row->t = 0;
    row->eps = s->eps;
    row->L = s->L;
    row->eps_used = NAN;
    row->eevpd = NAN;
    row->eevpd_wanted = NAN;
    row->dtilde = NAN;
    row->max_delta = NAN;
    row->acc = NAN;
    row->grads = s->grads;
    state_stats(s, row);
}

static int finite_chain(const ora_state* s, int64_t m) {
    const int64_t d = s->d;
    if (!isfinite(s->logp[m]) || !isfinite(s->delta[m])) return 0;
    for (int64_t i = 0; i < d; ++i)
        if (!isfinite(s->y[m * d + i]) || !isfinite(s->u[m * d + i]) || !isfinite(s->g[m * d + i]))
            return 0;
    return 1;
}

/* one unadjusted chain update: phi = O_{eps/2} Phi_eps O_{eps/2}
 * (App. E, Eq. "discrete update"), leapfrog for Phi */
static void unadjusted_chain(ora_state* s, int64_t m, double* z) {
    const int64_t d = s->d;
    double* y = s->y + m * d;
    double* u = s->u + m * d;
    double* g = s->g + m * d;
    const double inv_sqrt_d = 1.0 / sqrt((double)d);
    memcpy(s->y0 + m * d, y, (size_t)d * sizeof(double));
    memcpy(s->u0 + m * d, u, (size_t)d * sizeof(double));
    memcpy(s->g0 + m * d, g, (size_t)d * sizeof(double));
    s->logp0[m] = s->logp[m];

    ora_normals(s->seed, (uint32_t)m, (uint32_t)s->t, ORA_TAG_O1, s->pid, d, z);
    for (int64_t i = 0; i < d; ++i) z[i] *= inv_sqrt_d;
    ora_O(d, 0.5 * s->eps, s->L, z, u);
    round_f32(d, u);
    s->delta[m] = phi_y(&s->tg, NULL, ORA_LF, s->eps, y, u, g, &s->logp[m], s->xbuf + m * d);
    ora_normals(s->seed, (uint32_t)m, (uint32_t)s->t, ORA_TAG_O2, s->pid, d, z);
    for (int64_t i = 0; i < d; ++i) z[i] *= inv_sqrt_d;
    ora_O(d, 0.5 * s->eps, s->L, z, u);
    round_f32(d, u);

    s->bad[m] = !finite_chain(s, m);
    if (s->bad[m]) { /* revert the chain to its state before the step */
        memcpy(y, s->y0 + m * d, (size_t)d * sizeof(double));
        memcpy(u, s->u0 + m * d, (size_t)d * sizeof(double));
        memcpy(g, s->g0 + m * d, (size_t)d * sizeof(double));
        s->logp[m] = s->logp0[m];
    }
}

/* App. F: one MAMS proposal for one chain in sampler coordinates y (x = sigma o
 * y; sigma NULL is the identity).  z, y0, g0, xb are d-long scratch. */
static double mams_core(const ora_target* tg, const double* sigma, int integ, double eps,
                        double L, int n_steps, uint64_t seed, uint32_t pid, uint32_t m,
                        uint32_t t0, uint32_t p, double* y, double* g, double* logp, double* u,
                        double* z, double* y0, double* g0, double* xb, int mh_mode,
                        int* accepted, int* finite_out, double* delta_out) {
    const int64_t d = tg->d;
    memcpy(y0, y, (size_t)d * sizeof(double));
    memcpy(g0, g, (size_t)d * sizeof(double));
    const double lp0 = *logp;
    const double inv_sqrt_d = 1.0 / sqrt((double)d);

    /* step 2: u uniform on the sphere, u = Z / |Z|, Z ~ N(0, I) */
    ora_normals(seed, m, p, ORA_TAG_REFRESH, pid, d, u);
    double n2 = 0.0;
    for (int64_t i = 0; i < d; ++i) n2 += u[i] * u[i];
    n2 = sqrt(n2);
    for (int64_t i = 0; i < d; ++i) u[i] /= n2;
    /* steps 3-4: N steps of phi (partial refreshes included), energy error */
    double delta = 0.0;
    for (int n = 0; n < n_steps; ++n) {
        ora_normals(seed, m, t0 + (uint32_t)n, ORA_TAG_O1, pid, d, z);
        for (int64_t i = 0; i < d; ++i) z[i] *= inv_sqrt_d;
        ora_O(d, 0.5 * eps, L, z, u);
        round_f32(d, u);
        delta += phi_y(tg, sigma, integ, eps, y, u, g, logp, xb);
        ora_normals(seed, m, t0 + (uint32_t)n, ORA_TAG_O2, pid, d, z);
        for (int64_t i = 0; i < d; ++i) z[i] *= inv_sqrt_d;
        ora_O(d, 0.5 * eps, L, z, u);
        round_f32(d, u);
    }
    int finite = isfinite(delta) && isfinite(*logp);
    for (int64_t i = 0; i < d && finite; ++i) finite = isfinite(y[i]) && isfinite(g[i]);
    /* step 5: accept with probability min(1, e^-Delta), else stay at the start */
    uint32_t ctr[4] = {0u, m, p, (uint32_t)ORA_TAG_MH | (pid << 8)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    const double U = ora_uniform(r[0]);
    int acc = finite && (log(U) < -delta);
    if (mh_mode == 1) acc = finite;                      /* planted: accept all */
    if (mh_mode == 2) acc = finite && (log(U) < delta);  /* planted: sign flip */
    const double a = finite ? (delta <= 0 ? 1.0 : exp(-delta)) : 0.0;
    if (!acc) {
        memcpy(y, y0, (size_t)d * sizeof(double));
        memcpy(g, g0, (size_t)d * sizeof(double));
        *logp = lp0;
    }
    *accepted = acc;
    if (finite_out) *finite_out = finite;
    if (delta_out) *delta_out = delta;
    return a;
}

double ora_mams_proposal(const ora_target* tg, int integ, double eps, double L, int n_steps,
                         uint64_t seed, uint32_t pid, uint32_t m, uint32_t t0, uint32_t p,
                         double* x, double* g, double* logp, double* u, int* accepted,
                         double* delta_out) {
    const int64_t d = tg->d;
    double* buf = (double*)malloc((size_t)(4 * d) * sizeof(double));
    double a = mams_core(tg, NULL, integ, eps, L, n_steps, seed, pid, m, t0, p, x, g, logp, u,
                         buf, buf + d, buf + 2 * d, buf + 3 * d, 0, accepted, NULL, delta_out);
    free(buf);
    return a;
}

static void switch_to_adjusted(ora_state* s, const double* var) {
    const int64_t M = s->M, d = s->d;
    /* Sec. 4: y_i = x_i / Var[x_i]^{1/2}, fixed from now on */
    s->sigma = (double*)xcalloc(d, sizeof(double));
    double sum_var = 0.0;
    for (int64_t i = 0; i < d; ++i) {
        s->sigma[i] = var[i] > 0 ? sqrt(var[i]) : 1.0;
        sum_var += var[i];
    }
    for (int64_t m = 0; m < M; ++m)
        for (int64_t i = 0; i < d; ++i) {
            s->y[m * d + i] /= s->sigma[i];
            s->g[m * d + i] *= s->sigma[i];
        }
    /* step size carried into whitened coordinates (keeps eps/L) */
    if (sum_var > 0) s->eps *= sqrt((double)d / sum_var);
    s->integ = (d > s->cfg.mn4_min_dim) ? ORA_MN4 : ORA_MN2;
    s->a_target = (s->integ == ORA_MN4) ? s->cfg.a_target_mn4 : s->cfg.a_target_mn2;
    s->L = s->cfg.adj_L_factor * (double)s->cfg.steps_per_proposal * s->eps;
    s->lo = 0.0;
    s->hi = 0.0;
    s->adapting = 1;
    s->p = 0;
    s->phase = 1;
    s->t_switch = s->t;
}

static double mams_chain(ora_state* s, int64_t m, uint32_t t0, double* z) {
    const int64_t d = s->d;
    int acc, finite;
    double delta;
    double a = mams_core(&s->tg, s->sigma, s->integ, s->eps, s->L, s->cfg.steps_per_proposal,
                         s->seed, s->pid, (uint32_t)m, t0, (uint32_t)s->p, s->y + m * d,
                         s->g + m * d, &s->logp[m], s->u + m * d, z, s->y0 + m * d,
                         s->g0 + m * d, s->xbuf + m * d, 0, &acc, &finite, &delta);
    s->bad[m] = !finite;
    s->delta[m] = delta;
    return a;
}

static int iterate_body(ora_state* s, ora_trace_row* row);

int ora_iterate(ora_state* s, ora_trace_row* row) {
    g_round_f32 = s->cfg.round_state_f32;
    const int r = iterate_body(s, row);
    g_round_f32 = 0;
    return r;
}

static int iterate_body(ora_state* s, ora_trace_row* row) {
    const int64_t M = s->M, d = s->d;
    const ora_config* c = &s->cfg;
    if (s->done) return 0;
    memset(row, 0, sizeof(*row));
    row->eevpd = row->eevpd_wanted = row->dtilde = row->max_delta = row->acc = NAN;

    if (s->phase == 0) {
        if (s->t >= c->n_total_steps) { s->done = 1; return 0; }
        /* --- Alg. 1, unadjusted loop body --- */
        row->eps_used = s->eps;
#pragma omp parallel
        {
            double* z = (double*)malloc((size_t)d * sizeof(double));
#pragma omp for schedule(static)
            for (int64_t m = 0; m < M; ++m) unadjusted_chain(s, m, z);
            free(z);
        }
        s->grads += grads_per_step(ORA_LF);
        s->t += 1;
        /* ensemble expectations (Eq. ECA), serial and in chain order */
        int nbad = 0;
        double sd = 0.0, sdd = 0.0;
        int64_t nfin = 0;
        for (int64_t m = 0; m < M; ++m) {
            if (s->bad[m]) { nbad++; continue; }
            sd += s->delta[m];
            sdd += s->delta[m] * s->delta[m];
            nfin++;
        }
        double* var = (double*)malloc((size_t)d * sizeof(double));
        double sum_var = 0.0;
        for (int64_t i = 0; i < d; ++i) { var[i] = var_col(M, d, s->y, i); sum_var += var[i]; }
        const double dt = c->dtilde_K > 0
                              ? ora_dtilde_full(M, d, s->y, s->g, c->dtilde_K, s->seed, s->pid,
                                                (uint32_t)(s->t - 1))
                              : ora_dtilde_diag(M, d, s->y, s->g);
        double eevpd = NAN;
        if (nfin > 0) {
            const double mean = sd / (double)nfin;
            eevpd = c->eevpd_centered ? (sdd / (double)nfin - mean * mean) / (double)d
                                      : (sdd / (double)nfin) / (double)d;
        }
        /* Sec. 3.1 steps 2-5 */
        const double wanted = ora_F(c->C * dt);
        if (c->fixed_eps > 0)
            s->eps = c->fixed_eps;  /* the fixed-step ablation: no controller */
        else if (nbad > 0 || !(eevpd > 0) || !isfinite(eevpd) || !isfinite(wanted))
            s->eps = 0.5 * s->eps;
        else
            s->eps = s->eps * pow(wanted / eevpd, 1.0 / 6.0);
        s->L = c->alpha * sqrt(sum_var);        /* Eq. "L" */
        /* Sec. 4: window of E[x_i^2] and its relative fluctuations */
        const int64_t slot = s->win_n % s->T;
        for (int64_t i = 0; i < d; ++i) {
            double e = 0.0;
            for (int64_t m = 0; m < M; ++m) e += s->y[m * d + i] * s->y[m * d + i];
            s->window[slot * d + i] = e / (double)M;
        }
        s->win_n++;
        double maxdel = NAN;
        if (s->win_n >= s->T) {
            double* hist = (double*)malloc((size_t)s->T * sizeof(double));
            maxdel = 0.0;
            for (int64_t i = 0; i < d; ++i) {
                for (int64_t k = 0; k < s->T; ++k) {
                    const int64_t age = s->T - 1 - k;             /* k: oldest first */
                    const int64_t sl = (s->win_n - 1 - age) % s->T;
                    hist[k] = s->window[sl * d + i];
                }
                const double del = ora_rel_fluct(s->T, hist);
                if (!(del <= maxdel)) maxdel = del; /* NaN propagates */
            }
            free(hist);
        }
        row->phase = 0;
        row->eevpd = eevpd;
        row->eevpd_wanted = wanted;
        row->dtilde = dt;
        row->max_delta = maxdel;
        row->nonfinite = nbad;
        row->t = s->t;
        row->grads = s->grads;
        state_stats(s, row);
        row->eps = s->eps;
        row->L = s->L;
        /* Alg. 1: leave the unadjusted loop once every delta is below tol */
        int do_switch = (s->win_n >= s->T) && (maxdel < c->switch_tol);
        if (c->force_switch_at > 0) do_switch = (s->t >= c->force_switch_at);
        if (do_switch && c->adjusted && s->t < c->n_total_steps) {
            switch_to_adjusted(s, var);
            row->eps = s->eps;
            row->L = s->L;
        } else if (s->t >= c->n_total_steps) {
            s->done = 1;
        }
        free(var);
        return 1;
    }

    /* --- Alg. 1, adjusted loop body (one MAMS proposal per chain) --- */
    const int N = c->steps_per_proposal;
    if (s->t + N > c->n_total_steps) { s->done = 1; return 0; }
    row->eps_used = s->eps;
    s->L = c->adj_L_factor * (double)N * s->eps;      /* Sec. 5.2 */
    const uint32_t t0 = (uint32_t)s->t;
#pragma omp parallel
    {
        double* z = (double*)malloc((size_t)d * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t m = 0; m < M; ++m) s->acc[m] = mams_chain(s, m, t0, z);
        free(z);
    }
    s->grads += (long long)N * grads_per_step(s->integ);
    s->t += N;
    s->p += 1;
    double asum = 0.0;
    int nbad = 0;
    for (int64_t m = 0; m < M; ++m) { asum += s->acc[m]; nbad += s->bad[m]; }
    const double a = asum / (double)M;
    /* Sec. 5.1: adapt until |a - a*| <= tol once, then freeze */
    s->adapting = s->adapting && (fabs(a - s->a_target) > c->acc_tol);
    if (s->adapting) s->eps = ora_bisect(s->eps, a, s->a_target, &s->lo, &s->hi);
    s->L = c->adj_L_factor * (double)N * s->eps;
    row->phase = 1;
    row->acc = a;
    row->nonfinite = nbad;
    row->adapting = s->adapting;
    row->t = s->t;
    row->grads = s->grads;
    state_stats(s, row);
    row->eps = s->eps;
    row->L = s->L;
    if (s->t + N > c->n_total_steps) s->done = 1;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* batch helpers for tests (loops over the single-item functions above) */
void ora_philox_batch(int64_t n, const uint32_t* ctrs, const uint32_t key[2], uint32_t* out) {
    for (int64_t k = 0; k < n; ++k) ora_philox4x32_10(ctrs + 4 * k, key, out + 4 * k);
}

void ora_normals_chains(uint64_t seed, uint32_t m0, int64_t nm, uint32_t t, uint32_t tag,
                        uint32_t pid, int64_t d, double* z) {
    for (int64_t k = 0; k < nm; ++k) ora_normals(seed, m0 + (uint32_t)k, t, tag, pid, d, z + k * d);
}

void ora_logp_grad_batch(const ora_target* tg, int64_t M, const double* x, double* logp,
                         double* g) {
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m) logp[m] = ora_logp_grad(tg, x + m * tg->d, g + m * tg->d);
}

int ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* M independent MAMS proposals (chain m uses stream index m) for the
 * stationarity / detailed-balance pins.  mh_mode 0 is App. F as stated; the
 * other modes plant a mistake so a test can show that the pins detect it:
 * 1 accepts every proposal, 2 flips the sign of the energy error. */
void ora_mams_batch(const ora_target* tg, int integ, double eps, double L, int n_steps,
                    uint64_t seed, uint32_t pid, int64_t M, uint32_t t0, uint32_t p,
                    int mh_mode, double* X, double* acc_prob, int* accepted) {
    const int64_t d = tg->d;
#pragma omp parallel
    {
        double* buf = (double*)malloc((size_t)(6 * d) * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t m = 0; m < M; ++m) {
            double* x = X + m * d;
            double* g = buf;
            double lp = ora_logp_grad(tg, x, g);
            acc_prob[m] = mams_core(tg, NULL, integ, eps, L, n_steps, seed, pid, (uint32_t)m, t0,
                                    p, x, g, &lp, buf + d, buf + 2 * d, buf + 3 * d, buf + 4 * d,
                                    buf + 5 * d, mh_mode, &accepted[m], NULL, NULL);
        }
        free(buf);
    }
}
