/*
 * laps_oracle.h -- plain, slow FP64 CPU restatement of LAPS (Late Adjusted
 * Parallel Sampler, Robnik & Seljak).  TEST INFRASTRUCTURE ONLY: it exists so
 * that tests, the smoke check and the benchmark's CPU baseline can compare the
 * CUDA library against an obviously correct implementation.  The product path
 * never links, loads or calls it, and it shares no code with the CUDA sources.
 *
 * Everything is double precision, loops over chains and coordinates, in the
 * order Algorithm 1 and Apps. E-F of the paper state them.  The only thing it
 * has in common with the CUDA path is the *specification* of the random
 * stream (Philox4x32-10 counter layout, uniform mapping and Box-Muller), which
 * each side implements on its own.
 *
 * Parity status per function is listed in the header of laps_oracle.c.
 */
#ifndef LAPS_ORACLE_H
#define LAPS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based random numbers (Philox4x32-10, Salmon et al. 2011) ---- */
enum { ORA_TAG_X0 = 0, ORA_TAG_O1 = 1, ORA_TAG_O2 = 2, ORA_TAG_REFRESH = 3,
       ORA_TAG_MH = 4 };

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* r -> ((r >> 9) + 1/2) * 2^-23, in (0, 1), exactly representable in binary32 */
double ora_uniform(uint32_t r);
/* normals for coordinates 4j..4j+3 of chain m under (t, tag, pid): Box-Muller */
void ora_normals4(uint64_t seed, uint32_t j, uint32_t m, uint32_t t, uint32_t tag,
                  uint32_t pid, double z[4]);
/* d normals for chain m (coordinate i takes block i/4, lane i%4) */
void ora_normals(uint64_t seed, uint32_t m, uint32_t t, uint32_t tag, uint32_t pid,
                 int64_t d, double* z);

/* ---- targets ---- */
enum { ORA_GAUSS_DIAG = 0, ORA_BANANA = 1, ORA_FUNNEL = 2, ORA_LOGREG = 3, ORA_GAUSS_DENSE = 4 };
typedef struct {
    int kind;
    int64_t d;
    const double* prec;      /* GAUSS_DIAG: precision 1/sigma_i^2, [d];
                                GAUSS_DENSE: precision matrix P, row-major [d][d] (symmetric) */
    double banana_sb;        /* BANANA: std of x_b given x_a (0.1) */
    double funnel_sv;        /* FUNNEL: std of v (3) */
    int64_t n_data;          /* LOGREG: number of data rows */
    const double* X;         /* LOGREG: design matrix, row-major [n_data][d] */
    const double* y;         /* LOGREG: labels in {0,1}, [n_data] */
    double prior_var;        /* LOGREG: prior variance of every weight (1) */
} ora_target;

/* log p(x) up to a constant; writes grad log p into g */
double ora_logp_grad(const ora_target* tg, const double* x, double* g);

/* ---- the three maps of App. E ---- */
/* O: u <- (c1 u + c2 z) / |c1 u + c2 z|, c1 = exp(-eps/L), c2 = sqrt(1-c1^2);
 * z is passed in already scaled (std 1/sqrt(d) per coordinate) */
void ora_O(int64_t d, double eps, double L, const double* z, double* u);
/* A: x <- x + eps u */
void ora_A(int64_t d, double eps, const double* u, double* x);
/* B: closed-form isokinetic velocity kick; returns the kinetic energy change
 * (d-1) log(cosh delta + (e.u) sinh delta), delta = eps |g| / (d-1) */
double ora_B(int64_t d, double eps, const double* g, double* u);

/* ---- integrators (Table "integrators", Eq. "integrator") ---- */
enum { ORA_LF = 0, ORA_MN2 = 1, ORA_MN4 = 2 };
/* number of B stages K and the coefficient lists b[K], a[K-1] */
int ora_integrator_coefs(int integ, double* b, double* a);
/* deterministic part Phi_eps: B a B a ... B starting from (x,u,g,logp), which
 * must be consistent (g = grad log p(x)).  Returns the energy error of the
 * step (sum of the A and B contributions). */
double ora_Phi(const ora_target* tg, int integ, double eps, double* x, double* u,
               double* g, double* logp);

/* ---- ensemble estimators ---- */
/* F(D) = 4 D^{3/2} / (1 + D^{1/2})^2  (Eq. "bias bound") */
double ora_F(double D);
/* diagonal equipartition D~_diag of an ensemble (App. B, "Diagonal");
 * X, G are [M][d] positions and gradients */
double ora_dtilde_diag(int64_t M, int64_t d, const double* X, const double* G);
/* full-rank equipartition D~ by Hutchinson's estimator over K Rademacher
 * vectors of step t (App. B, "Full rank"); the vectors' entries are
 * ora_rademacher(seed, pid, t, k, i) */
double ora_rademacher(uint64_t seed, uint32_t pid, uint32_t t, uint32_t k, int64_t i);
double ora_dtilde_full(int64_t M, int64_t d, const double* X, const double* G, int K, uint64_t seed,
                       uint32_t pid, uint32_t t);
/* L = alpha * sqrt(sum_i Var[x_i])  (Eq. "L") */
double ora_L_of(int64_t M, int64_t d, const double* X, double alpha);
/* relative fluctuation sigma/mu of the last T values of a series (Eq.
 * "relative fluctuations"); hist is the window in time order */
double ora_rel_fluct(int64_t T, const double* hist);
/* one bisection update of the adjusted step size (Sec. 5.1); lo/hi <= 0 mean
 * unset.  Returns the new eps. */
double ora_bisect(double eps, double a, double a_target, double* lo, double* hi);

/* ---- LAPS (Algorithm 1) ---- */
typedef struct {
    double C;                 /* asymptotic/total bias ratio, 0.025 */
    double alpha;             /* L = alpha sqrt(sum Var), 2 */
    double switch_tol;        /* max_i delta[x_i^2] threshold, 0.01 */
    double window_frac;       /* T = ceil(window_frac * n_total_steps), 0.2 */
    double acc_tol;           /* bisection tolerance |a - a*|, 0.03 */
    double adj_L_factor;      /* L = adj_L_factor * N * eps, 1.25 */
    double eps0_coef;         /* eps0 = eps0_coef * sqrt(d), 0.01 */
    double a_target_mn2;      /* 0.7 */
    double a_target_mn4;      /* 0.9 */
    int n_total_steps;        /* maxiter, in integrator steps */
    int steps_per_proposal;   /* N = 15 */
    int mn4_min_dim;          /* MN4 when d > mn4_min_dim (200) */
    int eevpd_centered;       /* 1: Var[Delta]/d (Eq. EEVPD); 0: mean Delta^2 / d */
    int adjusted;             /* 0: stop after the unadjusted phase */
    int force_switch_at;      /* >0: switch after this many unadjusted steps */
    double fixed_eps;         /* >0: unadjusted step size held fixed (App. A, Fig. "stepsize") */
    int round_state_f32;      /* 1: round y and u to binary32 after every map and form
                                 logistic-regression logits in binary32, to measure how
                                 binary32 arithmetic perturbs the run (not LAPS) */
    int dtilde_K;             /* > 0: full-rank D~ with this many Rademacher vectors;
                                 0: D~_diag (App. B) */
} ora_config;

void ora_config_default(ora_config* c);

typedef struct {
    int phase;          /* 0 unadjusted, 1 adjusted */
    int t;              /* integrator steps done so far (after this iteration) */
    double eps;         /* step size that will be used next */
    double L;           /* L that will be used next */
    double eps_used;    /* step size the iteration used */
    double eevpd;       /* unadjusted: measured EEVPD of the iteration */
    double eevpd_wanted;
    double dtilde;      /* unadjusted: D~_diag after the iteration */
    double max_delta;   /* unadjusted: max_i delta[x_i^2] (NaN before window full) */
    double acc;         /* adjusted: mean acceptance probability */
    double b2_max, b2_avg;  /* second-moment bias, NaN without truth */
    double sum_var;     /* sum_i Var[x_i] after the iteration (x space) */
    int nonfinite;      /* chains reverted/rejected for non-finite values */
    int adapting;       /* adjusted: bisection still active */
    long long grads;    /* gradient evaluations per chain so far */
} ora_trace_row;

typedef struct ora_state ora_state;

/* x0: [M][d] initial positions (copied).  pid: problem id of the stream. */
ora_state* ora_create(const ora_target* tg, const ora_config* cfg, int64_t M,
                      const double* x0, uint64_t seed, uint32_t pid);
void ora_destroy(ora_state* s);
/* truth for b^2 (E_p[x_i^2] and Var_p[x_i^2]); copied */
void ora_set_truth(ora_state* s, const double* Ex2, const double* Varx2);
/* initial trace row (after initialisation) */
void ora_row0(const ora_state* s, ora_trace_row* row);
/* one iteration of Algorithm 1: an unadjusted step, or one MAMS proposal.
 * Returns 1 if an iteration ran, 0 if the run is finished. */
int ora_iterate(ora_state* s, ora_trace_row* row);
/* chain positions in the original (x) coordinates, [M][d] */
void ora_get_x(const ora_state* s, double* x_out);
/* sampler-coordinate state (y = x / sigma after the switch), [M][d] */
void ora_get_state(const ora_state* s, double* y, double* u, double* g, double* logp);
void ora_get_sigma(const ora_state* s, double* sigma);
int ora_phase(const ora_state* s);
int ora_t(const ora_state* s);
int ora_t_switch(const ora_state* s);
int ora_window_T(const ora_state* s);
int ora_integrator(const ora_state* s);

/* ---- a single MAMS proposal for one chain (App. F), noise drawn from the
 * stream of chain m, proposal index p, integrator steps starting at t0.
 * Updates x, g, logp in place (restored on reject); returns the acceptance
 * probability min(1, exp(-Delta)) and sets *accepted. */
double ora_mams_proposal(const ora_target* tg, int integ, double eps, double L,
                         int n_steps, uint64_t seed, uint32_t pid, uint32_t m,
                         uint32_t t0, uint32_t p, double* x, double* g,
                         double* logp, double* u_work, int* accepted,
                         double* delta_out);

/* ---- batch helpers for tests ---- */
void ora_philox_batch(int64_t n, const uint32_t* ctrs, const uint32_t key[2], uint32_t* out);
void ora_normals_chains(uint64_t seed, uint32_t m0, int64_t nm, uint32_t t, uint32_t tag,
                        uint32_t pid, int64_t d, double* z);
void ora_logp_grad_batch(const ora_target* tg, int64_t M, const double* x, double* logp,
                         double* g);
/* M independent MAMS proposals from the rows of X ([M][d], updated in place);
 * mh_mode 0: App. F; 1: accept all (planted mistake); 2: sign of Delta
 * flipped (planted mistake).  Used by the exactness pins. */
void ora_mams_batch(const ora_target* tg, int integ, double eps, double L, int n_steps,
                    uint64_t seed, uint32_t pid, int64_t M, uint32_t t0, uint32_t p,
                    int mh_mode, double* X, double* acc_prob, int* accepted);
/* OpenMP threads for the per-chain loops (<= 0: leave); returns the count */
int ora_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
