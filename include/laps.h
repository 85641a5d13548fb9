/*
 * laps.h -- C ABI of the GB300 (sm_103a) LAPS library, liblaps.so.
 *
 * LAPS (Late Adjusted Parallel Sampler; Robnik & Seljak, "Faster parallel
 * MCMC: Metropolis adjustment is best served warm") advances an ensemble of M
 * chains of a d-dimensional target: first by unadjusted microcanonical
 * Langevin (MCLMC) steps whose step size follows the ensemble's bias estimate
 * (Sec. 3), then, after the switch rule of Sec. 4 and a diagonal
 * preconditioner, by Metropolis-adjusted proposals (MAMS, App. F) whose step
 * size is bisected to a target acceptance (Sec. 5).  Algorithm 1 (App. C)
 * states the loop this library runs.  Per the paper's statement of the
 * problem (Sec. 1 "Our contributions", Alg. 1 input) the user supplies the
 * target log-density with its gradient and the initial positions.
 *
 * Conventions (every entry point):
 *  - Return laps_status; nothing throws across the ABI.  laps_last_error()
 *    gives a thread-local message for the last failing call.
 *  - Pointers named "device" are CUDA device pointers owned by the caller; the
 *    library never frees them.  "host" pointers are plain host memory.
 *  - Arrays are row-major, chain-major and contiguous: x[m*d + i] is
 *    coordinate i of chain m, FP32.  A device pointer that is not 4-byte
 *    aligned returns LAPS_ERR_INVALID_ARG.
 *  - All GPU work is ordered on the cudaStream_t argument (pass it as a
 *    void*; NULL is the legacy default stream).  These calls block the host:
 *     - set-up calls that allocate or copy host arrays in: laps_target_create,
 *       laps_create, laps_set_truth, laps_batch_create, laps_batch_set_truth,
 *       laps_batch_set_shape, laps_batch_set_ids (device-synchronous);
 *     - calls that read results back: laps_get_stats, laps_get_trace,
 *       laps_checkpoint, laps_restore, laps_adapt_freeze, laps_target_status,
 *       laps_batch_get_stats, laps_batch_get_trace, laps_batch_tune,
 *       laps_measure_peaks, and laps_run_noalloc when stats_out is not NULL;
 *     - laps_step and laps_run of a context on the streamed path (a LOGREG or
 *       USER target, a GAUSS_DENSE target beyond d = 128 or with
 *       dense_streamed): the host enqueues a different launch sequence for an
 *       unadjusted step and for a MAMS proposal, so it reads the phase machine
 *       back (a stream synchronisation) every 32 unadjusted iterations or 4
 *       proposals, and at the switch.
 *    Every other call (laps_init, laps_step and laps_run of the
 *    register-resident path, laps_sample, laps_get_state, laps_philox,
 *    laps_normals, laps_target_logp_grad[_prec], laps_batch_init,
 *    laps_batch_step, laps_batch_run, laps_batch_sample) only enqueues work
 *    and returns; laps_batch_partition is host arithmetic and touches no GPU.
 *  - Errors raised inside a kernel (a bounded wait that expired, a bad
 *    parameter) are latched in a device status word and returned by the next
 *    call that reads it (laps_get_stats, or any synchronising call).
 *  - A laps_ctx is not thread-safe; different contexts are independent.
 */
#ifndef LAPS_H
#define LAPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LAPS_OK = 0,
    LAPS_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or config value */
    LAPS_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has details) */
    LAPS_ERR_OOM = 3,           /* device allocation failed */
    LAPS_ERR_TIMEOUT = 4,       /* a bounded device-side wait (grid barrier) expired */
    LAPS_ERR_NONFINITE = 5,     /* every chain produced non-finite values */
    LAPS_ERR_UNSUPPORTED = 6    /* shape/target combination not built */
} laps_status;

/* Targets with hand-written log-density and gradient kernels. */
typedef enum {
    LAPS_GAUSS_DIAG = 0,  /* log p = -1/2 sum_i prec_i x_i^2 */
    LAPS_BANANA = 1,      /* pairs (a,b) = (x_2k, x_2k+1): a ~ N(0,1), b|a ~ N(a^2, sb^2); d even */
    LAPS_FUNNEL = 2,      /* v = x_0 ~ N(0, sv^2), x_i|v ~ N(0, e^v), i = 1..d-1 */
    LAPS_LOGREG = 3,      /* sum_n [y_n z_n - softplus(z_n)] - |w|^2/(2 prior_var), z = X w */
    LAPS_GAUSS_DENSE = 4, /* -1/2 x^T P x with a dense symmetric positive-definite precision P
                             (Sec. 6, the randomly oriented ill-conditioned Gaussian); d <= 512;
                             sampled on the streamed path, its gradient -P x as one
                             chains-by-coordinates contraction per step */
    LAPS_USER = 5         /* the caller's log-density: user_fn (below) evaluates it and its
                             gradient for the ensemble's points at every gradient evaluation;
                             d <= 512; sampled on the streamed path */
} laps_target_kind;

/* Log-density of a LAPS_USER target (Sec. 1: the user supplies log p and its
 * gradient).  Called on the host thread that enqueues the sampler's work,
 * once per gradient evaluation of the ensemble (not fused with the chain
 * updates).  x: device [M][ld] points, row stride ld >= d floats, entries
 * past d are zero; logp: device [M] output; grad: device [M][ld] output,
 * entries past d ignored.  The function must enqueue its work on `stream`
 * (a cudaStream_t), must not synchronise it, and must not keep the pointers
 * after it returns.  Return 0 on success; any other value makes the calling
 * laps entry point return LAPS_ERR_CUDA with a message naming the callback. */
typedef int (*laps_logp_grad_fn)(const float* x, int64_t M, int64_t ld, float* logp, float* grad,
                                 void* stream, void* user_data);

/* Arithmetic of the logistic-regression contraction in each phase.  The
   tensor-core forms are built for d <= 128. */
typedef enum {
    LAPS_FP32 = 0,          /* FP32 on the CUDA cores in both phases */
    LAPS_MIXED = 1,         /* BF16 tensor-core contraction (FP32 accumulate) while unadjusted,
                               FP32 on the CUDA cores once adjusted */
    LAPS_BF16X3 = 2,        /* tensor cores at FP32 accuracy in both phases: every operand as
                               three BF16 terms, the six cross products of order >= 2^-16 */
    LAPS_MIXED_BF16X3 = 3   /* BF16 tensor-core contraction while unadjusted, the three-term
                               form of LAPS_BF16X3 once adjusted */
} laps_precision;

typedef struct {
    laps_target_kind kind;
    int64_t d;              /* dimension, >= 2 */
    const float* prec;      /* GAUSS_DIAG: device [d] precisions 1/sigma_i^2;
                               GAUSS_DENSE: device [d][d] precision matrix, row-major, symmetric
                               (the target keeps its own zero-padded copy) */
    double banana_sb;       /* BANANA: conditional std of x_b (0.1) */
    double funnel_sv;       /* FUNNEL: std of v (3) */
    int64_t n_data;         /* LOGREG: rows of X */
    const float* X;         /* LOGREG: device [n_data][d] design matrix (intercept included) */
    const float* y;         /* LOGREG: device [n_data] labels in {0, 1} */
    double prior_var;       /* LOGREG: prior variance of each weight (1) */
    laps_logp_grad_fn user_fn; /* USER: the log-density callback */
    void* user_data;        /* USER: passed to user_fn unchanged */
} laps_target_desc;

typedef struct laps_target laps_target;
typedef struct laps_ctx laps_ctx;

/* Algorithm settings; laps_config_default fills the paper's values. */
typedef struct {
    double C;                /* asymptotic / total bias ratio, 0.025 (Sec. 3.1) */
    double alpha;            /* L = alpha sqrt(sum_i Var x_i), 2 (Eq. "L") */
    double switch_tol;       /* switch when max_i delta[x_i^2] < tol, 0.01 (Sec. 4) */
    double window_frac;      /* window T = ceil(window_frac * n_total_steps), 0.2 (Sec. 4) */
    double acc_tol;          /* stop bisecting once |a - a*| <= acc_tol, 0.03 (Sec. 5.1) */
    double adj_L_factor;     /* adjusted L = adj_L_factor * N * eps, 1.25 (Sec. 5.2) */
    double eps0_coef;        /* eps0 = eps0_coef * sqrt(d), 0.01 (Alg. 1) */
    double a_target_mn2;     /* target acceptance with MN2, 0.7 (Sec. 5.1) */
    double a_target_mn4;     /* target acceptance with MN4, 0.9 (Sec. 5.1) */
    int n_total_steps;       /* maxiter in integrator steps (Alg. 1) */
    int steps_per_proposal;  /* N = 15 (Sec. 5.2) */
    int mn4_min_dim;         /* MN4 when d > mn4_min_dim, 200 (App. E) */
    int eevpd_centered;      /* 1: EEVPD = Var[Delta]/d (Eq. EEVPD); 0: mean Delta^2/d (Alg. 1) */
    int adjusted;            /* 0: never switch (unadjusted only) */
    int force_switch_at;     /* > 0: switch after exactly this many unadjusted steps */
    double fixed_eps;        /* > 0: unadjusted step size held at this value (the fixed-step
                                comparison of App. A, Fig. "stepsize"); 0: Sec. 3.1 controller */
    double stop_b2;          /* > 0 (needs laps_set_truth): finish once b^2 < stop_b2 */
    int stop_b2_max;         /* 0: use b^2_avg for stop_b2; 1: use b^2_max */
    laps_precision precision;
    int64_t barrier_timeout_ns;  /* bound of every device-side wait; default 2e9 */
    int chains_per_block;    /* 0: chosen by the library; else chains per thread block */
    int lanes_per_chain;     /* 0: chosen; else 4, 8, 16 or 32 lanes hold one chain */
    int coords_per_lane;     /* 0: chosen; else 4, 8 or 16 coordinates per lane */
    int barrier_extra_arrivals;  /* test hook, 0 in use: every grid barrier also waits for
                                    this many arrivals that never come, so its bounded wait
                                    expires and the launch ends with LAPS_ERR_TIMEOUT */
    int dtilde_K;            /* 0: the diagonal bias proxy D~_diag (App. B, the paper's default);
                                K > 0: the full-rank D~ by Hutchinson's estimator over K
                                Rademacher vectors per step (App. B "Full rank"; the paper
                                uses 100); register-resident targets only */
    int dense_streamed;      /* GAUSS_DENSE: 0 runs the register-resident kernel (P in shared
                                memory) when d <= 128 and the streamed path beyond; 1 always
                                the streamed path */
} laps_config;

/* Snapshot of the sampler (laps_get_stats). */
typedef struct {
    int phase;               /* 0 unadjusted, 1 adjusted */
    int t;                   /* integrator steps taken */
    int t_switch;            /* step of the switch, -1 before */
    int integrator;          /* 0 LF, 1 MN2, 2 MN4 */
    int adapting;            /* adjusted phase: bisection still active */
    int done;                /* the run reached n_total_steps or stop_b2 */
    int iterations;          /* Alg. 1 loop iterations run (steps or proposals) */
    int nonfinite_total;     /* chain updates reverted/rejected for non-finite values */
    long long grads;         /* gradient evaluations per chain so far (init included) */
    double eps, L;           /* hyperparameters of the next iteration */
    double eevpd, eevpd_wanted, dtilde, max_delta; /* last unadjusted iteration */
    double acc;              /* last adjusted iteration: mean acceptance probability */
    double b2_max, b2_avg;   /* current second-moment bias (NaN without truth) */
    double sum_var;          /* sum_i Var[x_i] of the current ensemble */
    int b2_first_t;          /* first t with b^2 (stop kind) < 0.01, -1 if never */
    long long b2_first_grads;
    double b2_first_ns;      /* device time from the start of laps_init to that row */
} laps_stats;

/* One row per Alg. 1 iteration; row 0 describes the initial ensemble. */
typedef struct {
    int phase, t;
    double eps, L, eps_used, eevpd, eevpd_wanted, dtilde, max_delta, acc;
    double b2_max, b2_avg, sum_var;
    int nonfinite, adapting;
    long long grads;
    double time_ns;          /* device %globaltimer relative to laps_init */
} laps_trace_row;

void laps_config_default(laps_config* cfg);
const char* laps_last_error(void);
const char* laps_version(void);

/* ---- targets ------------------------------------------------------------
 * laps_target_create copies the descriptor (the device arrays it points to
 * must outlive the target; LOGREG keeps BF16/FP32 copies of X it owns). */
laps_status laps_target_create(const laps_target_desc* desc, laps_target** out);
void laps_target_destroy(laps_target* tg);

/* log p and grad log p of M points: x device [M][d], logp device [M],
 * grad device [M][d] (M = 0: nothing is done and the pointers may be NULL).  Forward and hand-written backward of the target (the
 * kernels the sampler uses), FP32 in and out with compensated sums. */
laps_status laps_target_logp_grad(const laps_target* tg, const float* x, int64_t M,
                                  float* logp, float* grad, void* stream);
/* The same in a given arithmetic: LAPS_FP32 is laps_target_logp_grad;
 * LAPS_MIXED (LOGREG with d <= 128) is the tensor-core form the sampler's
 * unadjusted phase uses: the target on the BF16-rounded data, each point as a
 * sum of two BF16 terms, residuals y - sigmoid(z) in BF16, FP32 accumulation;
 * LAPS_BF16X3 (LOGREG with d <= 128) is the tensor-core form at FP32
 * accuracy: points, data and residuals each as three BF16 terms, the six
 * cross products of order >= 2^-16, FP32 accumulation, the FP32 epilogue of
 * laps_target_logp_grad.  Stream-ordered; a bounded device wait that expired is latched in the
 * target's status word, which laps_target_status returns. */
laps_status laps_target_logp_grad_prec(const laps_target* tg, const float* x, int64_t M,
                                       float* logp, float* grad, int precision, void* stream);
/* Synchronises the device, returns and clears the target's latched status. */
laps_status laps_target_status(laps_target* tg);

/* ---- one sampling problem ---------------------------------------------- */
/* Allocates the ensemble state (x, u, g, log p in the sampler's layout), the
 * reduction scratch, the moving window of Sec. 4 and the trace.  The target
 * must outlive the context. */
laps_status laps_create(const laps_target* tg, int64_t M, const laps_config* cfg,
                        laps_ctx** out);
void laps_destroy(laps_ctx* ctx);

/* Alg. 1 initialisation: x0 device [M][d] (copied), or NULL to draw
 * x0 = x0_scale * N(0, I) from the Philox stream (tag 0) of `seed`; then
 * g0, log p0, u0 = g0/|g0|, eps0 = eps0_coef sqrt(d), L0 = Eq. "L". */
laps_status laps_init(laps_ctx* ctx, const float* x0, double x0_scale, uint64_t seed,
                      void* stream);

/* Runs up to n_iters iterations of Alg. 1 (an unadjusted step, or one MAMS
 * proposal of N steps), fewer if the run finishes.  One cooperative launch. */
laps_status laps_step(laps_ctx* ctx, int n_iters, void* stream);

/* Runs to the end (n_total_steps, or stop_b2). */
laps_status laps_run(laps_ctx* ctx, void* stream);

/* Freezes (frozen = 1) or re-enables the adjusted-phase bisection. */
laps_status laps_adapt_freeze(laps_ctx* ctx, int frozen);

/* Chain positions in the target's coordinates (x = sigma o y after the
 * switch): x_out device [M][d]. */
laps_status laps_sample(const laps_ctx* ctx, float* x_out, void* stream);

/* Raw sampler state in sampler coordinates: y, u, grad_y device [M][d] and
 * logp device [M] (double); sigma device [d] (1 before the switch).  Any
 * pointer may be NULL. */
laps_status laps_get_state(const laps_ctx* ctx, float* y, float* u, float* g, double* logp,
                           float* sigma, void* stream);

/* Truth for b^2 (Eq. "bias"): Ex2, Varx2 host [d] = E_p[x_i^2], Var_p[x_i^2]. */
laps_status laps_set_truth(laps_ctx* ctx, const double* Ex2, const double* Varx2);

/* Synchronises the stream of the last launch, then reports. */
laps_status laps_get_stats(laps_ctx* ctx, laps_stats* out);
/* Copies up to cap rows (row 0 = initial ensemble); *n = rows available. */
laps_status laps_get_trace(laps_ctx* ctx, laps_trace_row* rows, int cap, int* n);

/* Checkpoint of everything the run depends on (state, hyperparameters,
 * window, preconditioner, trace, seed).  host_blob NULL: *size = bytes
 * needed.  Restoring into a context created with the same target, M and
 * config continues bit-exactly (the random stream is a function of t). */
laps_status laps_checkpoint(laps_ctx* ctx, void* host_blob, size_t* size);
laps_status laps_restore(laps_ctx* ctx, const void* host_blob, size_t size);

/* ---- the random stream --------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11): ctr device [n][4] counters, key =
 * (seed low word, seed high word), out device [n][4].  The sampler draws with
 * counter (coordinate block j, chain m, step t, tag | pid << 8); tags: 0
 * initial positions, 1 first O map of a step, 2 second O map, 3 full velocity
 * refresh of a MAMS proposal (t = proposal index), 4 Metropolis uniform
 * (j = 0, t = proposal index). */
laps_status laps_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                        void* stream);
/* The sampler's standard normals: out device [nm][d] for chains m0..m0+nm-1
 * under (t, tag, pid); coordinate i uses block i/4, Box-Muller pair (i%4)/2,
 * uniforms ((r >> 9) + 1/2) 2^-23. */
laps_status laps_normals(uint64_t seed, uint32_t m0, int64_t nm, uint32_t t, uint32_t tag,
                         uint32_t pid, int64_t d, float* out, void* stream);

/* ---- a run that allocates nothing ---------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (a process whose device memory belongs to a pool
 * allocator that reserved the GPU at start-up, code that must not add the
 * device-wide synchronisation cudaMalloc/cudaFree imply, a plug-in that may
 * not grow the device footprint after loading).
 * One complete run (laps_init with x0 / x0_scale / seed, then laps_run) of a
 * GAUSS_DIAG, BANANA or FUNNEL target described by desc (its device arrays
 * are read, not copied into any allocation), in FP32 (cfg->precision must be
 * LAPS_FP32, cfg->stop_b2 0 and cfg->dtilde_K 0, else LAPS_ERR_UNSUPPORTED);
 * the samples go to x_out device [M][d].  With stats_out NULL the call only
 * enqueues work on the stream; otherwise it synchronises the stream and fills
 * stats_out.  No trace is kept and laps_set_truth does not apply (b^2 fields
 * NaN).
 * All scratch lives in one fixed 16 MiB __device__ array of the library, held
 * on a device until the process exits once the library's device code is
 * loaded there.  Under CUDA's lazy module loading (the default) that happens
 * at the first call on the device, so that call may still grow the device
 * footprint: a caller that hands the rest of the device to a pool should make
 * it first, or make the set-up-only call laps_run_noalloc(NULL, 0, NULL, NULL,
 * 0, 0, NULL, NULL, NULL), which loads the array and looks up its address and
 * does nothing else (CUDA_MODULE_LOADING=EAGER loads it when the library is
 * loaded instead).  A problem needing more (about 12 M d bytes of state plus
 * the window and reduction buffers) returns LAPS_ERR_INVALID_ARG before any
 * launch.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it: make that first call before any
 * stream capture, and do not cudaDeviceReset a device this entry point has
 * run on (the cached address would be stale).  Every call on a device shares
 * the array and clears what must start at zero; calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised. */
laps_status laps_run_noalloc(const laps_target_desc* desc, int64_t M, const laps_config* cfg,
                             const float* x0, double x0_scale, uint64_t seed, float* x_out,
                             laps_stats* stats_out, void* stream);

/* ---- a chain-sharded ensemble ------------------------------------------
 * Chains are independent between the ensemble reductions (Sec. 2, Eq. "ECA";
 * Alg. 1), so one ensemble of M_total chains can be split over ranks (one
 * process per GPU): each rank advances its own chains m0 .. m0 + M_local - 1
 * (their Philox counters carry the global chain index, so the union of the
 * ranks' chains is the unsharded ensemble) and, once per Alg. 1 iteration,
 * exchanges only its totals of the per-coordinate and per-chain sums the
 * finalise needs (4 d_pad + 5 float-float pairs).  Every rank then adds the
 * totals in rank order and runs the identical finalise, so every rank holds
 * the same step size, L, window and phase machine.
 * The exchange is the caller's: allgather(send, recv, bytes, stream, user)
 * must gather `bytes` of device memory from every rank's `send` into `recv`
 * [n_ranks][bytes], in rank order, stream-ordered on `stream` (e.g. an NCCL
 * all-gather), and return 0; it is called on the host thread that enqueues the
 * iteration, once per iteration (also for the initialisation).  With
 * n_ranks = 1 it may be NULL (a local copy), and that rank holds the whole
 * ensemble (m0 = 0, M_local = M_total).  Served on the streamed path:
 * LOGREG and USER targets, GAUSS_DENSE beyond d = 128 or with dense_streamed;
 * other targets return LAPS_ERR_UNSUPPORTED.  With one rank the results equal
 * laps_create's bit for bit. */
typedef int (*laps_allgather_fn)(const void* send, void* recv, size_t bytes, void* stream,
                                 void* user_data);
typedef struct {
    int64_t M_total;             /* chains of the whole ensemble */
    int64_t m0;                  /* global index of this rank's first chain */
    int rank, n_ranks;
    laps_allgather_fn allgather;
    void* user_data;             /* passed to allgather unchanged */
} laps_shard;
laps_status laps_create_sharded(const laps_target* tg, int64_t M_local, const laps_shard* shard,
                                const laps_config* cfg, laps_ctx** out);

/* Launch shape the context uses (for tests and the autotuner). */
typedef struct {
    int chains_per_block, lanes_per_chain, coords_per_lane, threads, blocks;
    int resident;            /* 1: register-resident persistent kernel */
} laps_launch_info;
laps_status laps_get_launch_info(const laps_ctx* ctx, laps_launch_info* out);

/* Throughput probes of the current GPU, the denominators of the kernels'
 * roofline fractions at the clock the GPU actually runs at: FP32 and FP64
 * fused multiply-add throughput over all SMs, the special-function unit's
 * base-2 exponential per clock and SM, and the latency of the grid-wide
 * barrier the persistent kernels use (one block per SM, cooperative launch).
 * Each probe is timed with CUDA events on `stream` after one warm-up launch;
 * the call synchronises the stream and takes a few milliseconds.  Returns
 * LAPS_ERR_TIMEOUT if a barrier wait expired (2 s bound). */
typedef struct {
    int sm_count;
    double sm_mhz;            /* SM clock during the FP32 probe (cycle counter / global timer) */
    double fp32_tflops;       /* FFMA, 2 FLOP each */
    double fp64_tflops;       /* DFMA, 2 FLOP each */
    double ex2_per_clk_sm;    /* ex2.approx.f32 results per clock per SM */
    double grid_barrier_us;   /* one grid barrier of barrier_blocks blocks */
    int barrier_blocks;
} laps_peaks;
laps_status laps_measure_peaks(laps_peaks* out, void* stream);

/* ---- many problems in one launch -----------------------------------------
 * A batch of independent diagonal-Gaussian problems of uneven dimension and
 * ensemble size (the paper runs one problem per call; batching is this
 * library's: Alg. 1 runs for every problem in lockstep iterations inside one
 * persistent cooperative launch).  Problem k draws from the Philox stream of
 * the batch seed with problem id pid = k, so it reproduces a single-problem
 * run of the same seed and pid up to the order of the ensemble sums.  The
 * state streams from device memory (y and u per chain; the gradient and the
 * energy error are recomputed), so any d up to 10240 is served. */
typedef struct laps_batch laps_batch;
typedef struct {
    int64_t d;              /* dimension, 2 .. 10240 */
    int64_t M;              /* chains, >= 2 */
    const float* prec;      /* device [d]: precisions 1/sigma_i^2 (copied) */
    const float* x0;        /* device [M][d] initial positions (read at laps_batch_init),
                               or NULL for x0_scale N(0, I) from the Philox tag-0 stream */
    double x0_scale;
} laps_problem;

/* Shape of the persistent launch: coordinates per lane (8, 12, 16, 20),
 * warps per chain widened 2^widen times beyond the smallest that holds d,
 * coordinates per reduction slice task.  laps_batch_tune sets it. */
typedef struct {
    int coords_per_lane, widen, slice;
    int threads, blocks;    /* read only */
    int tuned;              /* 1 once laps_batch_tune chose it */
} laps_batch_shape;

/* Allocates every problem's state with cfg (n_total_steps, N, ... shared). */
laps_status laps_batch_create(const laps_problem* probs, int n, const laps_config* cfg,
                              laps_batch** out);
void laps_batch_destroy(laps_batch* b);
/* Truth for problem k's b^2 (host [d] arrays, as laps_set_truth). */
laps_status laps_batch_set_truth(laps_batch* b, int k, const double* Ex2, const double* Varx2);
/* Initialises every problem (Alg. 1 first lines); one launch. */
laps_status laps_batch_init(laps_batch* b, uint64_t seed, void* stream);
/* Up to n_iters lockstep iterations in one persistent launch (a problem that
 * finished idles).  Capturable in a CUDA graph. */
laps_status laps_batch_step(laps_batch* b, int n_iters, void* stream);
/* Runs every problem to its end: a CUDA graph of one launch of
 * iters_per_launch iterations, replayed n_total_steps / iters_per_launch + 2
 * times (enough for a run that never switches); a launch that finds every
 * problem done returns at once.  Enqueues only: read the outcome with
 * laps_batch_get_stats. */
laps_status laps_batch_run(laps_batch* b, int iters_per_launch, void* stream);
/* Autotuner: times every feasible shape for two iterations from the current
 * state (restored afterwards) and keeps the fastest; synchronises. */
laps_status laps_batch_tune(laps_batch* b, void* stream);
laps_status laps_batch_get_shape(const laps_batch* b, laps_batch_shape* out);
laps_status laps_batch_set_shape(laps_batch* b, const laps_batch_shape* shape);
/* Per problem, as the single-problem calls (these synchronise). */
laps_status laps_batch_get_stats(laps_batch* b, int k, laps_stats* out);
laps_status laps_batch_get_trace(laps_batch* b, int k, laps_trace_row* rows, int cap, int* n);
/* Problem k's chain positions x = sigma o y: x_out device [M_k][d_k]. */
laps_status laps_batch_sample(laps_batch* b, int k, float* x_out, void* stream);

/* ---- a batch split over ranks by problems ---------------------------------
 * The problems of a batch are independent, so ranks (one GPU each) can run
 * disjoint sub-batches with no exchange at all.  laps_batch_partition assigns
 * problem k (d[k], M[k], host arrays [n]) to rank owner[k] (host [n], written)
 * by longest processing time first on the cost d_pad M: problems by falling
 * cost, ties by lower index, each to the least-loaded rank, ties by lower
 * rank.  Deterministic, so every rank computes the same owner array.  The
 * largest rank load is at most the total / n_ranks plus the largest cost.
 * INVALID_ARG on null arrays, n < 1, n_ranks < 1 or a non-positive d or M.
 *
 * laps_batch_set_ids gives problem k of b the Philox problem id ids[k] (host
 * [n] int32, distinct, in [0, 2^24); the default is k), so a problem drawn
 * into a sub-batch under its index in the whole batch draws the same noise as
 * in the whole batch.  Device-synchronous (it rewrites the parameter blocks);
 * takes effect at the next launch.  INVALID_ARG on null arguments, ids out of
 * range or repeated. */
laps_status laps_batch_partition(const int64_t* d, const int64_t* M, int n, int n_ranks, int32_t* owner);
laps_status laps_batch_set_ids(laps_batch* b, const int32_t* ids);

#ifdef __cplusplus
}
#endif
#endif
