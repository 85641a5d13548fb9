// laps_api.cu -- host side of the C ABI declared in include/laps.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "laps_internal.h"

namespace laps {
const void* resident_kernel_0(int lpc, int cpl, bool fr);
const void* resident_kernel_1(int lpc, int cpl, bool fr);
const void* resident_kernel_2(int lpc, int cpl, bool fr);
const void* resident_kernel_4(int lpc, int cpl, bool fr);

static thread_local std::string g_err;

cudaError_t ensure_dyn_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> granted;
    std::lock_guard<std::mutex> lock(mu);
    size_t& g = granted[fn];
    if (bytes <= g) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g = bytes;
    return e;
}

laps_status fail(laps_status st, const std::string& msg) {
    g_err = msg;
    return st;
}
laps_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LAPS_ERR_OOM : LAPS_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

static const void* resident_fn(int kind, int lpc, int cpl, bool fr) {
    switch (kind) {
    case TGT_GAUSS: return resident_kernel_0(lpc, cpl, fr);
    case TGT_BANANA: return resident_kernel_1(lpc, cpl, fr);
    case TGT_FUNNEL: return resident_kernel_2(lpc, cpl, fr);
    case TGT_GAUSS_DENSE: return resident_kernel_4(lpc, cpl, fr);
    }
    return nullptr;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ------------------------------------------------------------------ small kernels
__global__ void unpack_rows_kernel(const float* __restrict__ src, const float* __restrict__ scale,
                                   float* __restrict__ dst, int64_t M, int d, int d_pad) {
    const int64_t n = M * (int64_t)d;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k / d;
        const int i = (int)(k - m * d);
        dst[k] = (scale ? scale[i] : 1.0f) * src[m * d_pad + i];
    }
}
__global__ void ff_to_double_kernel(const float2* __restrict__ src, double* __restrict__ dst,
                                    int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = (double)src[k].x + (double)src[k].y;
}
__global__ void fill_kernel(float* p, float v, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        p[k] = v;
}
// the start of a run: the phase machine (taken by value, so no host memory is
// referenced once the launch is enqueued), the status word and sigma = 1
__global__ void run_start_kernel(Hyper* hyper, const Hyper h, int* status, float* sigma, int64_t d_pad) {
    const int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k0 == 0) {
        *hyper = h;
        *status = 0;
    }
    for (int64_t k = k0; k < d_pad; k += (int64_t)gridDim.x * blockDim.x) sigma[k] = 1.0f;
}
__global__ void set_coefs_kernel(Coefs* dst, const Coefs cf) { *dst = cf; }

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

void launch_fill(float* p, float v, int64_t n, cudaStream_t st) {
    fill_kernel<<<grid_for(n), 256, 0, st>>>(p, v, n);
}
void launch_set_coefs(Coefs* dst, const Coefs& cf, cudaStream_t st) {
    set_coefs_kernel<<<1, 1, 0, st>>>(dst, cf);
}
void launch_unpack(const float* src, const float* scale, float* dst, int64_t M, int d, int d_pad,
                   cudaStream_t st) {
    unpack_rows_kernel<<<grid_for(M * d), 256, 0, st>>>(src, scale, dst, M, d, d_pad);
}

void coefs_table(Coefs& cf) {
    std::memset(&cf, 0, sizeof(cf));
    // LF: B_{eps/2} A_eps B_{eps/2}
    cf.K[INTEG_LF] = 2;
    cf.b[INTEG_LF][0] = 0.5f; cf.b[INTEG_LF][1] = 0.5f;
    cf.a[INTEG_LF][0] = 1.0f;
    // MN2 (Omelyan minimal norm, second order): b1, 1/2, b2 = 1 - 2 b1, 1/2, b1
    const double m2b1 = 0.1931833275;
    cf.K[INTEG_MN2] = 3;
    cf.b[INTEG_MN2][0] = (float)m2b1; cf.b[INTEG_MN2][1] = (float)(1.0 - 2.0 * m2b1);
    cf.b[INTEG_MN2][2] = (float)m2b1;
    cf.a[INTEG_MN2][0] = 0.5f; cf.a[INTEG_MN2][1] = 0.5f;
    // MN4: b1 a1 b2 a2 b3 a3 b3 a2 b2 a1 b1; b3 and a3 from sum b = sum a = 1
    const double b1 = 0.0839831526, b2 = 0.6822365335, a1 = 0.2539785108, a2 = -0.032302867;
    const double b3 = 0.5 - b1 - b2, a3 = 1.0 - 2.0 * (a1 + a2);
    const double bb[6] = {b1, b2, b3, b3, b2, b1}, aa[5] = {a1, a2, a3, a2, a1};
    cf.K[INTEG_MN4] = 6;
    for (int k = 0; k < 6; ++k) cf.b[INTEG_MN4][k] = (float)bb[k];
    for (int k = 0; k < 5; ++k) cf.a[INTEG_MN4][k] = (float)aa[k];
}

// ------------------------------------------------------------------ launch shape
static const int kShapes[][2] = {{4, 4}, {8, 4}, {8, 8}, {16, 4}, {16, 8}, {32, 4}, {32, 8}, {32, 16}};

// per-coordinate quantities reduced per shared-memory pass (all four when they fit)
static int resident_qpp(int d_pad, int threads) {
    const size_t per_q = (size_t)(threads / 32) * d_pad * sizeof(float);
    int q = (int)std::min<size_t>(NQ, (64 * 1024) / std::max<size_t>(per_q, 1));
    return std::max(1, q);
}
// largest slice of coordinates a block owns in the reduction
static int resident_smax(int d, int G) { return (d + G - 1) / G; }
static size_t resident_smem(int d_pad, int threads, int lpc, int smax, int K, int kind) {
    const int nwarps = threads / 32, slots = threads / lpc;
    const int qpp = resident_qpp(d_pad, threads);
    size_t b = (size_t)qpp * nwarps * d_pad * sizeof(float) + (size_t)slots * NCSF * sizeof(float) +
               (size_t)d_pad * sizeof(float) + ((size_t)NQ * smax + NCS) * sizeof(float2);
    if (kind == TGT_GAUSS_DENSE) b += dense_smem(d_pad, slots);
    return b + fullrank_smem(d_pad, slots, smax, K, threads);
}

laps_status choose_shape(laps_ctx* c) {
    int dev;
    CK(cudaGetDevice(&dev));
    int nsm;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int kind = c->tg->kind;
    struct Cand { int lpc, cpl, threads, G; size_t smem; double score; };
    Cand ok[3 * sizeof(kShapes) / sizeof(kShapes[0])];  // fixed storage: no heap use
    int n_ok = 0;
    for (auto& sh : kShapes) {
        const int lpc = sh[0], cpl = sh[1];
        if (lpc * cpl < c->d_pad) continue;
        if (c->cfg.lanes_per_chain && lpc != c->cfg.lanes_per_chain) continue;
        if (c->cfg.coords_per_lane && cpl != c->cfg.coords_per_lane) continue;
        const void* fn = resident_fn(kind, lpc, cpl, c->cfg.dtilde_K > 0);
        if (!fn) continue;
        std::vector<int> tlist;
        if (c->cfg.chains_per_block > 0) tlist.push_back(c->cfg.chains_per_block * lpc);
        else tlist = {128, 256, 512};
        for (int threads : tlist) {
            if (threads < 32 || threads > kMaxThreads || threads % 32) continue;
            // the full-rank proxy keeps one coordinate of its shifts per thread
            if (c->cfg.dtilde_K > 0 && threads < c->d_pad) continue;
            const int cpb = threads / lpc;
            const int G = (int)((c->M + cpb - 1) / cpb);
            const size_t smem =
                resident_smem(c->d_pad, threads, lpc, resident_smax(c->d, G), c->cfg.dtilde_K, kind);
            if (smem > 200 * 1024) continue;
            CK(ensure_dyn_smem(fn, smem));
            int bps = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem));
            if ((long long)bps * nsm < G) continue;
            // fewest blocks (one barrier arrival and one set of atomics per block),
            // then the smallest per-lane footprint
            const double score = (double)G * 100.0 + cpl;
            if (n_ok < (int)(sizeof(ok) / sizeof(ok[0]))) ok[n_ok++] = {lpc, cpl, threads, G, smem, score};
        }
    }
    if (n_ok == 0)
        return fail(LAPS_ERR_UNSUPPORTED,
                    "no register-resident launch shape holds M=" + std::to_string(c->M) +
                        " chains of d=" + std::to_string(c->d) + " co-resident on this GPU");
    Cand best = ok[0];
    for (int k = 1; k < n_ok; ++k)
        if (ok[k].score < best.score) best = ok[k];
    c->lpc = best.lpc;
    c->cpl = best.cpl;
    c->threads = best.threads;
    c->G = best.G;
    c->smem = best.smem;
    c->qpp = resident_qpp(c->d_pad, best.threads);
    c->smax = resident_smax(c->d, best.G);
    c->fn = resident_fn(kind, best.lpc, best.cpl, c->cfg.dtilde_K > 0);
    return LAPS_OK;
}

// ------------------------------------------------------------------ launch
void fill_params(const laps_ctx* c, int mode, const float* x0, float x0_scale, KParams& P) {
    std::memset(&P, 0, sizeof(P));
    P.M = (int)c->M;
    P.d = c->d;
    P.d_pad = c->d_pad;
    P.nblk = c->d_pad / 4;
    P.kind = c->tg->kind;
    P.inv_s2 = (float)(1.0 / (c->tg->desc.banana_sb * c->tg->desc.banana_sb));
    P.inv_sv2 = (float)(1.0 / (c->tg->desc.funnel_sv * c->tg->desc.funnel_sv));
    P.prec = c->tg->kind == TGT_GAUSS_DENSE ? c->tg->prec_dense : c->tg->prec_pad;
    P.y = c->y;
    P.u = c->u;
    P.g = c->g;
    P.logp_ff = c->logp_ff;
    P.sigma = c->sigma;
    P.x0 = x0;
    P.x0_scale = x0_scale;
    P.part = c->part;
    P.cstat = c->cstat;
    P.ctot = c->ctot;
    P.ring = c->ring;
    P.win_sums = c->win_sums;
    P.Ex2 = c->have_truth ? c->Ex2 : nullptr;
    P.inv_varx2 = c->inv_varx2;
    P.hyper = c->hyper;
    P.trace = c->trace;
    P.trace_cap = c->trace_cap;
    P.bar_count = c->bar;
    P.status = c->status;
    const laps_config& g = c->cfg;
    P.C = (float)g.C;
    P.alpha = (float)g.alpha;
    P.switch_tol = (float)g.switch_tol;
    P.acc_tol = (float)g.acc_tol;
    P.adj_L_factor = (float)g.adj_L_factor;
    P.eps0 = (float)(g.eps0_coef * std::sqrt((double)c->d));
    P.a_target_mn2 = (float)g.a_target_mn2;
    P.a_target_mn4 = (float)g.a_target_mn4;
    P.stop_b2 = (float)g.stop_b2;
    P.fixed_eps = (float)g.fixed_eps;
    P.stop_b2_max = g.stop_b2_max;
    P.T = c->T;
    P.n_total = g.n_total_steps;
    P.N = g.steps_per_proposal;
    P.mn4_min_dim = g.mn4_min_dim;
    P.eevpd_centered = g.eevpd_centered;
    P.adjusted = g.adjusted;
    P.force_switch_at = g.force_switch_at;
    P.timeout_ns = g.barrier_timeout_ns;
    P.seed_lo = (uint32_t)c->seed;
    P.seed_hi = (uint32_t)(c->seed >> 32);
    P.pid = 0;
    P.mode = mode;
    P.n_iters = 1;
    P.G = c->G;
    P.qpp = c->qpp;
    P.smax = c->smax;
    P.bar_extra = g.barrier_extra_arrivals;
    P.dfull_K = g.dtilde_K;
    P.m0 = (int)c->m0;
    P.Mn = c->sharded ? (int)c->M_total : 0;
    P.phase_ns = c->phase_ns;
    P.yw = c->yw;
    P.uw = c->uw;
    P.dlw = c->dlw;
    P.lpw = c->lpw;
    P.W = c->W;
    P.gpart = c->gpart;
    P.lpart = c->lpart;
    P.nsplit = c->nsplit;
    P.go = c->go;
    P.Wb = c->mixed ? c->Wb : nullptr;
}

laps_status launch_resident(laps_ctx* c, int mode, int n_iters, const float* x0, float x0_scale,
                            cudaStream_t st) {
    KParams P;
    fill_params(c, mode, x0, x0_scale, P);
    P.n_iters = n_iters;
    CK(cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), st));
    const Coefs* cf = c->coefs;
    void* args[] = {&P, &cf};
    CK(cudaLaunchCooperativeKernel(c->fn, dim3(c->G), dim3(c->threads), args, c->smem, st));
    c->last_stream = st;
    return LAPS_OK;
}

}  // namespace laps

using namespace laps;

// =================================================================== C ABI
extern "C" {

const char* laps_last_error(void) { return g_err.c_str(); }
const char* laps_version(void) { return "laps-gb300 0.1 (sm_103a)"; }

void laps_config_default(laps_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
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
    c->stop_b2 = 0.0;
    c->stop_b2_max = 0;
    c->precision = LAPS_FP32;
    c->barrier_timeout_ns = 2000000000LL;
    c->fixed_eps = 0.0;
    c->chains_per_block = 0;
    c->lanes_per_chain = 0;
    c->coords_per_lane = 0;
}

laps_status laps_target_create(const laps_target_desc* desc, laps_target** out) {
    if (!desc || !out) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    const int64_t d = desc->d;
    if (d < 2 || d > (1 << 24)) return fail(LAPS_ERR_INVALID_ARG, "d must be in [2, 2^24]");
    switch (desc->kind) {
    case LAPS_GAUSS_DIAG:
        if (!desc->prec || !aligned(desc->prec, 4))
            return fail(LAPS_ERR_INVALID_ARG, "GAUSS_DIAG needs a device prec[d]");
        break;
    case LAPS_BANANA:
        if (d % 2) return fail(LAPS_ERR_INVALID_ARG, "BANANA needs an even d");
        if (!(desc->banana_sb > 0)) return fail(LAPS_ERR_INVALID_ARG, "banana_sb must be > 0");
        break;
    case LAPS_FUNNEL:
        if (!(desc->funnel_sv > 0)) return fail(LAPS_ERR_INVALID_ARG, "funnel_sv must be > 0");
        break;
    case LAPS_LOGREG:
        if (!desc->X || !desc->y || !aligned(desc->X, 4) || !aligned(desc->y, 4))
            return fail(LAPS_ERR_INVALID_ARG, "LOGREG needs device X[n_data][d] and y[n_data]");
        if (desc->n_data < 1 || desc->n_data > (1LL << 30))
            return fail(LAPS_ERR_INVALID_ARG, "n_data must be in [1, 2^30]");
        if (!(desc->prior_var > 0)) return fail(LAPS_ERR_INVALID_ARG, "prior_var must be > 0");
        if ((d + 63) / 64 * 64 > kLogregMaxKp)
            return fail(LAPS_ERR_UNSUPPORTED, "LOGREG is built for d <= " + std::to_string(kLogregMaxKp));
        break;
    case LAPS_USER:
        if (!desc->user_fn) return fail(LAPS_ERR_INVALID_ARG, "USER needs user_fn");
        if (d > kDenseMaxDim)
            return fail(LAPS_ERR_UNSUPPORTED, "USER targets are built for d <= " + std::to_string(kDenseMaxDim));
        break;
    case LAPS_GAUSS_DENSE:
        if (!desc->prec || !aligned(desc->prec, 4))
            return fail(LAPS_ERR_INVALID_ARG, "GAUSS_DENSE needs a device prec[d][d]");
        if (d > kDenseMaxDim)
            return fail(LAPS_ERR_UNSUPPORTED, "GAUSS_DENSE is built for d <= " + std::to_string(kDenseMaxDim));
        break;
    default:
        return fail(LAPS_ERR_INVALID_ARG, "unknown target kind");
    }
    laps_target* t = new laps_target();
    t->desc = *desc;
    t->kind = (int)desc->kind;
    t->d = (int)d;
    t->d_pad = (int)((d + 3) / 4 * 4);
    if (desc->kind == LAPS_GAUSS_DIAG) {
        cudaError_t e = cudaMalloc(&t->prec_pad, t->d_pad * sizeof(float));
        if (e != cudaSuccess) { delete t; return cuda_fail(e, "cudaMalloc prec"); }
        cudaMemset(t->prec_pad, 0, t->d_pad * sizeof(float));
        e = cudaMemcpy(t->prec_pad, desc->prec, d * sizeof(float), cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) { cudaFree(t->prec_pad); delete t; return cuda_fail(e, "copy prec"); }
    }
    if (desc->kind == LAPS_GAUSS_DENSE) {
        // padded to whole 32-column tiles of the contraction; padding rows and columns are zero
        t->d_pad = (int)((d + 31) / 32 * 32);
        const size_t pb = (size_t)t->d_pad * t->d_pad * sizeof(float);
        cudaError_t e = cudaMalloc(&t->prec_dense, pb);
        if (e == cudaSuccess) e = cudaMemset(t->prec_dense, 0, pb);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(t->prec_dense, t->d_pad * sizeof(float), desc->prec, d * sizeof(float),
                             d * sizeof(float), d, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            laps_target_destroy(t);
            return cuda_fail(e, "GAUSS_DENSE precision copy");
        }
    }
    if (desc->kind == LAPS_LOGREG) {
        // padded row stride: a multiple of 64 features for the contraction kernels
        t->d_pad = (int)((d + 63) / 64 * 64);
        LogregData& L = t->lr;
        L.n = (int)desc->n_data;
        L.d = (int)d;
        L.kp = t->d_pad;
        L.inv_v = (float)(1.0 / desc->prior_var);
        const size_t xb = (size_t)L.n * L.kp * sizeof(float);
        cudaError_t e = cudaMalloc(&L.X, xb);
        if (e == cudaSuccess) e = cudaMalloc(&L.y, (size_t)L.n * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(L.X, 0, xb);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(L.X, L.kp * sizeof(float), desc->X, d * sizeof(float), d * sizeof(float),
                             L.n, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(L.y, desc->y, (size_t)L.n * sizeof(float), cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            laps_target_destroy(t);
            return cuda_fail(e, "LOGREG data copy");
        }
        // BF16 copies for the tensor-core gradient (mixed precision); a target
        // without them serves the FP32 form only
        if (logreg_mma_supported(L.kp) && logreg_mma_prepare(L) != cudaSuccess) {
            cudaGetLastError();
            if (L.Xb) cudaFree(L.Xb);
            if (L.Xtb) cudaFree(L.Xtb);
            L.Xb = L.Xtb = nullptr;
        }
        // the three-term split of X for the tensor-core form at FP32 accuracy
        if (logreg_x3_supported(L.kp) && logreg_x3_prepare(L) != cudaSuccess) {
            cudaGetLastError();
            if (L.X3b) cudaFree(L.X3b);
            L.X3b = nullptr;
        }
        if (cudaMalloc(&t->status, sizeof(int)) != cudaSuccess ||
            cudaMemset(t->status, 0, sizeof(int)) != cudaSuccess) {
            laps_target_destroy(t);
            return fail(LAPS_ERR_OOM, "LOGREG status word");
        }
    }
    *out = t;
    return LAPS_OK;
}

void laps_target_destroy(laps_target* t) {
    if (!t) return;
    if (t->prec_pad) cudaFree(t->prec_pad);
    if (t->prec_dense) cudaFree(t->prec_dense);
    if (t->lr.X) cudaFree(t->lr.X);
    if (t->lr.y) cudaFree(t->lr.y);
    if (t->lr.Xb) cudaFree(t->lr.Xb);
    if (t->lr.Xtb) cudaFree(t->lr.Xtb);
    if (t->lr.X3b) cudaFree(t->lr.X3b);
    if (t->status) cudaFree(t->status);
    delete t;
}

laps_status laps_create(const laps_target* tg, int64_t M, const laps_config* cfg, laps_ctx** out) {
    if (!tg || !cfg || !out) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (M < 2 || M > (1LL << 30)) return fail(LAPS_ERR_INVALID_ARG, "M must be in [2, 2^30]");
    if (cfg->n_total_steps < 1 || cfg->steps_per_proposal < 1 || !(cfg->window_frac > 0) ||
        !(cfg->alpha > 0) || !(cfg->C > 0) || cfg->barrier_timeout_ns <= 0 || cfg->dtilde_K < 0 ||
        cfg->dtilde_K > 1024)
        return fail(LAPS_ERR_INVALID_ARG, "invalid config value");
    // GAUSS_DENSE runs in the register-resident kernel while P fits its shared memory
    const bool streamed = streamed_kind(tg->kind) &&
                          !(tg->kind == TGT_GAUSS_DENSE && tg->d_pad <= kDenseResidentMax && !cfg->dense_streamed);
    if (cfg->dtilde_K > 0 && (streamed || tg->kind == TGT_GAUSS_DENSE))
        return fail(LAPS_ERR_UNSUPPORTED, "the full-rank bias proxy is built for the diagonal, banana and funnel targets");
    if ((int)cfg->precision < LAPS_FP32 || (int)cfg->precision > LAPS_MIXED_BF16X3)
        return fail(LAPS_ERR_INVALID_ARG, "unknown precision");
    if (cfg->precision != LAPS_FP32 && tg->kind != TGT_LOGREG)
        return fail(LAPS_ERR_UNSUPPORTED, "mixed precision applies to LOGREG targets only");
    laps_ctx* c = new laps_ctx();
    c->tg = tg;
    c->M = M;
    c->cfg = *cfg;
    c->d = tg->d;
    c->d_pad = tg->d_pad;
    c->T = std::max(2, (int)std::ceil(cfg->window_frac * (double)cfg->n_total_steps));
    c->trace_cap = cfg->n_total_steps + 2;
    laps_status st = streamed ? streamed_setup(c) : choose_shape(c);
    if (st != LAPS_OK) { delete c; return st; }
    const size_t Md = (size_t)M * c->d_pad;
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        c->allocs.push_back(*p);
        return true;
    };
    bool ok = alloc((void**)&c->y, Md * 4) && alloc((void**)&c->u, Md * 4) &&
              alloc((void**)&c->g, Md * 4) && alloc((void**)&c->logp_ff, M * 8) &&
              alloc((void**)&c->sigma, c->d_pad * 4) &&
              alloc((void**)&c->part, part_bytes(c->d_pad, c->G, cfg->dtilde_K)) &&
              alloc((void**)&c->cstat, (size_t)c->d_pad * NCO * 4) &&
              alloc((void**)&c->ctot, (size_t)NCS * 8) &&
              alloc((void**)&c->ring, (size_t)(c->T + 1) * c->d_pad * 8) &&
              alloc((void**)&c->win_sums, (size_t)c->d_pad * 16) &&
              alloc((void**)&c->Ex2, c->d_pad * 8) && alloc((void**)&c->inv_varx2, c->d_pad * 4) &&
              alloc((void**)&c->hyper, sizeof(Hyper)) &&
              alloc((void**)&c->trace, (size_t)c->trace_cap * sizeof(laps_trace_row)) &&
              alloc((void**)&c->bar, 4 * sizeof(unsigned)) && alloc((void**)&c->status, sizeof(int)) &&
              alloc((void**)&c->coefs, sizeof(Coefs));
    if (!ok) {
        laps_destroy(c);
        return fail(LAPS_ERR_OOM, "device allocation of the ensemble state failed");
    }
    if (c->streamed) {
        st = streamed_alloc(c);
        if (st != LAPS_OK) { laps_destroy(c); return st; }
    }
    Coefs cf;
    coefs_table(cf);
    cudaMemcpy(c->coefs, &cf, sizeof(cf), cudaMemcpyHostToDevice);
    cudaMemset(c->status, 0, sizeof(int));
    cudaMemset(c->y, 0, Md * 4);
    cudaMemset(c->u, 0, Md * 4);
    cudaMemset(c->g, 0, Md * 4);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { laps_destroy(c); return cuda_fail(e, "laps_create"); }
    *out = c;
    return LAPS_OK;
}

laps_status laps_create_sharded(const laps_target* tg, int64_t M_local, const laps_shard* sh,
                                const laps_config* cfg, laps_ctx** out) {
    if (!tg || !sh || !cfg || !out) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (sh->n_ranks < 1 || sh->rank < 0 || sh->rank >= sh->n_ranks || sh->m0 < 0 || M_local < 2 ||
        sh->m0 + M_local > sh->M_total || sh->M_total > (1LL << 30))
        return fail(LAPS_ERR_INVALID_ARG, "shard: need 0 <= rank < n_ranks and 0 <= m0, m0 + M_local <= M_total");
    if (sh->n_ranks > 1 && !sh->allgather)
        return fail(LAPS_ERR_INVALID_ARG, "shard: more than one rank needs an allgather callback");
    if (sh->n_ranks == 1 && (sh->m0 != 0 || M_local != sh->M_total))
        return fail(LAPS_ERR_INVALID_ARG, "shard: a single rank holds the whole ensemble (m0 = 0, M_local = M_total)");
    const bool streamed = streamed_kind(tg->kind) &&
                          !(tg->kind == TGT_GAUSS_DENSE && tg->d_pad <= kDenseResidentMax && !cfg->dense_streamed);
    if (!streamed)
        return fail(LAPS_ERR_UNSUPPORTED, "a chain-sharded ensemble runs on the streamed path (LOGREG, USER, "
                                          "GAUSS_DENSE beyond d = 128 or with dense_streamed)");
    laps_ctx* c = nullptr;
    laps_status st = laps_create(tg, M_local, cfg, &c);
    if (st != LAPS_OK) return st;
    c->sharded = true;
    c->M_total = sh->M_total;
    c->m0 = sh->m0;
    c->rank = sh->rank;
    c->n_ranks = sh->n_ranks;
    c->shard_fn = sh->allgather;
    c->shard_user = sh->user_data;
    const size_t rows = rows_fb(c->d_pad);
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        c->allocs.push_back(*p);
        return true;
    };
    if (!(alloc((void**)&c->shard_send, rows * sizeof(float2)) &&
          alloc((void**)&c->shard_recv, (size_t)c->n_ranks * rows * sizeof(float2)) &&
          alloc((void**)&c->shard_part, (size_t)c->n_ranks * rows * sizeof(float2)))) {
        laps_destroy(c);
        return fail(LAPS_ERR_OOM, "device allocation of the shard exchange buffers failed");
    }
    *out = c;
    return LAPS_OK;
}

void laps_destroy(laps_ctx* c) {
    if (!c) return;
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_hyper) cudaFreeHost(c->h_hyper);
    delete c;
}

laps_status laps_set_truth(laps_ctx* c, const double* Ex2, const double* Varx2) {
    if (!c || !Ex2 || !Varx2) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    std::vector<float2> a(c->d_pad, make_float2(0.0f, 0.0f));
    std::vector<float> b(c->d_pad, 0.0f);
    for (int i = 0; i < c->d; ++i) {
        if (!(Varx2[i] > 0)) return fail(LAPS_ERR_INVALID_ARG, "Varx2 must be > 0");
        const float hi = (float)Ex2[i];
        a[i] = make_float2(hi, (float)(Ex2[i] - (double)hi));  // float-float copy of E_p[x^2]
        b[i] = (float)(1.0 / Varx2[i]);
    }
    CK(cudaMemcpy(c->Ex2, a.data(), c->d_pad * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->inv_varx2, b.data(), c->d_pad * 4, cudaMemcpyHostToDevice));
    c->have_truth = true;
    return LAPS_OK;
}

}  // extern "C"

namespace laps {
// the phase machine before Alg. 1's first line
Hyper initial_hyper() {
    Hyper h;
    std::memset(&h, 0, sizeof(h));
    h.phase = 0;
    h.t = 0;
    h.t_switch = -1;
    h.integ = INTEG_LF;
    h.grads = 1;
    h.b2_first_t = -1;
    h.b2_first_grads = -1;
    h.b2_first_ns = NAN;
    h.eevpd = h.eevpd_wanted = h.dtilde = h.max_delta = h.acc = NAN;
    h.b2_max = h.b2_avg = NAN;
    return h;
}

// clears the run state (phase machine, status, window, preconditioner) and
// launches the initialisation; no allocation
laps_status start_run(laps_ctx* c, const float* x0, float x0_scale, cudaStream_t st) {
    CK(cudaMemsetAsync(c->ring, 0, (size_t)(c->T + 1) * c->d_pad * 8, st));
    CK(cudaMemsetAsync(c->win_sums, 0, (size_t)c->d_pad * 16, st));
    CK(cudaMemsetAsync(c->cstat, 0, (size_t)c->d_pad * NCO * 4, st));
    run_start_kernel<<<grid_for(c->d_pad), 256, 0, st>>>(c->hyper, initial_hyper(), c->status, c->sigma,
                                                         c->d_pad);
    CK(cudaGetLastError());
    c->initialized = true;
    if (c->streamed) return streamed_init(c, x0, x0_scale, st);
    return launch_resident(c, 0, 1, x0, x0_scale, st);
}

laps_status status_error(int s) {
    if (s == ST_OK) return LAPS_OK;
    if (s == ST_TIMEOUT) return fail(LAPS_ERR_TIMEOUT, "a grid barrier wait exceeded barrier_timeout_ns");
    if (s == ST_NONFINITE) return fail(LAPS_ERR_NONFINITE, "non-finite initial position, log p or gradient");
    return fail(LAPS_ERR_CUDA, "device status " + std::to_string(s));
}

void stats_from_hyper(const Hyper& h, laps_stats* o) {
    std::memset(o, 0, sizeof(*o));
    o->phase = h.phase;
    o->t = h.t;
    o->t_switch = h.t_switch;
    o->integrator = h.integ;
    o->adapting = h.adapting;
    o->done = h.done;
    o->iterations = h.iters;
    o->nonfinite_total = h.nonfinite_total;
    o->grads = h.grads;
    o->eps = h.eps;
    o->L = h.L;
    o->eevpd = h.eevpd;
    o->eevpd_wanted = h.eevpd_wanted;
    o->dtilde = h.dtilde;
    o->max_delta = h.max_delta;
    o->acc = h.acc;
    o->b2_max = h.b2_max;
    o->b2_avg = h.b2_avg;
    o->sum_var = h.sum_var;
    o->b2_first_t = h.b2_first_t;
    o->b2_first_grads = h.b2_first_grads;
    o->b2_first_ns = h.b2_first_ns;
}
}  // namespace laps

extern "C" {

laps_status laps_init(laps_ctx* c, const float* x0, double x0_scale, uint64_t seed, void* stream) {
    if (!c) return fail(LAPS_ERR_INVALID_ARG, "null ctx");
    if (x0 && !aligned(x0, 4)) return fail(LAPS_ERR_INVALID_ARG, "x0 must be 4-byte aligned");
    c->seed = seed;
    return start_run(c, x0, (float)x0_scale, (cudaStream_t)stream);
}

laps_status laps_step(laps_ctx* c, int n_iters, void* stream) {
    if (!c || n_iters < 0) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if (!c->initialized) return fail(LAPS_ERR_INVALID_ARG, "laps_init has not run");
    if (n_iters == 0) return LAPS_OK;
    if (c->streamed) return streamed_step(c, n_iters, (cudaStream_t)stream);
    return launch_resident(c, 1, n_iters, nullptr, 0.0f, (cudaStream_t)stream);
}

laps_status laps_run(laps_ctx* c, void* stream) {
    if (!c) return fail(LAPS_ERR_INVALID_ARG, "null ctx");
    return laps_step(c, c->cfg.n_total_steps + 1, stream);
}

laps_status laps_adapt_freeze(laps_ctx* c, int frozen) {
    if (!c) return fail(LAPS_ERR_INVALID_ARG, "null ctx");
    CK(cudaStreamSynchronize(c->last_stream));
    Hyper h;
    CK(cudaMemcpy(&h, c->hyper, sizeof(h), cudaMemcpyDeviceToHost));
    h.adapting = frozen ? 0 : 1;
    CK(cudaMemcpy(c->hyper, &h, sizeof(h), cudaMemcpyHostToDevice));
    return LAPS_OK;
}

laps_status laps_sample(const laps_ctx* c, float* x_out, void* stream) {
    if (!c || !x_out || !aligned(x_out, 4)) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    unpack_rows_kernel<<<grid_for(c->M * c->d), 256, 0, st>>>(c->y, c->sigma, x_out, c->M, c->d,
                                                             c->d_pad);
    CK(cudaGetLastError());
    return LAPS_OK;
}

laps_status laps_get_state(const laps_ctx* c, float* y, float* u, float* g, double* logp,
                           float* sigma, void* stream) {
    if (!c) return fail(LAPS_ERR_INVALID_ARG, "null ctx");
    cudaStream_t st = (cudaStream_t)stream;
    const float* src[3] = {c->y, c->u, c->g};
    float* dst[3] = {y, u, g};
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        if (!aligned(dst[k], 4)) return fail(LAPS_ERR_INVALID_ARG, "misaligned output");
        unpack_rows_kernel<<<grid_for(c->M * c->d), 256, 0, st>>>(src[k], nullptr, dst[k], c->M,
                                                                 c->d, c->d_pad);
        CK(cudaGetLastError());
    }
    if (logp) {
        if (!aligned(logp, 8)) return fail(LAPS_ERR_INVALID_ARG, "misaligned logp");
        ff_to_double_kernel<<<grid_for(c->M), 256, 0, st>>>(c->logp_ff, logp, c->M);
        CK(cudaGetLastError());
    }
    if (sigma) CK(cudaMemcpyAsync(sigma, c->sigma, c->d * 4, cudaMemcpyDeviceToDevice, st));
    return LAPS_OK;
}

static laps_status read_status(laps_ctx* c) {
    CK(cudaStreamSynchronize(c->last_stream));
    int s = 0;
    CK(cudaMemcpy(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    return status_error(s);
}

laps_status laps_get_stats(laps_ctx* c, laps_stats* o) {
    if (!c || !o) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    laps_status st = read_status(c);
    Hyper h;
    CK(cudaMemcpy(&h, c->hyper, sizeof(h), cudaMemcpyDeviceToHost));
    stats_from_hyper(h, o);
    return st;
}

laps_status laps_get_trace(laps_ctx* c, laps_trace_row* rows, int cap, int* n) {
    if (!c || !n) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    CK(cudaStreamSynchronize(c->last_stream));
    Hyper h;
    CK(cudaMemcpy(&h, c->hyper, sizeof(h), cudaMemcpyDeviceToHost));
    const int avail = std::min(h.iters + 1, c->trace_cap);
    *n = avail;
    if (rows && cap > 0)
        CK(cudaMemcpy(rows, c->trace, (size_t)std::min(cap, avail) * sizeof(laps_trace_row),
                      cudaMemcpyDeviceToHost));
    return LAPS_OK;
}

// checkpoint layout: header, then every device buffer the run depends on
struct CkptHeader {
    char magic[8];
    int64_t M;
    int d, d_pad, T, trace_cap;
    uint64_t seed;
    int have_truth, pad_;
};

static std::vector<std::pair<void*, size_t>> ckpt_buffers(laps_ctx* c) {
    const size_t Md = (size_t)c->M * c->d_pad;
    return {{c->y, Md * 4},           {c->u, Md * 4},          {c->g, Md * 4},
            {c->logp_ff, (size_t)c->M * 8}, {c->sigma, (size_t)c->d_pad * 4},
            {c->cstat, (size_t)c->d_pad * NCO * 4},
            {c->ring, (size_t)(c->T + 1) * c->d_pad * 8}, {c->win_sums, (size_t)c->d_pad * 16},
            {c->Ex2, (size_t)c->d_pad * 8},    {c->inv_varx2, (size_t)c->d_pad * 4},
            {c->hyper, sizeof(Hyper)},
            {c->trace, (size_t)c->trace_cap * sizeof(laps_trace_row)}};
}

laps_status laps_checkpoint(laps_ctx* c, void* blob, size_t* size) {
    if (!c || !size) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    auto bufs = ckpt_buffers(c);
    size_t need = sizeof(CkptHeader);
    for (auto& b : bufs) need += b.second;
    if (!blob) { *size = need; return LAPS_OK; }
    if (*size < need) return fail(LAPS_ERR_INVALID_ARG, "checkpoint buffer too small");
    CK(cudaStreamSynchronize(c->last_stream));
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "LAPSCK1", 8);
    h.M = c->M; h.d = c->d; h.d_pad = c->d_pad; h.T = c->T; h.trace_cap = c->trace_cap;
    h.seed = c->seed; h.have_truth = c->have_truth;
    char* p = static_cast<char*>(blob);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    for (auto& b : bufs) {
        CK(cudaMemcpy(p, b.first, b.second, cudaMemcpyDeviceToHost));
        p += b.second;
    }
    *size = need;
    return LAPS_OK;
}

laps_status laps_restore(laps_ctx* c, const void* blob, size_t size) {
    if (!c || !blob) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    CkptHeader h;
    if (size < sizeof(h)) return fail(LAPS_ERR_INVALID_ARG, "checkpoint too small");
    std::memcpy(&h, blob, sizeof(h));
    if (std::memcmp(h.magic, "LAPSCK1", 8) != 0 || h.M != c->M || h.d != c->d ||
        h.d_pad != c->d_pad || h.T != c->T || h.trace_cap != c->trace_cap)
        return fail(LAPS_ERR_INVALID_ARG, "checkpoint does not match this context");
    auto bufs = ckpt_buffers(c);
    size_t need = sizeof(h);
    for (auto& b : bufs) need += b.second;
    if (size < need) return fail(LAPS_ERR_INVALID_ARG, "checkpoint truncated");
    CK(cudaStreamSynchronize(c->last_stream));
    const char* p = static_cast<const char*>(blob) + sizeof(h);
    for (auto& b : bufs) {
        CK(cudaMemcpy(b.first, p, b.second, cudaMemcpyHostToDevice));
        p += b.second;
    }
    c->seed = h.seed;
    c->have_truth = h.have_truth != 0;
    c->initialized = true;
    // a checkpoint is taken between laps_step calls, after the switch's one-time work
    Hyper hh;
    CK(cudaMemcpy(&hh, c->hyper, sizeof(hh), cudaMemcpyDeviceToHost));
    c->refreshed = hh.phase == 1;
    CK(cudaMemset(c->status, 0, sizeof(int)));
    return LAPS_OK;
}

#ifdef LAPS_PHASE_TIMING
// diagnostic build only (not part of the ABI): per-phase device time of block 0
laps_status laps_debug_phase_ns(laps_ctx* c, unsigned long long* out) {
    if (!c->phase_ns) {
        CK(cudaMalloc(&c->phase_ns, 16 * sizeof(unsigned long long)));
        c->allocs.push_back(c->phase_ns);
        CK(cudaMemset(c->phase_ns, 0, 16 * sizeof(unsigned long long)));
    }
    if (out) {  // [16]: the iteration's phases (0-6), the full-rank sub-steps (8-11)
        CK(cudaStreamSynchronize(c->last_stream));
        CK(cudaMemcpy(out, c->phase_ns, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        CK(cudaMemset(c->phase_ns, 0, 16 * sizeof(unsigned long long)));
    }
    return LAPS_OK;
}
#endif

laps_status laps_get_launch_info(const laps_ctx* c, laps_launch_info* o) {
    if (!c || !o) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    if (c->streamed) {
        o->chains_per_block = (int)((c->M + c->seg_G - 1) / c->seg_G);
        o->lanes_per_chain = 32;
        o->coords_per_lane = c->seg_cpl;
        o->threads = 256;
        o->blocks = c->seg_G;
        o->resident = 0;
        return LAPS_OK;
    }
    o->chains_per_block = c->threads / c->lpc;
    o->lanes_per_chain = c->lpc;
    o->coords_per_lane = c->cpl;
    o->threads = c->threads;
    o->blocks = c->G;
    o->resident = 1;
    return LAPS_OK;
}

}  // extern "C"
