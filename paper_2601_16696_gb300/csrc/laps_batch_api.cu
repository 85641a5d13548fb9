// laps_batch_api.cu -- host side of the batch entry points (include/laps.h):
// allocation of every problem's state, the per-problem parameter blocks the
// persistent kernel reads, CUDA-graph replay, and the autotuner that picks the
// launch shape by timing it on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "laps_internal.h"

using namespace laps;

namespace {

constexpr int kCpl[] = {8, 12, 16, 20};
constexpr int kMaxD = 10240;

struct BProb {
    int64_t d = 0, M = 0;
    int d_pad = 0, T = 0, trace_cap = 0;
    float *prec = nullptr, *y = nullptr, *u = nullptr, *sigma = nullptr, *cstat = nullptr;
    float* inv_varx2 = nullptr;
    float2 *part = nullptr, *ctot = nullptr, *ring = nullptr, *Ex2 = nullptr;
    float4* win_sums = nullptr;
    laps_trace_row* trace = nullptr;
    const float* x0 = nullptr;
    float x0_scale = 1.0f;
    bool have_truth = false;
};

#define BCK(call)                                               \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

}  // namespace

struct laps_batch {
    int n = 0;
    laps_config cfg{};
    std::vector<BProb> P;
    std::vector<uint32_t> ids;   // Philox problem id of each problem (default: its index)
    std::vector<void*> allocs;
    Hyper* hyper = nullptr;      // [n] device, one block of phase machines
    Hyper* h_hyper = nullptr;    // [n] pinned host copy
    KParams* d_probs = nullptr;  // [n] parameter blocks the kernel reads
    int* d_gw = nullptr;         // [n] lanes per chain (4 .. 512)
    int2* d_sched = nullptr;     // [n] blocks that hold each problem's chains
    std::vector<int2> sched;     // host copy
    Coefs* d_coefs = nullptr;
    unsigned* bar = nullptr;
    int* status = nullptr;
    int nsm = 0, G = 0, G_max = 0;
    int cpl = 0, widen = 0, SL = 64, cap_pad = 0;
    bool tuned = false, initialized = false;
    uint64_t seed = 0;
    cudaStream_t last_stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream for graph capture
    cudaGraphExec_t gexec = nullptr;
    int g_iters = 0;
    uint64_t g_seed = 0;
};

namespace {

bool shape_fits(const laps_batch* b, int cpl, int widen, int SL) {
    for (const BProb& p : b->P)
        if (batch_gw(p.d, cpl, widen) == 0) return false;
    return batch_blocks_per_sm(cpl, b->cap_pad, SL) >= 1;
}

KParams make_params(const laps_batch* b, int k) {
    const BProb& p = b->P[k];
    const laps_config& g = b->cfg;
    KParams P;
    std::memset(&P, 0, sizeof(P));
    P.M = (int)p.M;
    P.d = (int)p.d;
    P.d_pad = p.d_pad;
    P.nblk = p.d_pad / 4;
    P.kind = TGT_GAUSS;
    P.prec = p.prec;
    P.y = p.y;
    P.u = p.u;
    P.sigma = p.sigma;
    P.x0 = p.x0;
    P.x0_scale = p.x0_scale;
    P.part = p.part;
    P.cstat = p.cstat;
    P.ctot = p.ctot;
    P.ring = p.ring;
    P.win_sums = p.win_sums;
    P.Ex2 = p.have_truth ? p.Ex2 : nullptr;
    P.inv_varx2 = p.inv_varx2;
    P.hyper = b->hyper + k;
    P.trace = p.trace;
    P.trace_cap = p.trace_cap;
    P.bar_count = b->bar;
    P.status = b->status;
    P.C = (float)g.C;
    P.alpha = (float)g.alpha;
    P.switch_tol = (float)g.switch_tol;
    P.acc_tol = (float)g.acc_tol;
    P.adj_L_factor = (float)g.adj_L_factor;
    P.eps0 = (float)(g.eps0_coef * std::sqrt((double)p.d));
    P.a_target_mn2 = (float)g.a_target_mn2;
    P.a_target_mn4 = (float)g.a_target_mn4;
    P.stop_b2 = (float)g.stop_b2;
    P.fixed_eps = (float)g.fixed_eps;
    P.stop_b2_max = g.stop_b2_max;
    P.T = p.T;
    P.n_total = g.n_total_steps;
    P.N = g.steps_per_proposal;
    P.mn4_min_dim = g.mn4_min_dim;
    P.eevpd_centered = g.eevpd_centered;
    P.adjusted = g.adjusted;
    P.force_switch_at = g.force_switch_at;
    P.timeout_ns = g.barrier_timeout_ns;
    P.seed_lo = (uint32_t)b->seed;
    P.seed_hi = (uint32_t)(b->seed >> 32);
    P.pid = b->ids[k];
    P.G = b->sched.empty() ? b->G : b->sched[k].y;  // columns the slice owners add
    P.qpp = 1;
    P.smax = b->SL;
    P.bar_extra = g.barrier_extra_arrivals;
    P.gauss_derived = 1;
    return P;
}

laps_status upload(laps_batch* b) {
    std::vector<int64_t> dd(b->n), mm(b->n);
    for (int k = 0; k < b->n; ++k) {
        dd[k] = b->P[k].d;
        mm[k] = b->P[k].M;
    }
    b->sched.assign(b->n, make_int2(0, 0));
    batch_schedule(dd.data(), mm.data(), b->n, b->cpl, b->widen, b->G, b->sched.data());
    std::vector<KParams> h(b->n);
    std::vector<int> gw(b->n);
    for (int k = 0; k < b->n; ++k) {
        h[k] = make_params(b, k);
        gw[k] = batch_gw(b->P[k].d, b->cpl, b->widen);
        if (gw[k] == 0) return fail(LAPS_ERR_UNSUPPORTED, "batch shape does not hold problem " + std::to_string(k));
    }
    BCK(cudaMemcpy(b->d_probs, h.data(), sizeof(KParams) * b->n, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_gw, gw.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_sched, b->sched.data(), sizeof(int2) * b->n, cudaMemcpyHostToDevice));
    return LAPS_OK;
}

laps_status set_shape(laps_batch* b, int cpl, int widen, int SL) {
    if (!shape_fits(b, cpl, widen, SL)) return fail(LAPS_ERR_UNSUPPORTED, "batch shape does not fit");
    b->cpl = cpl;
    b->widen = widen;
    b->SL = SL;
    b->G = b->nsm * batch_blocks_per_sm(cpl, b->cap_pad, SL);
    if (b->G > b->G_max) b->G = b->G_max;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return upload(b);
}

laps_status launch(laps_batch* b, int mode, int n_iters, cudaStream_t st) {
    cudaError_t e = batch_launch(b->cpl, b->G, b->d_probs, b->d_gw, b->d_sched, b->d_coefs, b->n, mode, n_iters,
                                 b->SL, b->cap_pad, b->bar, b->status, b->cfg.barrier_timeout_ns,
                                 b->cfg.barrier_extra_arrivals, b->seed, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch_kernel launch");
    b->last_stream = st;
    return LAPS_OK;
}

// the start of a run of every problem: its seed in the parameter block, its
// phase machine (h0, by value), a cleared window, column results and status,
// sigma = 1; block k takes problems k, k + gridDim.x, ...
__global__ void batch_start_kernel(KParams* probs, Hyper* hyper, int n, uint32_t seed_lo, uint32_t seed_hi,
                                   const Hyper h0, int* status) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        KParams& P = probs[k];
        if (threadIdx.x == 0) {
            P.seed_lo = seed_lo;
            P.seed_hi = seed_hi;
            hyper[k] = h0;
        }
        const int dp = P.d_pad;
        const size_t nring = (size_t)(P.T + 1) * dp;
        for (size_t i = threadIdx.x; i < nring; i += blockDim.x) P.ring[i] = make_float2(0.0f, 0.0f);
        for (int i = threadIdx.x; i < dp; i += blockDim.x) {
            P.win_sums[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            P.sigma[i] = 1.0f;
        }
        for (int i = threadIdx.x; i < dp * NCO; i += blockDim.x) P.cstat[i] = 0.0f;
    }
}

// problem k's positions x = sigma o y, except after a switch that no proposal
// followed (y is still in x then); the phase machine is read on the device
__global__ void batch_unpack_kernel(const float* __restrict__ y, const float* __restrict__ sigma,
                                    const Hyper* __restrict__ h, float* __restrict__ x, int64_t M, int d,
                                    int d_pad) {
    const bool pend = h->phase == 1 && h->p == 0;
    const int64_t n = M * (int64_t)d;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k / d;
        const int i = (int)(k - m * d);
        x[k] = (pend ? 1.0f : sigma[i]) * y[m * d_pad + i];
    }
}

laps_status read_hypers(laps_batch* b) {
    BCK(cudaStreamSynchronize(b->last_stream));
    BCK(cudaMemcpy(b->h_hyper, b->hyper, sizeof(Hyper) * b->n, cudaMemcpyDeviceToHost));
    int s = 0;
    BCK(cudaMemcpy(&s, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    return status_error(s);
}

// device copies of everything an iteration changes, for the autotuner
struct Snapshot {
    std::vector<std::pair<void*, size_t>> bufs;
    std::vector<void*> copies;
    ~Snapshot() {
        for (void* p : copies) cudaFree(p);
    }
};

laps_status snapshot(laps_batch* b, Snapshot& s) {
    for (BProb& p : b->P) {
        const size_t Md = (size_t)p.M * p.d_pad * 4;
        s.bufs.push_back({p.y, Md});
        s.bufs.push_back({p.u, Md});
        s.bufs.push_back({p.sigma, (size_t)p.d_pad * 4});
        s.bufs.push_back({p.ring, (size_t)(p.T + 1) * p.d_pad * 8});
        s.bufs.push_back({p.win_sums, (size_t)p.d_pad * 16});
        s.bufs.push_back({p.cstat, (size_t)p.d_pad * NCO * 4});
    }
    s.bufs.push_back({b->hyper, sizeof(Hyper) * b->n});
    for (auto& q : s.bufs) {
        void* c = nullptr;
        if (cudaMalloc(&c, q.second) != cudaSuccess) return fail(LAPS_ERR_OOM, "autotuner snapshot");
        s.copies.push_back(c);
        BCK(cudaMemcpy(c, q.first, q.second, cudaMemcpyDeviceToDevice));
    }
    return LAPS_OK;
}

laps_status restore(Snapshot& s) {
    for (size_t k = 0; k < s.bufs.size(); ++k)
        BCK(cudaMemcpy(s.bufs[k].first, s.copies[k], s.bufs[k].second, cudaMemcpyDeviceToDevice));
    return LAPS_OK;
}

}  // namespace

extern "C" {

laps_status laps_batch_create(const laps_problem* probs, int n, const laps_config* cfg, laps_batch** out) {
    if (!probs || !cfg || !out || n < 1 || n > 4096) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    if (cfg->n_total_steps < 1 || cfg->steps_per_proposal < 1 || !(cfg->window_frac > 0) ||
        !(cfg->alpha > 0) || !(cfg->C > 0) || cfg->barrier_timeout_ns <= 0)
        return fail(LAPS_ERR_INVALID_ARG, "invalid config value");
    if (cfg->dtilde_K != 0) return fail(LAPS_ERR_UNSUPPORTED, "the batch serves the diagonal bias proxy");
    for (int k = 0; k < n; ++k) {
        const laps_problem& q = probs[k];
        if (q.d < 2 || q.d > kMaxD) return fail(LAPS_ERR_INVALID_ARG, "problem d must be in [2, 10240]");
        if (q.M < 2 || q.M > (1LL << 30)) return fail(LAPS_ERR_INVALID_ARG, "problem M must be in [2, 2^30]");
        if (!q.prec || reinterpret_cast<uintptr_t>(q.prec) % 4 || reinterpret_cast<uintptr_t>(q.x0) % 4)
            return fail(LAPS_ERR_INVALID_ARG, "problem prec (and x0) must be 4-byte aligned device arrays");
    }
    laps_batch* b = new laps_batch();
    b->n = n;
    b->cfg = *cfg;
    b->P.resize(n);
    b->ids.resize(n);
    for (int k = 0; k < n; ++k) b->ids[k] = (uint32_t)k;
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        b->allocs.push_back(*p);
        return true;
    };
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < n; ++k) b->cap_pad = std::max(b->cap_pad, (int)((probs[k].d + 3) / 4 * 4));
    for (int k = 0; k < n; ++k) {
        BProb& p = b->P[k];
        p.d = probs[k].d;
        p.M = probs[k].M;
        p.d_pad = (int)((p.d + 3) / 4 * 4);
        p.T = std::max(2, (int)std::ceil(cfg->window_frac * (double)cfg->n_total_steps));
        p.trace_cap = cfg->n_total_steps + 2;
        p.x0 = probs[k].x0;
        p.x0_scale = (float)probs[k].x0_scale;
    }
    // blocks of the widest feasible shape bound the per-block column buffers
    for (int cpl : kCpl)
        if (shape_fits(b, cpl, 0, b->SL)) b->G_max = std::max(b->G_max, b->nsm * batch_blocks_per_sm(cpl, b->cap_pad, b->SL));
    if (b->G_max == 0) {
        delete b;
        return fail(LAPS_ERR_UNSUPPORTED, "no batch shape holds these problems");
    }
    bool ok = alloc((void**)&b->hyper, sizeof(Hyper) * n) && alloc((void**)&b->d_probs, sizeof(KParams) * n) &&
              alloc((void**)&b->d_gw, sizeof(int) * n) && alloc((void**)&b->d_sched, sizeof(int2) * n) &&
              alloc((void**)&b->d_coefs, sizeof(Coefs)) &&
              alloc((void**)&b->bar, 4 * sizeof(unsigned)) && alloc((void**)&b->status, sizeof(int));
    for (int k = 0; k < n && ok; ++k) {
        BProb& p = b->P[k];
        const size_t Md = (size_t)p.M * p.d_pad;
        ok = alloc((void**)&p.prec, p.d_pad * 4) && alloc((void**)&p.y, Md * 4) && alloc((void**)&p.u, Md * 4) &&
             alloc((void**)&p.sigma, p.d_pad * 4) &&
             alloc((void**)&p.part, ((size_t)NQ * p.d_pad + NCS) * b->G_max * 8) &&
             alloc((void**)&p.cstat, (size_t)p.d_pad * NCO * 4) && alloc((void**)&p.ctot, NCS * 8) &&
             alloc((void**)&p.ring, (size_t)(p.T + 1) * p.d_pad * 8) && alloc((void**)&p.win_sums, (size_t)p.d_pad * 16) &&
             alloc((void**)&p.Ex2, p.d_pad * 8) && alloc((void**)&p.inv_varx2, p.d_pad * 4) &&
             alloc((void**)&p.trace, (size_t)p.trace_cap * sizeof(laps_trace_row));
        if (ok) {
            cudaMemset(p.prec, 0, p.d_pad * 4);
            cudaMemcpy(p.prec, probs[k].prec, p.d * 4, cudaMemcpyDeviceToDevice);
            cudaMemset(p.y, 0, Md * 4);
            cudaMemset(p.u, 0, Md * 4);
        }
    }
    if (ok && cudaMallocHost((void**)&b->h_hyper, sizeof(Hyper) * n) != cudaSuccess) ok = false;
    if (ok && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) ok = false;
    if (!ok) {
        laps_batch_destroy(b);
        return fail(LAPS_ERR_OOM, "device allocation of the batch failed");
    }
    Coefs cf;
    coefs_table(cf);
    cudaMemcpy(b->d_coefs, &cf, sizeof(cf), cudaMemcpyHostToDevice);
    cudaMemset(b->status, 0, sizeof(int));
    // default shape: the fewest coordinates per lane that hold every problem
    laps_status st = LAPS_ERR_UNSUPPORTED;
    for (int cpl : kCpl)
        if (shape_fits(b, cpl, 0, b->SL)) {
            st = set_shape(b, cpl, 0, b->SL);
            break;
        }
    cudaError_t e = cudaDeviceSynchronize();
    if (st == LAPS_OK && e != cudaSuccess) st = cuda_fail(e, "laps_batch_create");
    if (st != LAPS_OK) {
        laps_batch_destroy(b);
        return st;
    }
    *out = b;
    return LAPS_OK;
}

void laps_batch_destroy(laps_batch* b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_hyper) cudaFreeHost(b->h_hyper);
    delete b;
}

laps_status laps_batch_set_truth(laps_batch* b, int k, const double* Ex2, const double* Varx2) {
    if (!b || k < 0 || k >= b->n || !Ex2 || !Varx2) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    BProb& p = b->P[k];
    std::vector<float2> a(p.d_pad, make_float2(0.0f, 0.0f));
    std::vector<float> v(p.d_pad, 0.0f);
    for (int64_t i = 0; i < p.d; ++i) {
        if (!(Varx2[i] > 0)) return fail(LAPS_ERR_INVALID_ARG, "Varx2 must be > 0");
        const float hi = (float)Ex2[i];
        a[i] = make_float2(hi, (float)(Ex2[i] - (double)hi));
        v[i] = (float)(1.0 / Varx2[i]);
    }
    BCK(cudaMemcpy(p.Ex2, a.data(), p.d_pad * 8, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(p.inv_varx2, v.data(), p.d_pad * 4, cudaMemcpyHostToDevice));
    p.have_truth = true;
    return upload(b);
}

laps_status laps_batch_init(laps_batch* b, uint64_t seed, void* stream) {
    if (!b) return fail(LAPS_ERR_INVALID_ARG, "null batch");
    cudaStream_t st = (cudaStream_t)stream;
    b->seed = seed;  // later uploads of the parameter blocks carry it
    const int blocks = std::min(b->n, 1024);
    batch_start_kernel<<<blocks, 256, 0, st>>>(b->d_probs, b->hyper, b->n, (uint32_t)seed,
                                               (uint32_t)(seed >> 32), initial_hyper(), b->status);
    BCK(cudaGetLastError());
    b->initialized = true;
    return launch(b, 0, 1, st);
}

laps_status laps_batch_step(laps_batch* b, int n_iters, void* stream) {
    if (!b || n_iters < 0) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if (!b->initialized) return fail(LAPS_ERR_INVALID_ARG, "laps_batch_init has not run");
    if (n_iters == 0) return LAPS_OK;
    return launch(b, 1, n_iters, (cudaStream_t)stream);
}

laps_status laps_batch_run(laps_batch* b, int iters_per_launch, void* stream) {
    if (!b || iters_per_launch < 1) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if (!b->initialized) return fail(LAPS_ERR_INVALID_ARG, "laps_batch_init has not run");
    cudaStream_t st = (cudaStream_t)stream;
    // the launch carries the seed's Philox round keys: a new seed needs a new graph
    if (!b->gexec || b->g_iters != iters_per_launch || b->g_seed != b->seed) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        laps_status s = launch(b, 1, iters_per_launch, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (s != LAPS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "capturing the batch launch");
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "instantiating the batch graph");
        b->g_iters = iters_per_launch;
        b->g_seed = b->seed;
    }
    b->last_stream = st;
    // enough launches for a run that never switches (one step per iteration); a
    // launch that finds every problem done (or a latched error) returns at once
    const long long max_launches = (long long)b->cfg.n_total_steps / iters_per_launch + 2;
    for (long long r = 0; r < max_launches; ++r) BCK(cudaGraphLaunch(b->gexec, st));
    return LAPS_OK;
}

laps_status laps_batch_tune(laps_batch* b, void* stream) {
    if (!b) return fail(LAPS_ERR_INVALID_ARG, "null batch");
    if (!b->initialized) return fail(LAPS_ERR_INVALID_ARG, "laps_batch_init has not run");
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaStreamSynchronize(st));
    Snapshot snap;
    laps_status s = snapshot(b, snap);
    if (s != LAPS_OK) return s;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bc = b->cpl, bw = b->widen, bs = b->SL;
    for (int cpl : kCpl)
        for (int widen = 0; widen < 2; ++widen)
            for (int SL : {32, 128}) {
                if (!shape_fits(b, cpl, widen, SL)) continue;
                if (set_shape(b, cpl, widen, SL) != LAPS_OK) continue;
                if (restore(snap) != LAPS_OK || launch(b, 1, 1, st) != LAPS_OK) break;  // warm-up
                if (restore(snap) != LAPS_OK) break;
                cudaEventRecord(e0, st);
                if (launch(b, 1, 2, st) != LAPS_OK) break;
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    bc = cpl;
                    bw = widen;
                    bs = SL;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s = set_shape(b, bc, bw, bs);
    if (s != LAPS_OK) return s;
    s = restore(snap);
    if (s != LAPS_OK) return s;
    BCK(cudaDeviceSynchronize());
    b->tuned = true;
    return LAPS_OK;
}

laps_status laps_batch_get_shape(const laps_batch* b, laps_batch_shape* o) {
    if (!b || !o) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    o->coords_per_lane = b->cpl;
    o->widen = b->widen;
    o->slice = b->SL;
    o->threads = batch_threads();
    o->blocks = b->G;
    o->tuned = b->tuned ? 1 : 0;
    return LAPS_OK;
}

laps_status laps_batch_set_shape(laps_batch* b, const laps_batch_shape* s) {
    if (!b || !s || s->slice < 1 || s->slice > 4096 || s->widen < 0 || s->widen > 4)
        return fail(LAPS_ERR_INVALID_ARG, "bad shape");
    return set_shape(b, s->coords_per_lane, s->widen, s->slice);
}

laps_status laps_batch_set_ids(laps_batch* b, const int32_t* ids) {
    if (!b || !ids) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    std::vector<int32_t> seen(ids, ids + b->n);
    std::sort(seen.begin(), seen.end());
    for (int k = 0; k < b->n; ++k) {
        if (seen[k] < 0 || seen[k] >= (1 << 24)) return fail(LAPS_ERR_INVALID_ARG, "problem ids must be in [0, 2^24)");
        if (k > 0 && seen[k] == seen[k - 1]) return fail(LAPS_ERR_INVALID_ARG, "problem ids must be distinct");
    }
    for (int k = 0; k < b->n; ++k) b->ids[k] = (uint32_t)ids[k];
    return upload(b);
}

laps_status laps_batch_partition(const int64_t* d, const int64_t* M, int n, int n_ranks, int32_t* owner) {
    if (!d || !M || !owner || n < 1 || n_ranks < 1) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    std::vector<int64_t> cost(n);
    for (int k = 0; k < n; ++k) {
        if (d[k] < 1 || M[k] < 1) return fail(LAPS_ERR_INVALID_ARG, "problem d and M must be positive");
        cost[k] = (d[k] + 3) / 4 * 4 * M[k];
    }
    // longest processing time first: problems by falling cost (ties: lower
    // index first), each to the rank with the least load (ties: lower rank)
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<int64_t> load(n_ranks, 0);
    for (int k : order) {
        int r = 0;
        for (int q = 1; q < n_ranks; ++q)
            if (load[q] < load[r]) r = q;
        owner[k] = r;
        load[r] += cost[k];
    }
    return LAPS_OK;
}

laps_status laps_batch_get_stats(laps_batch* b, int k, laps_stats* o) {
    if (!b || !o || k < 0 || k >= b->n) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    laps_status s = read_hypers(b);
    stats_from_hyper(b->h_hyper[k], o);
    return s;
}

laps_status laps_batch_get_trace(laps_batch* b, int k, laps_trace_row* rows, int cap, int* n) {
    if (!b || !n || k < 0 || k >= b->n) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    read_hypers(b);
    const BProb& p = b->P[k];
    const int avail = std::min(b->h_hyper[k].iters + 1, p.trace_cap);
    *n = avail;
    if (rows && cap > 0)
        BCK(cudaMemcpy(rows, p.trace, (size_t)std::min(cap, avail) * sizeof(laps_trace_row),
                       cudaMemcpyDeviceToHost));
    return LAPS_OK;
}

laps_status laps_batch_sample(laps_batch* b, int k, float* x_out, void* stream) {
    if (!b || !x_out || k < 0 || k >= b->n || reinterpret_cast<uintptr_t>(x_out) % 4)
        return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    const BProb& p = b->P[k];
    const int64_t n = p.M * p.d;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
    batch_unpack_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(p.y, p.sigma, b->hyper + k, x_out, p.M,
                                                                  (int)p.d, p.d_pad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "laps_batch_sample");
}

}  // extern "C"
