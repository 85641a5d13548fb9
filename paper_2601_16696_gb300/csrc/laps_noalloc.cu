// laps_noalloc.cu -- a complete LAPS run that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned
// by a pool allocator that reserved the GPU at start-up (a cudaMalloc there
// fails or fragments the pool), code that must not add the device-wide
// synchronisation that cudaMalloc/cudaFree imply, or a plug-in that may not
// grow the process's device footprint after it is loaded.  laps_run_noalloc
// serves them: every buffer the run needs besides the caller's inputs and
// outputs lives in one file-scope __device__ array of fixed size,
// kNoAllocScratchBytes (16 MiB), which every GPU that loads the library holds
// until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "laps_internal.h"

namespace laps {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code `g_noalloc_scratch` names a host-side stand-in, not a device
// address; the device address is looked up once per device and cached.  The
// cache outlives a cudaDeviceReset, after which the address is stale: this
// entry point does not support a reset of a device it has run on.
constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

static laps_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(LAPS_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LAPS_OK;
}

// hands out 256-byte aligned pieces of the scratch array (a null base only counts)
struct Carver {
    char* base;
    size_t off;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

static void carve(laps_ctx& c, laps_target& t, Carver& cv) {
    const size_t Md = (size_t)c.M * c.d_pad;
    t.prec_pad = t.kind == TGT_GAUSS ? (float*)cv.take((size_t)c.d_pad * 4) : nullptr;
    c.y = (float*)cv.take(Md * 4);
    c.u = (float*)cv.take(Md * 4);
    c.g = (float*)cv.take(Md * 4);
    c.logp_ff = (float2*)cv.take((size_t)c.M * 8);
    c.sigma = (float*)cv.take((size_t)c.d_pad * 4);
    c.part = (float2*)cv.take(((size_t)NQ * c.d_pad + NCS) * c.G * 8);
    c.cstat = (float*)cv.take((size_t)c.d_pad * NCO * 4);
    c.ctot = (float2*)cv.take((size_t)NCS * 8);
    c.ring = (float2*)cv.take((size_t)(c.T + 1) * c.d_pad * 8);
    c.win_sums = (float4*)cv.take((size_t)c.d_pad * 16);
    c.hyper = (Hyper*)cv.take(sizeof(Hyper));
    c.bar = (unsigned*)cv.take(4 * sizeof(unsigned));
    c.status = (int*)cv.take(sizeof(int));
    c.coefs = (Coefs*)cv.take(sizeof(Coefs));
}

}  // namespace laps

using namespace laps;

extern "C" laps_status laps_run_noalloc(const laps_target_desc* desc, int64_t M,
                                        const laps_config* cfg, const float* x0, double x0_scale,
                                        uint64_t seed, float* x_out, laps_stats* stats_out,
                                        void* stream) {
    if (!desc && M == 0 && !cfg && !x_out) {
        // set-up only: loads the library's device code on the current device (which
        // reserves the scratch array there) and looks up the array's address
        void* base = nullptr;
        return scratch_address(&base);
    }
    if (!desc || !cfg || !x_out) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    const int64_t d = desc->d;
    if (d < 2 || d > (1 << 24)) return fail(LAPS_ERR_INVALID_ARG, "d must be in [2, 2^24]");
    if (M < 2 || M > (1LL << 30)) return fail(LAPS_ERR_INVALID_ARG, "M must be in [2, 2^30]");
    if (cfg->n_total_steps < 1 || cfg->steps_per_proposal < 1 || !(cfg->window_frac > 0) ||
        !(cfg->alpha > 0) || !(cfg->C > 0) || cfg->barrier_timeout_ns <= 0)
        return fail(LAPS_ERR_INVALID_ARG, "invalid config value");
    if (cfg->dtilde_K != 0) return fail(LAPS_ERR_UNSUPPORTED, "laps_run_noalloc serves the diagonal bias proxy");
    if (cfg->precision != LAPS_FP32)
        return fail(LAPS_ERR_UNSUPPORTED, "laps_run_noalloc computes in FP32 (precision = LAPS_FP32)");
    if (cfg->stop_b2 > 0)
        return fail(LAPS_ERR_UNSUPPORTED, "laps_run_noalloc keeps no truth for b^2, so stop_b2 must be 0");
    if ((x0 && reinterpret_cast<uintptr_t>(x0) % 4) || reinterpret_cast<uintptr_t>(x_out) % 4)
        return fail(LAPS_ERR_INVALID_ARG, "x0 and x_out must be 4-byte aligned");
    switch (desc->kind) {
    case LAPS_GAUSS_DIAG:
        if (!desc->prec) return fail(LAPS_ERR_INVALID_ARG, "GAUSS_DIAG needs a device prec[d]");
        break;
    case LAPS_BANANA:
        if (d % 2 || !(desc->banana_sb > 0))
            return fail(LAPS_ERR_INVALID_ARG, "BANANA needs an even d and banana_sb > 0");
        break;
    case LAPS_FUNNEL:
        if (!(desc->funnel_sv > 0)) return fail(LAPS_ERR_INVALID_ARG, "funnel_sv must be > 0");
        break;
    default:
        return fail(LAPS_ERR_UNSUPPORTED, "laps_run_noalloc serves GAUSS_DIAG, BANANA and FUNNEL");
    }
    // handles on the stack; nothing below allocates device memory
    laps_target t;
    t.desc = *desc;
    t.kind = (int)desc->kind;
    t.d = (int)d;
    t.d_pad = (int)((d + 3) / 4 * 4);
    laps_ctx c;
    c.tg = &t;
    c.M = M;
    c.cfg = *cfg;
    c.d = t.d;
    c.d_pad = t.d_pad;
    c.T = std::max(2, (int)std::ceil(cfg->window_frac * (double)cfg->n_total_steps));
    c.trace_cap = 0;  // no trace: laps_stats reports the outcome
    laps_status st = choose_shape(&c);
    if (st != LAPS_OK) return st;
    Carver count{nullptr, 0};
    carve(c, t, count);
    if (count.off > kNoAllocScratchBytes)
        return fail(LAPS_ERR_INVALID_ARG,
                    "laps_run_noalloc: this problem needs " + std::to_string(count.off) +
                        " bytes of scratch; the fixed array holds " +
                        std::to_string(kNoAllocScratchBytes) + " (use laps_create instead)");
    void* base = nullptr;
    st = scratch_address(&base);
    if (st != LAPS_OK) return st;
    Carver cv{static_cast<char*>(base), 0};
    carve(c, t, cv);

    cudaStream_t s = (cudaStream_t)stream;
    Coefs cf;
    coefs_table(cf);
    launch_set_coefs(c.coefs, cf, s);  // by value: nothing on this stack is read later
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "write integrator table");
    if (t.kind == TGT_GAUSS) {
        e = cudaMemsetAsync(t.prec_pad, 0, (size_t)t.d_pad * 4, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t.prec_pad, desc->prec, (size_t)d * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy prec");
    }
    c.seed = seed;
    st = start_run(&c, x0, (float)x0_scale, s);  // clears the shared state the run reads
    if (st != LAPS_OK) return st;
    st = launch_resident(&c, 1, cfg->n_total_steps + 1, nullptr, 0.0f, s);
    if (st != LAPS_OK) return st;
    launch_unpack(c.y, c.sigma, x_out, M, c.d, c.d_pad, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "unpack samples");
    if (!stats_out) return LAPS_OK;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "laps_run_noalloc");
    int dev_status = 0;
    Hyper h;
    e = cudaMemcpy(&dev_status, c.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h, c.hyper, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read run status");
    stats_from_hyper(h, stats_out);
    return status_error(dev_status);
}
