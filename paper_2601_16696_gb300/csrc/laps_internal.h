// laps_internal.h -- opaque handle layouts and host helpers of liblaps.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "laps_logreg.cuh"
#include "laps_params.h"
#include "laps_resident_kernel.cuh"

struct laps_target {
    laps_target_desc desc;
    int kind = 0, d = 0, d_pad = 0;
    float* prec_pad = nullptr;  // GAUSS_DIAG precisions, zero padded to d_pad (owned)
    laps::LogregData lr{};      // LOGREG: padded copies of X and y (owned)
    float* prec_dense = nullptr; // GAUSS_DENSE: P [d_pad][d_pad], zero padded, d_pad = 32 k (owned)
    int* status = nullptr;      // LOGREG: latched status of the tensor-core target call (owned)
};

struct laps_ctx {
    const laps_target* tg = nullptr;
    int64_t M = 0;
    laps_config cfg{};
    int d = 0, d_pad = 0, T = 0, trace_cap = 0;
    // ensemble state (sampler coordinates, [M][d_pad]) and phase machine
    float *y = nullptr, *u = nullptr, *g = nullptr, *sigma = nullptr;
    float2* logp_ff = nullptr;
    float2* part = nullptr;   // [NQ * d_pad + NCS][G] per-block sums
    float* cstat = nullptr;   // [d_pad][NCO] per-coordinate results
    float2* ctot = nullptr;   // [NCS] chain totals
    int smax = 1;             // largest coordinate slice of a block
    float2* ring = nullptr;
    float4* win_sums = nullptr;
    float2* Ex2 = nullptr;
    float* inv_varx2 = nullptr;
    int qpp = 1;
    unsigned long long* phase_ns = nullptr;  // diagnostic build: per-phase time (not owned)
    laps::Hyper* hyper = nullptr;
    laps_trace_row* trace = nullptr;
    unsigned* bar = nullptr;
    int* status = nullptr;
    laps::Coefs* coefs = nullptr;
    std::vector<void*> allocs;
    // launch shape
    int lpc = 0, cpl = 0, threads = 0, G = 0;
    size_t smem = 0;
    const void* fn = nullptr;
    cudaStream_t last_stream = nullptr;
    uint64_t seed = 0;
    bool initialized = false, have_truth = false;
    // streamed path (targets whose gradient is an ensemble contraction)
    bool streamed = false;
    float *yw = nullptr, *uw = nullptr, *W = nullptr, *gpart = nullptr;
    float* ulp = nullptr;            // USER targets: the callback's FP32 log p [M]
    float2 *dlw = nullptr, *lpw = nullptr, *lpart = nullptr;
    int* go = nullptr;
    int nsplit = 1, seg_cpl = 0, seg_G = 0, fin_G = 0, adj_integ = 0;
    size_t seg_smem = 0, fin_slice_smem = 0, fin_gather_smem = 0;
    laps::Hyper* h_hyper = nullptr;  // pinned host copy of the phase machine (owned)
    laps::Coefs cf{};                // integrator tables on the host
    // contraction form of each phase (GF_*); mixed: the unadjusted one is
    // the BF16 tensor-core form, which reads the hi | lo copy Wb
    int gf_unadj = 0, gf_adj = 0;
    bool mixed = false;
    bool refreshed = false;          // streamed: the switch's one-time work is done
    void* Wb = nullptr;              // [M_pad][2 d_pad] BF16 hi | lo copy of the points
    int64_t M_pad = 0;
    int nsplit_mma = 1, rps_mma = 64;
    int nsplit_x3 = 1, rps_x3 = 64;   // the three-term tensor-core form's data splits
    alignas(64) unsigned char tmW[128];  // CUtensorMap of Wb
    // chain-sharded ensemble (laps_create_sharded): chains m0 .. m0 + M - 1 of M_total
    bool sharded = false;
    int64_t M_total = 0, m0 = 0;
    int rank = 0, n_ranks = 1;
    laps_allgather_fn shard_fn = nullptr;
    void* shard_user = nullptr;
    float2* shard_send = nullptr;   // [rows] this rank's column totals
    float2* shard_recv = nullptr;   // [n_ranks][rows] every rank's, in rank order
    float2* shard_part = nullptr;   // [rows][n_ranks] the same, in the columns layout the finalise reads
};

namespace laps {
laps_status fail(laps_status st, const std::string& msg);
laps_status cuda_fail(cudaError_t e, const char* what);
// Let kernel fn use at least `bytes` of dynamic shared memory.  The limit is a
// process-wide attribute of the function, so it is only ever raised: a context
// that needs less must not lower it under another live context's launches.
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes);
// shared by the context API and the allocation-free entry point (laps_api.cu)
laps_status choose_shape(laps_ctx* c);
laps_status start_run(laps_ctx* c, const float* x0, float x0_scale, cudaStream_t st);
laps_status launch_resident(laps_ctx* c, int mode, int n_iters, const float* x0, float x0_scale,
                            cudaStream_t st);
void fill_params(const laps_ctx* c, int mode, const float* x0, float x0_scale, KParams& P);
Hyper initial_hyper();
// batched problems (laps_batch.cu)
const void* batch_fn(int cpl);
size_t batch_smem(int cpl, int cap_pad, int SL);
int batch_threads();
int batch_gw(int64_t d, int cpl, int widen);
int batch_blocks_per_sm(int cpl, int cap_pad, int SL);
cudaError_t batch_launch(int cpl, int G, const KParams* probs, const int* gw, const int2* sched,
                         const Coefs* coefs, int n, int mode, int n_iters, int SL, int cap_pad, unsigned* bar,
                         int* status, long long timeout_ns, int bar_extra, uint64_t seed, cudaStream_t st);
// Blocks that hold each problem's chains: sched[k] = (first block, blocks) for
// problems of dimension d[k] and M[k] chains on G blocks of the shape (cpl, widen).
void batch_schedule(const int64_t* d, const int64_t* M, int n, int cpl, int widen, int G, int2* sched);
// streamed path (laps_streamed.cu)
laps_status streamed_setup(laps_ctx* c);
laps_status streamed_alloc(laps_ctx* c);
laps_status streamed_init(laps_ctx* c, const float* x0, float x0_scale, cudaStream_t st);
laps_status streamed_step(laps_ctx* c, int n_iters, cudaStream_t st);
// dense-precision Gaussian (laps_gauss_dense.cu): G = -W P, LP = -1/2 sum W (P W)
constexpr int kDenseMaxDim = 512;
// forms of the logistic-regression contraction: FP32 on the CUDA cores, BF16
// tensor cores, tensor cores at FP32 accuracy (three-term BF16 split)
enum GradForm : int { GF_F32 = 0, GF_BF16 = 1, GF_X3 = 2 };
// (guard: as for the logistic-regression gradients, laps_logreg.cuh)
cudaError_t gauss_dense_grad(const float* P, int d_pad, int d, const float* W, int64_t M, float* G,
                             float2* LP, cudaStream_t st, const int* guard = nullptr);
inline bool streamed_kind(int kind) { return kind == TGT_LOGREG || kind == TGT_GAUSS_DENSE || kind == TGT_USER; }
// USER targets: calls the callback for W [M][ld] and converts its FP32 log p into
// the float-float partial the chain updates read (lp32: device [M] scratch)
laps_status user_grad(const laps_target* tg, const float* W, int64_t M, int ld, float* G, float* lp32,
                      float2* LP, cudaStream_t st);
// The data split of a contraction target's FP32 gradient (1 but for LOGREG), and
// the gradient with it: gpart [S][M][kp], lpart [S][M], summed in order by the caller.
int streamed_target_splits(const laps_target* tg, int64_t M);
laps_status streamed_target_grad(const laps_target* tg, const float* W, int64_t M, int S, float* gpart,
                                 float2* lpart, cudaStream_t st);
laps_status status_error(int device_status);
void stats_from_hyper(const Hyper& h, laps_stats* out);
void coefs_table(Coefs& cf);
void launch_fill(float* p, float v, int64_t n, cudaStream_t st);
// writes the integrator tables with a kernel that takes them by value (stream-ordered,
// nothing on the host is read after the call returns)
void launch_set_coefs(Coefs* dst, const Coefs& cf, cudaStream_t st);
void launch_unpack(const float* src, const float* scale, float* dst, int64_t M, int d, int d_pad,
                   cudaStream_t st);
}  // namespace laps
