// laps_streamed.cu -- the streamed LAPS path, for targets whose gradient is a
// contraction over the whole ensemble (logistic regression): the chain state
// lives in global memory (L2-resident at the sizes served) and one Algorithm 1
// iteration is a fixed sequence of launches on one stream,
//
//   unadjusted step (App. E):  seg[O1 B A] grad seg[B O2 close] fin_slice fin_gather switch
//   MAMS proposal (App. F):    seg[refresh O1 B A] (grad seg[B (O2 O1 B) A])... grad seg[B O2 close]
//                              fin_slice fin_gather
//
// seg applies the maps of one stretch between two gradient evaluations to every
// chain (a warp per chain, CPL coordinates per lane); grad is the target's
// ensemble gradient kernel; fin_slice / fin_gather are the reduction and the
// finalise shared with the register-resident kernel, split at a kernel
// boundary instead of a grid barrier.  The first launch of an iteration
// evaluates its guard (phase as expected, run not done) into go[0]; every
// later launch of the iteration reads it, so an iteration enqueued past the
// switch or past the end is a sequence of empty launches.  The host enqueues
// iterations in chunks and reads the phase machine between chunks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "laps_internal.h"
#include "laps_logreg.cuh"

namespace laps {

constexpr int kSegThreads = 256;
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kFinThreads = 256;

// ---------------------------------------------------------------- chain update
template <int CPL>
__global__ void __launch_bounds__(kSegThreads, CPL <= 4 ? 3 : 1) seg_kernel(const KParams P, const SegOp op) {
    constexpr int NB = CPL / 4;
    extern __shared__ __align__(16) float seg_smem[];
    __shared__ Hyper H;
    __shared__ float s_eps, s_c1, s_c2s;
    __shared__ int s_go;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dp = P.d_pad;
    if (tid == 0) {
        H = *P.hyper;
        int go = 1;
        if (op.init == 0) go = op.first ? ((!H.done && H.phase == op.phase) ? 1 : 0) : P.go[0];
        if (op.first && blockIdx.x == 0) {
            P.go[0] = go;
            if (op.init) P.go[1] = 0;
        }
        s_go = go;
        set_step_scalars(H, P.d, s_eps, s_c1, s_c2s);
    }
    __syncthreads();
    if (!s_go) return;

    const int cpb = (P.M + P.G - 1) / P.G;
    const int mb0 = blockIdx.x * cpb, mb1 = min(P.M, mb0 + cpb);
    const float eps = s_eps, c1 = s_c1, c2s = s_c2s;
    const float dm1 = (float)(P.d - 1), inv_dm1 = 1.0f / (float)(P.d - 1);
    const uint32_t t0 = (uint32_t)H.t;
    const bool columns = op.close || op.init == 2;

    float sg[CPL];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int j = lane + 32 * k;
        float4 s = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
        if (j < P.nblk) s = *reinterpret_cast<const float4*>(P.sigma + 4 * j);
        sg[4 * k] = s.x; sg[4 * k + 1] = s.y; sg[4 * k + 2] = s.z; sg[4 * k + 3] = s.w;
    }
    float qs[NQ][CPL];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int c = 0; c < CPL; ++c) qs[q][c] = 0.0f;
    ff cs[NCS];
#pragma unroll
    for (int k = 0; k < NCS; ++k) cs[k] = ff_make(0.0f);

    auto load = [&](const float* src, int64_t m, float(&v)[CPL]) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int j = lane + 32 * k;
            float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (j < P.nblk) a = *reinterpret_cast<const float4*>(src + (size_t)m * dp + 4 * j);
            v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
        }
    };
    auto store = [&](float* dst, int64_t m, const float(&v)[CPL]) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int j = lane + 32 * k;
            if (j < P.nblk)
                *reinterpret_cast<float4*>(dst + (size_t)m * dp + 4 * j) =
                    make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        }
    };
    // x-space gradient partials of the gradient kernel, summed in order, to y-space
    auto load_grad = [&](int64_t m, float(&g)[CPL], ff& lp) {
#pragma unroll
        for (int q = 0; q < CPL; ++q) g[q] = 0.0f;
        lp = ff_make(0.0f);
        for (int s = 0; s < P.nsplit; ++s) {
            float v[CPL];
            load(P.gpart + (size_t)s * P.M * dp, m, v);
#pragma unroll
            for (int q = 0; q < CPL; ++q) g[q] += v[q];
            const float2 l = P.lpart[(size_t)s * P.M + m];
            lp = ff_add(lp, ff{l.x, l.y});
        }
#pragma unroll
        for (int q = 0; q < CPL; ++q) g[q] *= sg[q];
    };
    // mixed precision, unadjusted phase: the tensor-core gradient reads x as two BF16 terms
    const bool wb = P.Wb != nullptr && op.phase == 0 && op.init != 3;
    auto store_W = [&](int64_t m, const float(&y)[CPL]) {
        float x[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) x[q] = sg[q] * y[q];
        store(P.W, m, x);
        if (wb) {
            __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(P.Wb) + (size_t)m * 2 * dp;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int j = lane + 32 * k;
                if (j >= P.nblk) continue;
                __nv_bfloat16 hi[4], lo[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    hi[c] = __float2bfloat16_rn(x[4 * k + c]);
                    lo[c] = __float2bfloat16_rn(x[4 * k + c] - __bfloat162float(hi[c]));
                }
                *reinterpret_cast<uint2*>(row + 4 * j) = *reinterpret_cast<const uint2*>(hi);
                *reinterpret_cast<uint2*>(row + dp + 4 * j) = *reinterpret_cast<const uint2*>(lo);
            }
        }
    };

    for (int m = mb0 + warp; m < mb1; m += kSegWarps) {
        const uint32_t mg = (uint32_t)(m + P.m0);  // the chain's index in the whole ensemble
        float y[CPL], u[CPL], g[CPL];
        ff lp = ff_make(0.0f), dl = ff_make(0.0f);
        if (op.init == 1) {
            // Alg. 1 input: x0 from the caller, or x0_scale N(0, I) from the tag-0 stream
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int j = lane + 32 * k;
                float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (j < P.nblk && P.x0 == nullptr)
                    normals4(j, mg, 0u, TAG_X0 | (P.pid << 8), P.seed_lo, P.seed_hi, z);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = 4 * j + c;
                    float v = 0.0f;
                    if (j < P.nblk && i < P.d) v = P.x0 ? P.x0[(size_t)m * P.d + i] : P.x0_scale * z[c];
                    y[4 * k + c] = v;
                }
            }
            store(P.y, m, y);
            store_W(m, y);
            continue;
        }
        if (op.init == 3) {  // re-evaluation: the accepted points as the gradient input
            load(P.y, m, y);
            store_W(m, y);
            continue;
        }
        if (op.init == 4) {  // re-evaluation: accepted g and log p from the gradient kernel
            load_grad(m, g, lp);
            store(P.g, m, g);
            if (lane == 0) P.logp_ff[m] = make_float2(lp.hi, lp.lo);
            continue;
        }
        if (op.init == 2) {
            // App. C "Initialization": u0 along the gradient (a random direction if it vanishes)
            load(P.y, m, y);
            load_grad(m, g, lp);
            float n2 = 0.0f;
#pragma unroll
            for (int q = 0; q < CPL; ++q) n2 = fmaf(g[q], g[q], n2);
            n2 = group_sum<32>(n2);
#pragma unroll
            for (int q = 0; q < CPL; ++q) u[q] = 0.0f;
            o_update<32, CPL>(P, lane, true, mg, 0xFFFFFFFFu, TAG_O1, 0.0f, 1.0f, u);
            if (n2 > 0.0f) {
                const float inv = 1.0f / sqrtf(n2);
#pragma unroll
                for (int q = 0; q < CPL; ++q) u[q] = g[q] * inv;
            }
            bool bad = !isfinite(lp.hi);
#pragma unroll
            for (int q = 0; q < CPL; ++q) bad = bad || !(finite_f(y[q]) && finite_f(g[q]));
            if (bad) atomicCAS(P.status, ST_OK, ST_NONFINITE);
            store(P.u, m, u);
            store(P.g, m, g);
            if (lane == 0) P.logp_ff[m] = make_float2(lp.hi, lp.lo);
        } else {
            load(op.first ? P.y : P.yw, m, y);
            load(op.first ? P.u : P.uw, m, u);
            if (op.first) {
                load(P.g, m, g);
                const float2 l = P.logp_ff[m];
                lp = ff{l.x, l.y};
            } else {
                const float2 l = P.lpw[m], e = P.dlw[m];
                lp = ff{l.x, l.y};
                dl = ff{e.x, e.y};
            }
            if (op.after_grad) {
                ff lpn;
                load_grad(m, g, lpn);
                dl = ff_add(dl, ff_neg(ff_add(lpn, ff_neg(lp))));  // -log p(x') + log p(x)
                lp = lpn;
            }
            if (op.refresh) {
                // App. F step 2: u uniform on the sphere
                float n2 = 0.0f;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const int j = lane + 32 * k;
                    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (j < P.nblk)
                        normals4(j, mg, (uint32_t)H.p, TAG_REFRESH | (P.pid << 8), P.seed_lo, P.seed_hi, z);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float v = (4 * j + c < P.d) ? z[c] : 0.0f;
                        u[4 * k + c] = v;
                        n2 = fmaf(v, v, n2);
                    }
                }
                n2 = group_sum<32>(n2);
                const float inv = n2 > 0.0f ? 1.0f / sqrtf(n2) : 0.0f;
#pragma unroll
                for (int q = 0; q < CPL; ++q) u[q] *= inv;
            }
            if (op.bA != 0.0f) b_update<32, CPL>(op.bA * eps, inv_dm1, dm1, g, u, dl);
            if (op.o2_step >= 0) o_update<32, CPL>(P, lane, true, mg, t0 + op.o2_step, TAG_O2, c1, c2s, u);
            if (op.o1_step >= 0) o_update<32, CPL>(P, lane, true, mg, t0 + op.o1_step, TAG_O1, c1, c2s, u);
            if (op.bB != 0.0f) b_update<32, CPL>(op.bB * eps, inv_dm1, dm1, g, u, dl);
            if (op.a != 0.0f) {
                const float ae = op.a * eps;
#pragma unroll
                for (int q = 0; q < CPL; ++q) y[q] = fmaf(ae, u[q], y[q]);
                store_W(m, y);
            }
            if (!op.close) {
                store(P.yw, m, y);
                store(P.uw, m, u);
                if (lane == 0) {
                    P.lpw[m] = make_float2(lp.hi, lp.lo);
                    P.dlw[m] = make_float2(dl.hi, dl.lo);
                }
                continue;
            }
            // ---- close: non-finite check, accept / reject (App. F step 5), keep or revert
            bool bad = !(isfinite(lp.hi) && isfinite(dl.hi));
#pragma unroll
            for (int q = 0; q < CPL; ++q) bad = bad || !(finite_f(y[q]) && finite_f(u[q]) && finite_f(g[q]));
            bad = __any_sync(0xffffffffu, bad);
            bool keep = !bad;
            float a_m = 0.0f;
            if (H.phase == 1) {
                const uint4 r = philox4x32_10(
                    make_uint4(0u, mg, (uint32_t)H.p, TAG_MH | (P.pid << 8)), P.seed_lo,
                    P.seed_hi);
                const ff s = ff_add(dl, logf(u01(r.x)));
                keep = !bad && (s.hi < 0.0f || (s.hi == 0.0f && s.lo < 0.0f));
                a_m = bad ? 0.0f : (dl.hi <= 0.0f ? 1.0f : expf(-(dl.hi + dl.lo)));
            }
            if (keep) {
                store(P.y, m, y);
                store(P.u, m, u);
                store(P.g, m, g);
                if (lane == 0) P.logp_ff[m] = make_float2(lp.hi, lp.lo);
            } else {
                load(P.y, m, y);  // the accepted state stays; its values enter the sums
                load(P.g, m, g);
            }
            if (H.phase == 0) {
                if (bad) {
                    cs[CS_NBAD] = ff_add(cs[CS_NBAD], 1.0f);
                } else {
                    cs[CS_DSUM] = ff_add(cs[CS_DSUM], dl);
                    cs[CS_DSQ] = ff_add(cs[CS_DSQ], ff_f(dl) * ff_f(dl));
                    cs[CS_NFIN] = ff_add(cs[CS_NFIN], 1.0f);
                }
            } else {
                cs[CS_ASUM] = ff_add(cs[CS_ASUM], a_m);
                if (bad) cs[CS_NBAD] = ff_add(cs[CS_NBAD], 1.0f);
            }
        }
        // per-coordinate sums of y, y^2, g, y g over this warp's chains (Eq. ECA)
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            qs[0][q] += y[q];
            qs[1][q] = fmaf(y[q], y[q], qs[1][q]);
            qs[2][q] += g[q];
            qs[3][q] = fmaf(y[q], g[q], qs[3][q]);
        }
    }
    if (!columns) return;

    // ---- block columns: warps in order, float-float
    const int nq = ens_nq(P, H);
    float* sq = seg_smem;                                        // [NQ][warps][dp]
    ff* scs = reinterpret_cast<ff*>(sq + (size_t)NQ * kSegWarps * dp);  // [warps][NCS]
    for (int qd = 0; qd < nq; ++qd)
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int j = lane + 32 * k;
            if (j < P.nblk)
#pragma unroll
                for (int c = 0; c < 4; ++c) sq[((size_t)qd * kSegWarps + warp) * dp + 4 * j + c] = qs[qd][4 * k + c];
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NCS; ++k) scs[warp * NCS + k] = cs[k];
    __syncthreads();
    const int G = P.G;
    for (int col = tid; col < nq * dp; col += blockDim.x) {
        const int qd = col / dp, i = col - qd * dp;
        if (i >= P.d) continue;
        ff s = ff_make(0.0f);
        for (int w = 0; w < kSegWarps; ++w) s = ff_add(s, sq[((size_t)qd * kSegWarps + w) * dp + i]);
        P.part[((size_t)qd * dp + i) * G + blockIdx.x] = make_float2(s.hi, s.lo);
    }
    if (tid < NCS) {
        ff s = ff_make(0.0f);
        for (int w = 0; w < kSegWarps; ++w) s = ff_add(s, scs[w * NCS + tid]);
        P.part[((size_t)NQ * dp + tid) * G + blockIdx.x] = make_float2(s.hi, s.lo);
    }
}

// ---------------------------------------------------------------- reduction and finalise
// One launch: every block reduces its slice of coordinates (ens_slice); the
// last block to finish, found by a ticket counter (no block waits for
// another), gathers and runs the finalise (ens_gather).
__global__ void __launch_bounds__(kFinThreads) fin_kernel(const KParams P) {
    // slice: [NQ smax + NCS] float-float; then, in the last block, [d_pad] Var y
    extern __shared__ __align__(16) float fin_smem[];
    __shared__ Hyper H;
    __shared__ FinShared FS;
    __shared__ unsigned s_ticket;
    unsigned* count = reinterpret_cast<unsigned*>(P.go + 2);
    if (threadIdx.x == 0) H = *P.hyper;
    __syncthreads();
    if (!P.go[0]) return;
    ens_slice(P, H, reinterpret_cast<ff*>(fin_smem), blockIdx.x, gridDim.x);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(count, 1u);
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    __threadfence();
    ens_gather(P, H, fin_smem, FS);
    if (threadIdx.x == 0) {
        *P.hyper = H;
        ens_trace_row(P, H, FS.now);
        P.go[1] = FS.sw;
        *count = 0u;  // ready for the next launch
    }
    if (FS.sw)  // Sec. 4: the diagonal preconditioner, fixed from now on
        for (int i = threadIdx.x; i < P.d; i += blockDim.x) {
            const float v = fin_smem[i];
            P.sigma[i] = v > 0.0f ? sqrtf(v) : 1.0f;
        }
}

// Chain-sharded ensemble: this rank's totals of every column row (the block
// columns added in the order and grouping the finalise's slice owners use, so
// that one rank reproduces the unsharded sums bit for bit).  One warp per row.
__global__ void rank_totals_kernel(const float2* __restrict__ part, int G, int rows, float2* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rows) return;
    ff s = lane_col_sum(part + (size_t)row * G, G, lane, 32);
    s = group_sum_ff<32>(s);
    if (lane == 0) out[row] = make_float2(s.hi, s.lo);
}
// every rank's totals [n][rows] (rank order) into the columns layout [rows][n]
__global__ void shard_columns_kernel(const float2* __restrict__ recv, int n, int rows, float2* __restrict__ part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * rows) return;
    const int r = k / rows, row = k - r * rows;
    part[(size_t)row * n + r] = recv[k];
}

// Sec. 4, once after the switch: y = x / sigma and g_y = sigma g_x of the accepted state
__global__ void precondition_kernel(const KParams P) {
    const int64_t n = (int64_t)P.M * P.d_pad;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % P.d_pad);
        if (i >= P.d) continue;
        const float s = P.sigma[i];
        P.y[k] = P.y[k] / s;
        P.g[k] = P.g[k] * s;
    }
}

// ---------------------------------------------------------------- host
namespace {

const void* seg_fn(int cpl) {
    switch (cpl) {
    case 4: return (const void*)seg_kernel<4>;
    case 8: return (const void*)seg_kernel<8>;
    case 16: return (const void*)seg_kernel<16>;
    }
    return nullptr;
}

laps_status launch_seg(laps_ctx* c, const KParams& P, const SegOp& op, cudaStream_t st) {
    void* args[] = {const_cast<KParams*>(&P), const_cast<SegOp*>(&op)};
    cudaError_t e = cudaLaunchKernel(seg_fn(c->seg_cpl), dim3(c->seg_G), dim3(kSegThreads), args,
                                     c->seg_smem, st);
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "seg_kernel");
}

// the gradient of the working points in contraction form `form` (GF_*; the
// dense Gaussian and user targets have one form).  guard: the iteration's guard
// word (the kernels return at once when it is 0: an iteration enqueued past a
// stop or a switch), or null outside the iteration protocol.  A user callback
// runs on the host's schedule and cannot read it.
laps_status launch_grad(laps_ctx* c, int form, cudaStream_t st, const int* guard) {
    cudaError_t e;
    if (c->tg->kind == TGT_GAUSS_DENSE) {
        e = gauss_dense_grad(c->tg->prec_dense, c->d_pad, c->d, c->W, c->M, c->gpart, c->lpart, st, guard);
        return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "dense Gaussian gradient");
    }
    if (c->tg->kind == TGT_USER) return user_grad(c->tg, c->W, c->M, c->d_pad, c->gpart, c->ulp, c->lpart, st);
    if (form == GF_BF16)
        e = logreg_grad_mma(c->tg->lr, c->tmW, c->W, c->M, c->nsplit_mma, c->rps_mma, c->gpart, c->lpart,
                            c->status, c->cfg.barrier_timeout_ns, st, guard);
    else if (form == GF_X3)
        e = logreg_grad_x3(c->tg->lr, c->W, c->M, c->nsplit_x3, c->rps_x3, c->gpart, c->lpart, c->status,
                           c->cfg.barrier_timeout_ns, st, guard);
    else
        e = logreg_grad_f32(c->tg->lr, c->W, c->M, c->nsplit, c->gpart, c->lpart, st, guard);
    return e == cudaSuccess ? LAPS_OK
                            : cuda_fail(e, form == GF_BF16 ? "logreg gradient (tensor cores)"
                                           : form == GF_X3 ? "logreg gradient (tensor cores, three-term split)"
                                                           : "logreg gradient");
}

// data splits (gradient partials) the given form writes
int nsplit_of(const laps_ctx* c, int form) {
    return form == GF_BF16 ? c->nsplit_mma : form == GF_X3 ? c->nsplit_x3 : c->nsplit;
}

laps_status launch_fin(laps_ctx* c, const KParams& P, cudaStream_t st) {
    if (!c->sharded) {
        fin_kernel<<<c->fin_G, kFinThreads, std::max(c->fin_slice_smem, c->fin_gather_smem), st>>>(P);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "finalise kernel");
    }
    // the one exchange of a chain-sharded iteration (Eq. ECA's sums): this rank's
    // column totals, gathered from every rank in rank order, then the finalise on
    // the gathered columns (one per rank), identical on every rank
    const int rows = (int)rows_fb(c->d_pad);
    rank_totals_kernel<<<(rows * 32 + 255) / 256, 256, 0, st>>>(c->part, P.G, rows, c->shard_send);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rank totals kernel");
    const size_t bytes = (size_t)rows * sizeof(float2);
    if (c->shard_fn) {
        const int r = c->shard_fn(c->shard_send, c->shard_recv, bytes, (void*)st, c->shard_user);
        if (r != 0) return fail(LAPS_ERR_CUDA, "allgather callback returned " + std::to_string(r));
    } else {
        e = cudaMemcpyAsync(c->shard_recv, c->shard_send, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy of the rank totals");
    }
    const int n = c->n_ranks;
    shard_columns_kernel<<<(n * rows + 255) / 256, 256, 0, st>>>(c->shard_recv, n, rows, c->shard_part);
    KParams Q = P;
    Q.part = c->shard_part;
    Q.G = n;
    fin_kernel<<<c->fin_G, kFinThreads, std::max(c->fin_slice_smem, c->fin_gather_smem), st>>>(Q);
    e = cudaGetLastError();
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "finalise kernel");
}

SegOp seg_op(int phase) {
    SegOp o;
    std::memset(&o, 0, sizeof(o));
    o.phase = phase;
    o.o2_step = -1;
    o.o1_step = -1;
    return o;
}

#define LCK(call)                              \
    do {                                       \
        laps_status s_ = (call);               \
        if (s_ != LAPS_OK) return s_;          \
    } while (0)

// one Alg. 1 iteration of the given phase
laps_status enqueue_iteration(laps_ctx* c, int phase, cudaStream_t st) {
    KParams P;
    fill_params(c, 1, nullptr, 0.0f, P);
    P.nsplit = nsplit_of(c, phase == 0 ? c->gf_unadj : c->gf_adj);
    if (phase == 0) {
        // O_{eps/2} B_{eps/2} A_eps [grad] B_{eps/2} O_{eps/2}  (leapfrog, App. E)
        SegOp a = seg_op(0);
        a.first = 1;
        a.o1_step = 0;
        a.bB = c->cf.b[INTEG_LF][0];
        a.a = c->cf.a[INTEG_LF][0];
        LCK(launch_seg(c, P, a, st));
        LCK(launch_grad(c, c->gf_unadj, st, c->go));
        SegOp b = seg_op(0);
        b.after_grad = 1;
        b.bA = c->cf.b[INTEG_LF][1];
        b.o2_step = 0;
        b.close = 1;
        LCK(launch_seg(c, P, b, st));
        return launch_fin(c, P, st);
    }
    // MAMS proposal: full refresh, N steps of O Phi O, accept / reject (App. F)
    const int I = c->adj_integ, K = c->cf.K[I], N = c->cfg.steps_per_proposal;
    SegOp a = seg_op(1);
    a.first = 1;
    a.refresh = 1;
    a.o1_step = 0;
    a.bB = c->cf.b[I][0];
    a.a = c->cf.a[I][0];
    LCK(launch_seg(c, P, a, st));
    for (int n = 0; n < N; ++n) {
        for (int s = 1; s < K - 1; ++s) {
            LCK(launch_grad(c, c->gf_adj, st, c->go));
            SegOp m = seg_op(1);
            m.after_grad = 1;
            m.bA = c->cf.b[I][s];
            m.a = c->cf.a[I][s];
            LCK(launch_seg(c, P, m, st));
        }
        LCK(launch_grad(c, c->gf_adj, st, c->go));
        SegOp e = seg_op(1);
        e.after_grad = 1;
        e.bA = c->cf.b[I][K - 1];
        e.o2_step = n;
        if (n + 1 < N) {
            e.o1_step = n + 1;
            e.bB = c->cf.b[I][0];
            e.a = c->cf.a[I][0];
        } else {
            e.close = 1;
        }
        LCK(launch_seg(c, P, e, st));
    }
    return launch_fin(c, P, st);
}

laps_status read_hyper(laps_ctx* c, cudaStream_t st, Hyper& h) {
    cudaError_t e = cudaMemcpyAsync(c->h_hyper, c->hyper, sizeof(Hyper), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the phase machine");
    h = *c->h_hyper;
    return LAPS_OK;
}

}  // namespace

laps_status streamed_setup(laps_ctx* c) {
    const int dp = c->d_pad;
    if (!streamed_kind(c->tg->kind)) return fail(LAPS_ERR_UNSUPPORTED, "streamed path: LOGREG and GAUSS_DENSE only");
    c->streamed = true;
    c->seg_cpl = dp <= 128 ? 4 : dp <= 256 ? 8 : dp <= 512 ? 16 : 0;
    if (c->seg_cpl == 0) return fail(LAPS_ERR_UNSUPPORTED, "streamed path: d_pad > 512");
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    // A chain update is a chain of dependent reductions and Philox rounds, so the
    // kernel wants many chains in flight; but every block's columns are one more
    // partial for the finalise to add.  Up to four chains per warp, as long as
    // every SM keeps a block (M = 8192: 256 blocks, 0.149 -> 0.143 ms per
    // mixed-precision logistic-regression step against one chain per warp).
    const int64_t g1 = (c->M + kSegWarps - 1) / kSegWarps, g4 = (c->M + 4 * kSegWarps - 1) / (4 * kSegWarps);
    c->seg_G = (int)std::min<int64_t>(g1, std::max<int64_t>(g4, nsm));
    c->G = c->seg_G;
    c->seg_smem = (size_t)NQ * kSegWarps * dp * sizeof(float) + (size_t)kSegWarps * NCS * sizeof(ff);
    e = ensure_dyn_smem((const void*)seg_fn(c->seg_cpl), c->seg_smem);
    if (e != cudaSuccess) return cuda_fail(e, "seg_kernel attribute");
    c->fin_G = std::max(1, std::min(2 * nsm, c->d));
    c->smax = (c->d + c->fin_G - 1) / c->fin_G;
    c->fin_slice_smem = ((size_t)NQ * c->smax + NCS) * sizeof(ff);
    c->fin_gather_smem = (size_t)dp * sizeof(float);
    // data splits of the FP32 gradient: whole waves of (chain tile, row range) blocks
    c->nsplit = c->tg->kind == TGT_LOGREG ? logreg_f32_splits(c->tg->lr, c->M, nsm)
                                          : 1;  // one evaluation writes every coordinate of its chains
    c->adj_integ = (c->d > c->cfg.mn4_min_dim) ? INTEG_MN4 : INTEG_MN2;
    coefs_table(c->cf);
    const int pr = (int)c->cfg.precision;
    c->gf_unadj = pr == LAPS_MIXED || pr == LAPS_MIXED_BF16X3 ? GF_BF16 : pr == LAPS_BF16X3 ? GF_X3 : GF_F32;
    c->gf_adj = pr == LAPS_BF16X3 || pr == LAPS_MIXED_BF16X3 ? GF_X3 : GF_F32;
    if (c->gf_unadj == GF_BF16 && (!logreg_mma_supported(dp) || c->tg->lr.Xb == nullptr))
        return fail(LAPS_ERR_UNSUPPORTED, "mixed precision is built for LOGREG with d <= 128");
    if (c->gf_adj == GF_X3 && (!logreg_x3_supported(dp) || c->tg->lr.X3b == nullptr))
        return fail(LAPS_ERR_UNSUPPORTED, "the three-term tensor-core form is built for LOGREG with d <= 128");
    c->mixed = c->gf_unadj == GF_BF16;
    if (c->gf_unadj == GF_BF16) c->nsplit_mma = logreg_mma_splits(c->tg->lr, c->M, nsm, &c->rps_mma);
    if (c->gf_unadj == GF_X3 || c->gf_adj == GF_X3)
        c->nsplit_x3 = logreg_x3_splits(c->tg->lr, c->M, nsm, &c->rps_x3);
    if (c->mixed) c->M_pad = (c->M + 127) / 128 * 128;
    return LAPS_OK;
}

laps_status streamed_alloc(laps_ctx* c) {
    const size_t Md = (size_t)c->M * c->d_pad;
    const int S = std::max({c->nsplit, c->nsplit_mma, c->nsplit_x3});
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        c->allocs.push_back(*p);
        return true;
    };
    bool ok = alloc((void**)&c->yw, Md * 4) && alloc((void**)&c->uw, Md * 4) &&
              alloc((void**)&c->W, Md * 4) && alloc((void**)&c->dlw, c->M * 8) &&
              alloc((void**)&c->lpw, c->M * 8) && alloc((void**)&c->gpart, (size_t)S * Md * 4) &&
              alloc((void**)&c->lpart, (size_t)S * c->M * 8) && alloc((void**)&c->go, 4 * sizeof(int));
    if (ok && c->mixed) ok = alloc(&c->Wb, (size_t)c->M_pad * 2 * c->d_pad * 2);
    if (ok && c->tg->kind == TGT_USER) ok = alloc((void**)&c->ulp, (size_t)c->M * 4);
    if (!ok) return fail(LAPS_ERR_OOM, "device allocation of the streamed working state failed");
    if (cudaMallocHost((void**)&c->h_hyper, sizeof(Hyper)) != cudaSuccess)
        return fail(LAPS_ERR_OOM, "pinned host allocation failed");
    cudaMemset(c->W, 0, Md * 4);
    cudaMemset(c->go, 0, 4 * sizeof(int));
    if (c->mixed) {
        cudaMemset(c->Wb, 0, (size_t)c->M_pad * 2 * c->d_pad * 2);  // rows past M stay zero
        cudaError_t e = logreg_mma_wmap(c->tmW, c->Wb, c->M_pad, c->d_pad);
        if (e != cudaSuccess) return cuda_fail(e, "tensor map of the points");
    }
    return LAPS_OK;
}

namespace {
// after the switch of a mixed-precision run: the accepted g and log p again in
// the adjusted phase's arithmetic (the unadjusted phase computed them on the
// BF16 data), so that every Metropolis test compares log p of one arithmetic
laps_status reevaluate_adjusted(laps_ctx* c, cudaStream_t st) {
    KParams P;
    fill_params(c, 1, nullptr, 0.0f, P);
    P.nsplit = nsplit_of(c, c->gf_adj);
    SegOp a = seg_op(1);
    a.init = 3;
    LCK(launch_seg(c, P, a, st));
    LCK(launch_grad(c, c->gf_adj, st, nullptr));
    SegOp b = seg_op(1);
    b.init = 4;
    LCK(launch_seg(c, P, b, st));
    return LAPS_OK;
}

// the one-time work of the switch, enqueued by the host once it reads the new
// phase (the iterations enqueued after the switching one are empty): the
// accepted state into preconditioned coordinates, then, for the mixed forms,
// its g and log p again in the adjusted phase's arithmetic
laps_status after_switch(laps_ctx* c, cudaStream_t st) {
    KParams P;
    fill_params(c, 1, nullptr, 0.0f, P);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (c->M * c->d_pad + 255) / 256));
    precondition_kernel<<<blocks, 256, 0, st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "precondition_kernel");
    if (c->gf_unadj != c->gf_adj) LCK(reevaluate_adjusted(c, st));
    c->refreshed = true;
    return LAPS_OK;
}
}  // namespace

laps_status streamed_init(laps_ctx* c, const float* x0, float x0_scale, cudaStream_t st) {
    KParams P;
    fill_params(c, 0, x0, x0_scale, P);
    P.nsplit = nsplit_of(c, c->gf_unadj);
    SegOp a = seg_op(0);
    a.first = 1;
    a.init = 1;
    LCK(launch_seg(c, P, a, st));
    LCK(launch_grad(c, c->gf_unadj, st, nullptr));
    SegOp b = seg_op(0);
    b.init = 2;
    LCK(launch_seg(c, P, b, st));
    LCK(launch_fin(c, P, st));
    c->last_stream = st;
    c->refreshed = false;
    return LAPS_OK;
}

laps_status streamed_step(laps_ctx* c, int n_iters, cudaStream_t st) {
    c->last_stream = st;
    Hyper h;
    LCK(read_hyper(c, st, h));
    if (h.phase == 1 && !c->refreshed) LCK(after_switch(c, st));
    const long long target = (long long)h.iters + n_iters;
    while (!h.done && h.iters < target) {
        const int chunk = h.phase == 0 ? 32 : 4;
        const int k = (int)std::min<long long>(chunk, target - h.iters);
        for (int i = 0; i < k; ++i) LCK(enqueue_iteration(c, h.phase, st));
        LCK(read_hyper(c, st, h));
        int s = 0;
        cudaError_t e = cudaMemcpy(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
        if (s != ST_OK) return status_error(s);
        if (h.phase == 1 && !c->refreshed) LCK(after_switch(c, st));
    }
    return LAPS_OK;
}

int streamed_target_splits(const laps_target* tg, int64_t M) {
    if (tg->kind != TGT_LOGREG) return 1;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return logreg_f32_splits(tg->lr, M, nsm);
}

laps_status streamed_target_grad(const laps_target* tg, const float* W, int64_t M, int S, float* gpart,
                                 float2* lpart, cudaStream_t st) {
    if (tg->kind == TGT_GAUSS_DENSE) {
        cudaError_t e = gauss_dense_grad(tg->prec_dense, tg->d_pad, tg->d, W, M, gpart, lpart, st);
        return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "dense Gaussian gradient");
    }
    cudaError_t e = logreg_grad_f32(tg->lr, W, M, S, gpart, lpart, st);
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "logreg gradient");
}

}  // namespace laps
