// laps_finalise.cuh -- the ensemble reductions and the finalise of one
// Algorithm 1 iteration, shared by the register-resident kernel and the
// streamed path.
//
// Input: per-block columns P.part[(q * d_pad + i) * G + b] (float-float sums
// over block b's chains of y_i, y_i^2, g_i, y_i g_i) and per-chain sums
// P.part[(NQ * d_pad + k) * G + b] (energy error, its square, counts,
// acceptance).  Two steps separated by a grid-wide ordering point (a grid
// barrier, or a kernel boundary):
//   ens_slice   block bs of nsb reduces, in block order, the columns of its
//               slice of coordinates and derives Var, V_ii (App. B), the
//               window statistic delta[x_i^2] (Eq. "relative fluctuations")
//               and b^2 (Eq. "bias"); the last block also reduces the
//               per-chain sums;
//   ens_gather  reads the d per-coordinate results and runs the finalise
//               (Sec. 3.1 controller, Eq. "L", the switch of Sec. 4, the
//               bisection of Sec. 5.1) on lane 0 of warp 0.
// Every sum has a fixed order, so the result does not depend on timing.
#pragma once
#include "laps_resident.cuh"

namespace laps {

__device__ __forceinline__ float fmax_nan(float a, float b) { return (b > a || b != b) ? b : a; }

// block-shared scratch and outputs of ens_gather
struct FinShared {
    ff wsum[4][kMaxThreads / 32];    // per-warp sums: Var x, (1 - V)^2, b^2, full-rank terms
    float wmax[2][kMaxThreads / 32];  // per-warp maxima: delta, b^2
    int sw;                           // 1: this iteration switched to the adjusted phase
    float eps, c1, c2s;               // step scalars of the next iteration
    unsigned long long now;           // %globaltimer at the finalise
};

// quantities per coordinate reduced this iteration (the g sums are unused after the
// switch; a diagonal Gaussian derives them from the y sums)
__device__ __forceinline__ int ens_nq(const KParams& P, const Hyper& H) {
    return (P.gauss_derived || (H.phase == 1 && P.mode == 1)) ? 2 : NQ;
}

// Step 3.  s_q: shared [NQ][P.smax] + [NCS] float-float; s_fr (full-rank proxy
// only, else nullptr): shared [P.smax K + K] float-float.  All threads of the
// block call it.
// Sum of src[c] over c = c0, c0 + step, ... < n (float-float pairs), added in
// that order; the loads are issued eight at a time so that their L2 latencies
// overlap.
__device__ __forceinline__ ff lane_col_sum(const float2* __restrict__ src, int n, int c0, int step) {
    ff s = ff_make(0.0f);
    for (int c = c0; c < n; c += 8 * step) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = c + u * step < n ? __ldcg(src + c + u * step) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c + u * step < n) s = ff_add(s, ff{v[u].x, v[u].y});
    }
    return s;
}

__device__ __forceinline__ void ens_slice(const KParams& P, const Hyper& H, ff* s_q, int bs,
                                          int nsb, ff* s_fr = nullptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int G = P.G, dp = P.d_pad;
    const int i0 = (int)(((long long)bs * P.d) / nsb);
    const int i1 = (int)(((long long)(bs + 1) * P.d) / nsb);
    const bool chain_owner = bs == nsb - 1;
    const int nq = ens_nq(P, H);
    const int ns = i1 - i0;
    const bool push = (P.mode == 1 && H.phase == 0);
    const int win_n = H.win_n;
    // the window values this thread will update, loaded before the reductions
    float4 w_pre = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 o_pre = make_float2(0.0f, 0.0f), e_pre = make_float2(0.0f, 0.0f);
    float sg_pre = 1.0f, pr_pre = 0.0f, iv_pre = 0.0f;
    // full-rank proxy: the means this iteration's block products were shifted by,
    // kept before this slice replaces them with the current means
    const bool fr_live = P.dfull_K > 0 && s_fr != nullptr;
    float* s_old = fr_live ? reinterpret_cast<float*>(s_fr + 2 * blockDim.x) : nullptr;  // [ns]
    if (tid < ns) {
        const int i = i0 + tid;
        if (fr_live) s_old[tid] = __ldcg(P.cstat + (size_t)i * NCO + CO_MY);
        if (push) {
            w_pre = P.win_sums[i];
            if (win_n >= P.T) o_pre = P.ring[(size_t)((win_n - P.T) % (P.T + 1)) * dp + i];
        }
        sg_pre = P.sigma[i];
        if (P.gauss_derived) pr_pre = P.prec[i];
        if (P.Ex2) {
            e_pre = P.Ex2[i];
            iv_pre = P.inv_varx2[i];
        }
    }
    // column sums over the blocks, in block order: one warp per (quantity, coordinate)
    const int n_pairs = nq * ns + (chain_owner ? NCS : 0);
    for (int pidx = warp; pidx < n_pairs; pidx += nwarps) {
        size_t row;
        if (pidx < nq * ns) row = (size_t)(pidx / ns) * dp + i0 + (pidx % ns);
        else row = (size_t)NQ * dp + (pidx - nq * ns);
        ff s = lane_col_sum(P.part + row * G, G, lane, 32);
        s = group_sum_ff<32>(s);
        if (lane == 0) {
            if (pidx < nq * ns) s_q[(pidx / ns) * P.smax + (pidx % ns)] = s;
            else s_q[NQ * P.smax + (pidx - nq * ns)] = s;
        }
    }
    __syncthreads();
    const float iM = 1.0f / (float)ens_chains(P);
    for (int k = tid; k < ns; k += blockDim.x) {
        const int i = i0 + k;
        const ff mean = ff_mulf(s_q[0 * P.smax + k], iM);
        const ff ey2 = ff_mulf(s_q[1 * P.smax + k], iM);
        const float var_y = ff_f(ff_add(ey2, ff_neg(ff_mul(mean, mean))));
        const float sgi = k == tid ? sg_pre : P.sigma[i];
        const float s2i = sgi * sgi;
        const ff ex2 = ff_mulf(ey2, s2i);
        float dv = 0.0f, del = 0.0f, b2 = 0.0f;
        if (nq == NQ) {
            // V_ii = -(E[y g] - E[y] E[g])  (App. B, Eq. ECA)
            const ff eg = ff_mulf(s_q[2 * P.smax + k], iM);
            const ff eyg = ff_mulf(s_q[3 * P.smax + k], iM);
            const float V = -ff_f(ff_add(eyg, ff_neg(ff_mul(mean, eg))));
            dv = (1.0f - V) * (1.0f - V);
        } else if (P.gauss_derived && (P.mode == 0 || H.phase == 0)) {
            // diagonal Gaussian: g_i = -prec_i sigma_i^2 y_i, so V_ii = prec_i sigma_i^2 Var[y_i]
            const float V = (k == tid ? pr_pre : P.prec[i]) * s2i * var_y;
            dv = (1.0f - V) * (1.0f - V);
        }
        if (push) {
            // moving window of E[x_i^2]: running sums over the last T values
            const float4 w = k == tid ? w_pre : P.win_sums[i];
            ff s1{w.x, w.y}, s2{w.z, w.w};
            float2* ring_i = P.ring + i;
            if (win_n >= P.T) {
                const float2 o = k == tid ? o_pre : ring_i[(size_t)((win_n - P.T) % (P.T + 1)) * dp];
                const ff old{o.x, o.y};
                s1 = ff_add(s1, ff_neg(old));
                s2 = ff_add(s2, ff_neg(ff_mul(old, old)));
            }
            s1 = ff_add(s1, ex2);
            s2 = ff_add(s2, ff_mul(ex2, ex2));
            P.win_sums[i] = make_float4(s1.hi, s1.lo, s2.hi, s2.lo);
            ring_i[(size_t)(win_n % (P.T + 1)) * dp] = make_float2(ex2.hi, ex2.lo);
            if (win_n + 1 >= P.T) {
                const float Tf = (float)P.T;
                const ff mu = ff_divf(s1, Tf);
                const float vv = ff_f(ff_add(s2, ff_neg(ff_mul(s1, mu)))) / (Tf - 1.0f);
                del = sqrtf(vv > 0.0f ? vv : 0.0f) / ff_f(mu);
            }
        }
        if (P.Ex2) {
            const float2 e = k == tid ? e_pre : P.Ex2[i];
            const float dd = ff_f(ff_add(ex2, ff_neg(ff{e.x, e.y})));
            b2 = dd * dd * (k == tid ? iv_pre : P.inv_varx2[i]);
        }
        float* co = P.cstat + (size_t)i * NCO;
        if (fr_live) {
            co[CO_MY] = ff_f(mean);
            co[CO_MG] = nq == NQ ? ff_f(ff_mulf(s_q[2 * P.smax + k], iM)) : 0.0f;
        }
        co[CO_VARY] = var_y;
        co[CO_VARX] = s2i * var_y;
        co[CO_DV] = dv;
        co[CO_DEL] = del;
        co[CO_B2] = b2;
    }
    if (chain_owner && tid < NCS) {
        const ff v = s_q[NQ * P.smax + tid];
        P.ctot[tid] = make_float2(v.hi, v.lo);
    }
    if (P.dfull_K > 0 && s_fr != nullptr && P.mode == 1 && H.phase == 0) {
        // App. B "Full rank": c_ik = Cov(y_i, s_k) with s_mk = g^m . z_k; the slice's
        // coordinates receive sum_k (z_ki + c_ik)^2 (Hutchinson over the K vectors).
        // With the blocks' shifted records (y' = y - ybar', s' = s - gbar'.z, see
        // fr_stride()):  M c_ik = sum_b Q_b,ik - (ybar_i - ybar'_i) sum_b S'_b,k.
        // Thread (group gb, vector k) adds the blocks gb, gb + BG, ...; the BG
        // partials are then added in group order.
        const int K = P.dfull_K, K4 = fr_k4(K);
        const size_t st = fr_stride(dp, K), oS = (size_t)dp * K4;
        const float* FR = reinterpret_cast<const float*>(reinterpret_cast<const char*>(P.part) + fr_offset(dp, G));
        const int KT = min(((K + 31) / 32) * 32, (int)blockDim.x), BG = (int)blockDim.x / KT;
        const int kt = tid % KT, gb = tid / KT;
#ifdef LAPS_PHASE_TIMING
        unsigned long long frs_t_ = global_ns();
#define FRS_MARK(k)                                                                   \
    do {                                                                              \
        __syncthreads();                                                              \
        if (blockIdx.x == LAPS_PHASE_BLOCK && threadIdx.x == 0 && P.phase_ns) {       \
            const unsigned long long now_ = global_ns();                              \
            P.phase_ns[12 + (k)] += now_ - frs_t_;                                    \
            frs_t_ = now_;                                                            \
        }                                                                             \
    } while (0)
#else
#define FRS_MARK(k) \
    do {            \
    } while (0)
#endif
        ff* s_part = s_fr;                                                   // [2][blockDim.x]
        float* s_sq = s_old + P.smax;                                        // [ns][K]
        const size_t step = (size_t)BG * st;
        for (int kk = 0; kk < ns; ++kk) {
            const int i = i0 + kk;
            const float dyb = ff_f(ff_mulf(s_q[kk], iM)) - s_old[kk];
            for (int k0 = 0; k0 < K; k0 += KT) {
                const int k = k0 + kt;
                ff vq = ff_make(0.0f), vs = vq;
                if (gb < BG && k < K) {
                    constexpr int U = 8;
                    const float* Rq = FR + (size_t)gb * st + (size_t)i * K4 + k;
                    const float* Rs = FR + (size_t)gb * st + oS + k;
                    for (int c = gb; c < G; c += U * BG, Rq += U * step, Rs += U * step) {
                        float lq[U], ls[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const size_t o = c + u * BG < G ? u * step : 0;  // a valid block for the tail
                            lq[u] = __ldcg(Rq + o);
                            ls[u] = __ldcg(Rs + o);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (c + u * BG >= G) break;
                            vq = ff_add(vq, lq[u]);
                            vs = ff_add(vs, ls[u]);
                        }
                    }
                }
                FRS_MARK(0);
                if (gb < BG) {
                    s_part[gb * KT + kt] = vq;
                    s_part[blockDim.x + gb * KT + kt] = vs;
                }
                __syncthreads();
                if (tid < KT && k0 + tid < K) {
                    ff A = s_part[tid], S = s_part[blockDim.x + tid];
                    for (int q = 1; q < BG; ++q) {
                        A = ff_add(A, s_part[q * KT + tid]);
                        S = ff_add(S, s_part[blockDim.x + q * KT + tid]);
                    }
                    const float mc = ff_f(ff_add(A, ff_make(-dyb * ff_f(S))));
                    const float z = rademacher((uint32_t)i, (uint32_t)(k0 + tid), (uint32_t)H.t, P.pid, P.seed_lo,
                                               P.seed_hi);
                    const float zc = z + mc * iM;
                    s_sq[kk * K + k0 + tid] = zc * zc;
                }
                __syncthreads();
                FRS_MARK(1);
            }
        }
        for (int kk = warp; kk < ns; kk += nwarps) {
            float a = 0.0f;
            for (int k = lane; k < K; k += 32) a += s_sq[kk * K + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) P.cstat[(size_t)(i0 + kk) * NCO + CO_DFULL] = a;
        }
    }
}

// Steps 4-5.  Reads the per-coordinate results (s_var receives Var y_i) and
// the chain totals, then lane 0 of warp 0 updates H and FS.{sw, eps, c1, c2s,
// now}.  Ends with __syncthreads(); all threads of the block call it.
__device__ __forceinline__ void ens_gather(const KParams& P, Hyper& H, float* s_var,
                                           FinShared& FS) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    float2 tot_pre = make_float2(0.0f, 0.0f);  // warp 0, lanes < NCS: the chain totals
    if (warp == 0 && lane < NCS) tot_pre = __ldcg(P.ctot + lane);
    {
        ff a_var = ff_make(0.0f), a_dv = ff_make(0.0f), a_b2 = ff_make(0.0f), a_df = ff_make(0.0f);
        float a_del = 0.0f, a_b2m = 0.0f;
        const bool full = P.dfull_K > 0 && P.mode == 1 && H.phase == 0;
        for (int i = tid; i < P.d; i += blockDim.x) {
            const float* co = P.cstat + (size_t)i * NCO;
            const float vy = __ldcg(co + CO_VARY), vx = __ldcg(co + CO_VARX);
            const float dv = __ldcg(co + CO_DV), del = __ldcg(co + CO_DEL);
            const float b2 = __ldcg(co + CO_B2);
            s_var[i] = vy;
            a_var = ff_add(a_var, vx);
            a_dv = ff_add(a_dv, dv);
            a_b2 = ff_add(a_b2, b2);
            if (full) a_df = ff_add(a_df, __ldcg(co + CO_DFULL));
            a_del = fmax_nan(a_del, del);
            a_b2m = fmax_nan(a_b2m, b2);
        }
        // one fused block reduction in a fixed order: warp butterflies, then warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const ff w0{__shfl_xor_sync(0xffffffffu, a_var.hi, o), __shfl_xor_sync(0xffffffffu, a_var.lo, o)};
            const ff w1{__shfl_xor_sync(0xffffffffu, a_dv.hi, o), __shfl_xor_sync(0xffffffffu, a_dv.lo, o)};
            const ff w3{__shfl_xor_sync(0xffffffffu, a_b2.hi, o), __shfl_xor_sync(0xffffffffu, a_b2.lo, o)};
            const ff w4{__shfl_xor_sync(0xffffffffu, a_df.hi, o), __shfl_xor_sync(0xffffffffu, a_df.lo, o)};
            a_var = ff_add(a_var, w0);
            a_dv = ff_add(a_dv, w1);
            a_b2 = ff_add(a_b2, w3);
            a_df = ff_add(a_df, w4);
            a_del = fmax_nan(a_del, __shfl_xor_sync(0xffffffffu, a_del, o));
            a_b2m = fmax_nan(a_b2m, __shfl_xor_sync(0xffffffffu, a_b2m, o));
        }
        if (lane == 0) {
            FS.wsum[0][warp] = a_var;
            FS.wsum[1][warp] = a_dv;
            FS.wsum[2][warp] = a_b2;
            FS.wsum[3][warp] = a_df;
            FS.wmax[0][warp] = a_del;
            FS.wmax[1][warp] = a_b2m;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // the per-warp partials combined by a butterfly over warp 0's lanes
        ff v0 = ff_make(0.0f), v1 = v0, v3 = v0, v5 = v0;
        float v2 = 0.0f, v4 = 0.0f;
        if (lane < nwarps) {
            v0 = FS.wsum[0][lane];
            v1 = FS.wsum[1][lane];
            v3 = FS.wsum[2][lane];
            v5 = FS.wsum[3][lane];
            v2 = FS.wmax[0][lane];
            v4 = FS.wmax[1][lane];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const ff w0{__shfl_xor_sync(0xffffffffu, v0.hi, o), __shfl_xor_sync(0xffffffffu, v0.lo, o)};
            const ff w1{__shfl_xor_sync(0xffffffffu, v1.hi, o), __shfl_xor_sync(0xffffffffu, v1.lo, o)};
            const ff w3{__shfl_xor_sync(0xffffffffu, v3.hi, o), __shfl_xor_sync(0xffffffffu, v3.lo, o)};
            const ff w5{__shfl_xor_sync(0xffffffffu, v5.hi, o), __shfl_xor_sync(0xffffffffu, v5.lo, o)};
            v0 = ff_add(v0, w0);
            v1 = ff_add(v1, w1);
            v3 = ff_add(v3, w3);
            v5 = ff_add(v5, w5);
            v2 = fmax_nan(v2, __shfl_xor_sync(0xffffffffu, v2, o));
            v4 = fmax_nan(v4, __shfl_xor_sync(0xffffffffu, v4, o));
        }
        ff tot[NCS];
#pragma unroll
        for (int k = 0; k < NCS; ++k)
            tot[k] = ff{__shfl_sync(0xffffffffu, tot_pre.x, k), __shfl_sync(0xffffffffu, tot_pre.y, k)};
        if (lane == 0) {
            Hyper h = H;  // work on a register copy
            const float d = (float)P.d;
            const float sum_var = ff_f(v0);
            int sw_flag = 0;
            if (P.mode == 0) {
                h.eps = P.fixed_eps > 0.0f ? P.fixed_eps : P.eps0;
                h.L = P.alpha * sqrtf(sum_var);
                h.t0_ns = global_ns();
            } else if (h.phase == 0) {
                // Sec. 3.1: EEVPD, D~, desired EEVPD, new step size; Eq. "L"
                const float nfin = ff_f(tot[CS_NFIN]), nbad = ff_f(tot[CS_NBAD]);
                float eevpd = NAN;
                if (nfin > 0.0f) {
                    const ff mean = ff_divf(tot[CS_DSUM], nfin);
                    const ff sq2 = ff_divf(tot[CS_DSQ], nfin);
                    eevpd = ff_f(P.eevpd_centered ? ff_add(sq2, ff_neg(ff_mul(mean, mean))) : sq2) / d;
                }
                // App. B: the diagonal proxy, or the full-rank one (Hutchinson over K vectors)
                const float D = P.dfull_K > 0 ? ff_f(v5) / (d * (float)P.dfull_K) : ff_f(v1) / d;
                const float cd = P.C * D, rt = sqrtf(cd);
                const float wanted = 4.0f * cd * rt / ((1.0f + rt) * (1.0f + rt));
                h.eps_used = h.eps;
                if (P.fixed_eps > 0.0f)
                    h.eps = P.fixed_eps;
                else if (nbad > 0.0f || !(eevpd > 0.0f) || !isfinite(eevpd) || !isfinite(wanted))
                    h.eps = 0.5f * h.eps;
                else
                    h.eps = h.eps * powf(wanted / eevpd, 1.0f / 6.0f);
                h.L = P.alpha * sqrtf(sum_var);
                h.t += 1;
                h.grads += 1;
                h.win_n += 1;
                h.eevpd = eevpd;
                h.eevpd_wanted = wanted;
                h.dtilde = D;
                h.max_delta = (h.win_n >= P.T) ? v2 : NAN;
                h.acc = NAN;
                h.nonfinite_last = (int)nbad;
                h.nonfinite_total += (int)nbad;
                bool sw = (h.win_n >= P.T) && (v2 < P.switch_tol);
                if (P.force_switch_at > 0) sw = h.t >= P.force_switch_at;
                if (sw && P.adjusted && h.t < P.n_total) {
                    sw_flag = 1;
                    if (sum_var > 0.0f) h.eps *= sqrtf(d / sum_var);
                    h.integ = (P.d > P.mn4_min_dim) ? INTEG_MN4 : INTEG_MN2;
                    h.a_target = (h.integ == INTEG_MN4) ? P.a_target_mn4 : P.a_target_mn2;
                    h.L = P.adj_L_factor * P.N * h.eps;
                    h.lo = 0.0f;
                    h.hi = 0.0f;
                    h.adapting = 1;
                    h.p = 0;
                    h.phase = 1;
                    h.t_switch = h.t;
                    if (h.t + P.N > P.n_total) h.done = 1;
                } else if (h.t >= P.n_total) {
                    h.done = 1;
                }
            } else {
                // Sec. 5.1: mean acceptance, bisection until |a - a*| <= tol
                const float a = ff_f(tot[CS_ASUM]) / (float)ens_chains(P);
                const float nbad = ff_f(tot[CS_NBAD]);
                h.eps_used = h.eps;
                h.adapting = h.adapting && (fabsf(a - h.a_target) > P.acc_tol);
                if (h.adapting) {
                    if (a > h.a_target) {
                        h.lo = h.eps;
                        h.eps = (h.hi > 0.0f) ? 0.5f * (h.lo + h.hi) : 2.0f * h.eps;
                    } else {
                        h.hi = h.eps;
                        h.eps = (h.lo > 0.0f) ? 0.5f * (h.lo + h.hi) : 0.5f * h.eps;
                    }
                }
                h.L = P.adj_L_factor * P.N * h.eps;
                h.acc = a;
                h.eevpd = h.eevpd_wanted = h.dtilde = h.max_delta = NAN;
                h.t += P.N;
                h.p += 1;
                h.grads += (long long)P.N * (h.integ == INTEG_MN4 ? 5 : 2);
                h.nonfinite_last = (int)nbad;
                h.nonfinite_total += (int)nbad;
                if (h.t + P.N > P.n_total) h.done = 1;
            }
            if (P.mode == 1) h.iters += 1;
            h.sum_var = sum_var;
            const uint64_t now = global_ns();
            if (P.Ex2) {
                h.b2_avg = ff_f(v3) / d;
                h.b2_max = v4;
                const float b2 = P.stop_b2_max ? h.b2_max : h.b2_avg;
                if (h.b2_first_t < 0 && b2 < 0.01f) {
                    h.b2_first_t = h.t;
                    h.b2_first_grads = h.grads;
                    h.b2_first_ns = (double)(now - h.t0_ns);
                }
                if (P.stop_b2 > 0.0f && b2 < P.stop_b2) h.done = 1;
            } else {
                h.b2_avg = h.b2_max = NAN;
            }
            set_step_scalars(h, P.d, FS.eps, FS.c1, FS.c2s);
            H = h;
            FS.sw = sw_flag;
            FS.now = now;
        }
    }
    __syncthreads();
}

// the trace row of the iteration just finalised (one thread)
__device__ __forceinline__ void ens_trace_row(const KParams& P, const Hyper& H,
                                              unsigned long long now) {
    if (H.iters >= P.trace_cap) return;
    laps_trace_row r;
    r.phase = H.phase;
    r.t = H.t;
    r.eps = H.eps;
    r.L = H.L;
    r.eps_used = P.mode == 0 ? NAN : H.eps_used;
    r.eevpd = P.mode == 0 ? NAN : H.eevpd;
    r.eevpd_wanted = P.mode == 0 ? NAN : H.eevpd_wanted;
    r.dtilde = P.mode == 0 ? NAN : H.dtilde;
    r.max_delta = P.mode == 0 ? NAN : H.max_delta;
    r.acc = P.mode == 0 ? NAN : H.acc;
    r.b2_max = H.b2_max;
    r.b2_avg = H.b2_avg;
    r.sum_var = H.sum_var;
    r.nonfinite = P.mode == 0 ? 0 : H.nonfinite_last;
    r.adapting = H.adapting;
    r.grads = H.grads;
    r.time_ns = (double)(now - H.t0_ns);
    P.trace[H.iters] = r;
}

}  // namespace laps
