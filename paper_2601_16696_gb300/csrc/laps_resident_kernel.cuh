// laps_resident_kernel.cuh -- the persistent, register-resident LAPS kernel.
//
// One cooperative launch runs many iterations of Algorithm 1.  Each chain is
// owned by a group of LPC lanes; lane `gl` of the group holds the coordinate
// blocks j = gl + LPC*k (k < CPL/4) of the chain's position y, velocity u and
// gradient g in registers for the whole launch.  An iteration is
//   1. the chain update: an unadjusted step O_{eps/2} Phi_eps O_{eps/2} with
//      leapfrog (App. E, Eq. "discrete update"), or a MAMS proposal of N such
//      steps with MN2/MN4 and the accept/reject test (App. F);
//   2. per-block compensated (float-float) sums over the block's chains of y,
//      y^2, g, y g per coordinate and of the energy error / acceptance per
//      chain (Eq. ECA), stored as one column per block;
//   3. grid barrier; block b reduces, in block order, the columns of its slice
//      of coordinates and derives for them Var, V_ii (App. B), the window
//      statistic delta[x_i^2] (Eq. "relative fluctuations") and b^2 (Eq.
//      "bias"); the last block also reduces the per-chain sums;
//   4. grid barrier; every block reads the d per-coordinate results and runs
//      the same finalise (Sec. 3.1 controller, Eq. "L", the switch of Sec. 4,
//      the bisection of Sec. 5.1), so all blocks hold bit-identical
//      hyperparameters without a broadcast.
// Every sum has a fixed order, so runs are bit-reproducible.
#pragma once
#include "laps_resident.cuh"

namespace laps {

// ---------------------------------------------------------------- phase timing
// Built only with -DLAPS_PHASE_TIMING (a diagnostic build): block 0 adds the
// %globaltimer time spent between consecutive marks to P.phase_ns[k].
#ifdef LAPS_PHASE_TIMING
#define LAPS_PHASE_MARK(k)                                                              \
    do {                                                                                \
        __syncthreads();                                                                \
        if (blockIdx.x == 0 && threadIdx.x == 0 && P.phase_ns) {                        \
            const unsigned long long now_ = global_ns();                                \
            if ((k) > 0) P.phase_ns[(k) - 1] += now_ - phase_t_;                        \
            phase_t_ = now_;                                                            \
        }                                                                               \
    } while (0)
#else
#define LAPS_PHASE_MARK(k) \
    do {                   \
    } while (0)
#endif

__device__ __forceinline__ float fmax_nan(float a, float b) { return (b > a || b != b) ? b : a; }

// ---------------------------------------------------------------- the kernel
template <int KIND, int LPC, int CPL>
__global__ void __launch_bounds__(kMaxThreads) laps_resident_kernel(const KParams P,
                                                                   const Coefs* __restrict__ coefs) {
    constexpr int NB = CPL / 4;
    constexpr int GPW = 32 / LPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Hyper H;
    __shared__ Coefs CF;
    __shared__ ff s_wsum[3][kMaxThreads / 32];    // per-warp sums: Var x, (1 - V)^2, b^2
    __shared__ float s_wmax[2][kMaxThreads / 32];  // per-warp maxima: delta, b^2
    __shared__ int s_switch;
    __shared__ float s_eps, s_c1, s_c2s;  // step scalars of the next iteration
    __shared__ unsigned long long s_now;  // %globaltimer at the last finalise

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int gl = lane & (LPC - 1), grp = lane / LPC;
    const int slot = warp * GPW + grp, slots = nwarps * GPW;
    const int G = P.G;
    const int m = blockIdx.x * slots + slot;
    const bool active = m < P.M;
    const int dp = P.d_pad;
    const unsigned gmask = ((LPC == 32) ? 0xffffffffu : ((1u << LPC) - 1u)) << (grp * LPC);
    // this block's slice of coordinates (step 3); the last block also owns the chain sums
    const int i0 = (int)(((long long)blockIdx.x * P.d) / G);
    const int i1 = (int)(((long long)(blockIdx.x + 1) * P.d) / G);
    const bool chain_owner = blockIdx.x == G - 1;

    // dynamic shared memory
    float* sq = reinterpret_cast<float*>(smem_raw);                  // [qpp][nwarps][dp]
    float* s_cs = sq + (size_t)P.qpp * nwarps * dp;                   // [slots][NCSF]
    float* s_var = s_cs + (size_t)slots * NCSF;                       // [dp] Var y (switch)
    ff* s_q = reinterpret_cast<ff*>(s_var + dp);                      // [NQ][smax] + [NCS]

    if (tid == 0) {
        H = *P.hyper;
        set_step_scalars(H, P.d, s_eps, s_c1, s_c2s);
    }
    for (int i = tid; i < (int)(sizeof(Coefs) / 4); i += blockDim.x)
        reinterpret_cast<int*>(&CF)[i] = reinterpret_cast<const int*>(coefs)[i];
    __syncthreads();

    // ---- registers: state and per-coordinate constants
    float y[CPL], u[CPL], g[CPL], pr[CPL], sg[CPL];
    ff lp = ff_make(0.0f);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int j = gl + LPC * k;
        const bool ok = active && j < P.nblk;
        const size_t off = (size_t)m * dp + 4 * j;
        float4 a = make_float4(0, 0, 0, 0), b = a, c = a, s = make_float4(1, 1, 1, 1), p = a;
        if (ok && P.mode == 1) {
            a = *reinterpret_cast<const float4*>(P.y + off);
            b = *reinterpret_cast<const float4*>(P.u + off);
            c = *reinterpret_cast<const float4*>(P.g + off);
        }
        if (j < P.nblk) {
            s = *reinterpret_cast<const float4*>(P.sigma + 4 * j);
            if (KIND == TGT_GAUSS) p = *reinterpret_cast<const float4*>(P.prec + 4 * j);
        }
        y[4 * k] = a.x; y[4 * k + 1] = a.y; y[4 * k + 2] = a.z; y[4 * k + 3] = a.w;
        u[4 * k] = b.x; u[4 * k + 1] = b.y; u[4 * k + 2] = b.z; u[4 * k + 3] = b.w;
        g[4 * k] = c.x; g[4 * k + 1] = c.y; g[4 * k + 2] = c.z; g[4 * k + 3] = c.w;
        sg[4 * k] = s.x; sg[4 * k + 1] = s.y; sg[4 * k + 2] = s.z; sg[4 * k + 3] = s.w;
        pr[4 * k] = p.x; pr[4 * k + 1] = p.y; pr[4 * k + 2] = p.z; pr[4 * k + 3] = p.w;
    }
    if (P.mode == 1 && active) {
        const float2 l = P.logp_ff[m];
        lp = ff{l.x, l.y};
    }

    // ---- initialisation (Alg. 1 first lines, App. C "Initialization")
    if (P.mode == 0) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int j = gl + LPC * k;
            float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (active && j < P.nblk) {
                if (P.x0 == nullptr) normals4(j, m, 0u, TAG_X0 | (P.pid << 8), P.seed_lo, P.seed_hi, z);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = 4 * j + c;
                    if (i < P.d)
                        y[4 * k + c] = P.x0 ? P.x0[(size_t)m * P.d + i] : P.x0_scale * z[c];
                }
            }
        }
        lp = eval_target<KIND, LPC, CPL>(P, gl, lane, y, g, pr, sg);
        float n2 = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) n2 = fmaf(g[q], g[q], n2);
        n2 = group_sum<LPC>(n2);
        // a uniformly random direction, used where the gradient vanishes
        // (drawn by every group so that the shuffles stay warp-uniform)
#pragma unroll
        for (int q = 0; q < CPL; ++q) u[q] = 0.0f;
        o_update<LPC, CPL>(P, gl, active, m, 0xFFFFFFFFu, TAG_O1, 0.0f, 1.0f, u);
        if (n2 > 0.0f) {
            const float inv = 1.0f / sqrtf(n2);
#pragma unroll
            for (int q = 0; q < CPL; ++q) u[q] = g[q] * inv;
        }
        // a non-finite initial point would poison every ensemble statistic: report it
        bool bad = active && !isfinite(lp.hi);
#pragma unroll
        for (int q = 0; q < CPL; ++q) bad = bad || (active && !(finite_f(y[q]) && finite_f(g[q])));
        if (bad) atomicCAS(P.status, ST_OK, ST_NONFINITE);
    }

    const int n_iter = (P.mode == 0) ? 1 : P.n_iters;
    unsigned n_bar = 0;  // grid barriers passed in this launch
#ifdef LAPS_PHASE_TIMING
    unsigned long long phase_t_ = 0;
#endif
    for (int it = 0; it < n_iter; ++it) {
        if (P.mode == 1 && H.done) break;
        LAPS_PHASE_MARK(0);
        // ------------------------------------------------ 1. chain update
        ff c_d = ff_make(0.0f);
        float c_d2 = 0.0f, c_fin = 0.0f, c_bad = 0.0f, c_a = 0.0f;
        if (P.mode == 1) {
            const float eps = s_eps, c1 = s_c1, c2s = s_c2s;
            float y0[CPL], g0[CPL], u0[CPL];
            const ff lp0 = lp;
#pragma unroll
            for (int q = 0; q < CPL; ++q) { y0[q] = y[q]; g0[q] = g[q]; u0[q] = u[q]; }
            ff dl = ff_make(0.0f);
            if (H.phase == 0) {
                const uint32_t t = (uint32_t)H.t;
                o_update<LPC, CPL>(P, gl, active, m, t, TAG_O1, c1, c2s, u);
                phi_step<KIND, LPC, CPL>(P, CF, INTEG_LF, eps, gl, lane, y, u, g, lp, dl, pr, sg);
                o_update<LPC, CPL>(P, gl, active, m, t, TAG_O2, c1, c2s, u);
            } else {
                // App. F step 2: u uniform on the sphere
                const uint32_t pidx = (uint32_t)H.p;
                float n2 = 0.0f;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const int j = gl + LPC * k;
                    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (active && j < P.nblk)
                        normals4(j, m, pidx, TAG_REFRESH | (P.pid << 8), P.seed_lo, P.seed_hi, z);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float v = (4 * j + c < P.d) ? z[c] : 0.0f;
                        u[4 * k + c] = v;
                        n2 = fmaf(v, v, n2);
                    }
                }
                n2 = group_sum<LPC>(n2);
                const float inv = n2 > 0.0f ? 1.0f / sqrtf(n2) : 0.0f;
#pragma unroll
                for (int q = 0; q < CPL; ++q) u[q] *= inv;
                // steps 3-4: N steps of phi with partial refreshes
                const uint32_t t0 = (uint32_t)H.t;
                for (int n = 0; n < P.N; ++n) {
                    o_update<LPC, CPL>(P, gl, active, m, t0 + n, TAG_O1, c1, c2s, u);
                    phi_step<KIND, LPC, CPL>(P, CF, H.integ, eps, gl, lane, y, u, g, lp, dl, pr, sg);
                    o_update<LPC, CPL>(P, gl, active, m, t0 + n, TAG_O2, c1, c2s, u);
                }
            }
            // non-finite check over the chain's group
            bool bad = !(isfinite(lp.hi) && isfinite(dl.hi));
#pragma unroll
            for (int q = 0; q < CPL; ++q)
                bad = bad || !(finite_f(y[q]) && finite_f(u[q]) && finite_f(g[q]));
            bad = (__ballot_sync(0xffffffffu, bad) & gmask) != 0u;
            bool keep = !bad;
            float a_m = 0.0f;
            if (H.phase == 1) {
                // step 5: accept with probability min(1, e^-Delta)
                const uint4 r = philox4x32_10(
                    make_uint4(0u, (uint32_t)m, (uint32_t)H.p, TAG_MH | (P.pid << 8)), P.seed_lo,
                    P.seed_hi);
                const ff s = ff_add(dl, logf(u01(r.x)));
                keep = !bad && (s.hi < 0.0f || (s.hi == 0.0f && s.lo < 0.0f));
                a_m = bad ? 0.0f : (dl.hi <= 0.0f ? 1.0f : expf(-(dl.hi + dl.lo)));
            }
            if (!keep) {
#pragma unroll
                for (int q = 0; q < CPL; ++q) { y[q] = y0[q]; g[q] = g0[q]; u[q] = u0[q]; }
                lp = lp0;
            }
            if (active) {
                if (H.phase == 0) {
                    if (bad) c_bad = 1.0f;
                    else { c_d = dl; c_d2 = ff_f(dl) * ff_f(dl); c_fin = 1.0f; }
                } else {
                    c_a = a_m;
                    c_bad = bad ? 1.0f : 0.0f;
                }
            }
        }
        LAPS_PHASE_MARK(1);
        // ------------------------------------------------ 2. block columns
        const int nq = (H.phase == 1 && P.mode == 1) ? 2 : NQ;  // g sums unused after the switch
        for (int q0 = 0; q0 < nq; q0 += P.qpp) {
            const int q1 = min(nq, q0 + P.qpp);
            for (int qd = q0; qd < q1; ++qd) {
#pragma unroll
                for (int k = 0; k < NB; ++k) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int q = 4 * k + c;
                        float v = qd == 0 ? y[q] : qd == 1 ? y[q] * y[q] : qd == 2 ? g[q] : y[q] * g[q];
                        v = active ? v : 0.0f;
                        v = across_groups<LPC>(v);
                        const int j = gl + LPC * k;
                        if (grp == 0 && j < P.nblk) sq[((size_t)(qd - q0) * nwarps + warp) * dp + 4 * j + c] = v;
                    }
                }
            }
            __syncthreads();
            for (int col = tid; col < (q1 - q0) * dp; col += blockDim.x) {
                const int qd = q0 + col / dp, i = col - (col / dp) * dp;
                if (i >= P.d) continue;
                ff s = ff_make(0.0f);
                const float* src = sq + (size_t)(qd - q0) * nwarps * dp + i;
                for (int w = 0; w < nwarps; ++w) s = ff_add(s, src[(size_t)w * dp]);
                P.part[((size_t)qd * dp + i) * G + blockIdx.x] = make_float2(s.hi, s.lo);
            }
            __syncthreads();
        }
        LAPS_PHASE_MARK(2);
        if (gl == 0) {
            float* cs = s_cs + (size_t)slot * NCSF;
            cs[0] = c_d.hi; cs[1] = c_d.lo; cs[2] = c_d2; cs[3] = c_fin; cs[4] = c_bad; cs[5] = c_a;
        }
        __syncthreads();
        // per-chain sums: warp k adds quantity k over the slots (lanes, then a butterfly)
        for (int k = warp; k < NCS; k += nwarps) {
            ff s = ff_make(0.0f);
            for (int sl = lane; sl < slots; sl += 32) {
                const float* cs = s_cs + (size_t)sl * NCSF;
                s = ff_add(s, k == CS_DSUM ? ff{cs[0], cs[1]} : ff_make(cs[k + 1]));
            }
            s = group_sum_ff<32>(s);
            if (lane == 0) P.part[((size_t)NQ * dp + k) * G + blockIdx.x] = make_float2(s.hi, s.lo);
        }
        LAPS_PHASE_MARK(3);
        // ------------------------------------------------ 3. barrier, then this block's slice
        n_bar += 1;
        if (!grid_sync_count(P.bar_count, P.status, n_bar * (unsigned)(G + P.bar_extra), P.timeout_ns))
            return;
        LAPS_PHASE_MARK(4);
        {
            const int ns = i1 - i0;
            const bool push = (P.mode == 1 && H.phase == 0);
            const int win_n = H.win_n;
            // the window values this thread will update, loaded before the reductions
            float4 w_pre = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float2 o_pre = make_float2(0.0f, 0.0f);
            if (push && tid < ns) {
                w_pre = P.win_sums[i0 + tid];
                if (win_n >= P.T) o_pre = P.ring[(size_t)((win_n - P.T) % (P.T + 1)) * dp + i0 + tid];
            }
            // column sums over the blocks, in block order: one warp per (quantity, coordinate)
            const int n_pairs = nq * ns + (chain_owner ? NCS : 0);
            for (int pidx = warp; pidx < n_pairs; pidx += nwarps) {
                size_t row;
                if (pidx < nq * ns) row = (size_t)(pidx / ns) * dp + i0 + (pidx % ns);
                else row = (size_t)NQ * dp + (pidx - nq * ns);
                const float2* src = P.part + row * G;
                ff s = ff_make(0.0f);
                for (int c = lane; c < G; c += 32) {
                    const float2 v = __ldcg(src + c);
                    s = ff_add(s, ff{v.x, v.y});
                }
                s = group_sum_ff<32>(s);
                if (lane == 0) {
                    if (pidx < nq * ns) s_q[(pidx / ns) * P.smax + (pidx % ns)] = s;
                    else s_q[NQ * P.smax + (pidx - nq * ns)] = s;
                }
            }
            __syncthreads();
            const float iM = 1.0f / (float)P.M;
            for (int k = tid; k < ns; k += blockDim.x) {
                const int i = i0 + k;
                const ff mean = ff_mulf(s_q[0 * P.smax + k], iM);
                const ff ey2 = ff_mulf(s_q[1 * P.smax + k], iM);
                const float var_y = ff_f(ff_add(ey2, ff_neg(ff_mul(mean, mean))));
                const float sgi = P.sigma[i];
                const float s2i = sgi * sgi;
                const ff ex2 = ff_mulf(ey2, s2i);
                float dv = 0.0f, del = 0.0f, b2 = 0.0f;
                if (nq == NQ) {
                    // V_ii = -(E[y g] - E[y] E[g])  (App. B, Eq. ECA)
                    const ff eg = ff_mulf(s_q[2 * P.smax + k], iM);
                    const ff eyg = ff_mulf(s_q[3 * P.smax + k], iM);
                    const float V = -ff_f(ff_add(eyg, ff_neg(ff_mul(mean, eg))));
                    dv = (1.0f - V) * (1.0f - V);
                }
                if (push) {
                    // moving window of E[x_i^2]: running sums over the last T values
                    const float4 w = k == tid ? w_pre : P.win_sums[i];
                    ff s1{w.x, w.y}, s2{w.z, w.w};
                    float2* ring_i = P.ring + i;
                    if (win_n >= P.T) {
                        const float2 o =
                            k == tid ? o_pre : ring_i[(size_t)((win_n - P.T) % (P.T + 1)) * dp];
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
                    const float2 e = P.Ex2[i];
                    const float dd = ff_f(ff_add(ex2, ff_neg(ff{e.x, e.y})));
                    b2 = dd * dd * P.inv_varx2[i];
                }
                float* co = P.cstat + (size_t)i * NCO;
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
        }
        LAPS_PHASE_MARK(5);
        // ------------------------------------------------ 4. barrier, then every block gathers
        n_bar += 1;
        if (!grid_sync_count(P.bar_count, P.status, n_bar * (unsigned)(G + P.bar_extra), P.timeout_ns))
            return;
        LAPS_PHASE_MARK(6);
        float2 tot_pre = make_float2(0.0f, 0.0f);  // warp 0, lanes < NCS: the chain totals
        if (warp == 0 && lane < NCS) tot_pre = __ldcg(P.ctot + lane);
        {
            ff a_var = ff_make(0.0f), a_dv = ff_make(0.0f), a_b2 = ff_make(0.0f);
            float a_del = 0.0f, a_b2m = 0.0f;
            for (int i = tid; i < P.d; i += blockDim.x) {
                const float* co = P.cstat + (size_t)i * NCO;
                const float vy = __ldcg(co + CO_VARY), vx = __ldcg(co + CO_VARX);
                const float dv = __ldcg(co + CO_DV), del = __ldcg(co + CO_DEL);
                const float b2 = __ldcg(co + CO_B2);
                s_var[i] = vy;
                a_var = ff_add(a_var, vx);
                a_dv = ff_add(a_dv, dv);
                a_b2 = ff_add(a_b2, b2);
                a_del = fmax_nan(a_del, del);
                a_b2m = fmax_nan(a_b2m, b2);
            }
            // one fused block reduction in a fixed order: warp butterflies, then warps in order
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const ff w0{__shfl_xor_sync(0xffffffffu, a_var.hi, o), __shfl_xor_sync(0xffffffffu, a_var.lo, o)};
                const ff w1{__shfl_xor_sync(0xffffffffu, a_dv.hi, o), __shfl_xor_sync(0xffffffffu, a_dv.lo, o)};
                const ff w3{__shfl_xor_sync(0xffffffffu, a_b2.hi, o), __shfl_xor_sync(0xffffffffu, a_b2.lo, o)};
                a_var = ff_add(a_var, w0);
                a_dv = ff_add(a_dv, w1);
                a_b2 = ff_add(a_b2, w3);
                a_del = fmax_nan(a_del, __shfl_xor_sync(0xffffffffu, a_del, o));
                a_b2m = fmax_nan(a_b2m, __shfl_xor_sync(0xffffffffu, a_b2m, o));
            }
            if (lane == 0) {
                s_wsum[0][warp] = a_var;
                s_wsum[1][warp] = a_dv;
                s_wsum[2][warp] = a_b2;
                s_wmax[0][warp] = a_del;
                s_wmax[1][warp] = a_b2m;
            }
        }
        __syncthreads();
        // ------------------------------------------------ 5. finalise (identical in every block)
        if (warp == 0) {
            // the per-warp partials combined by a butterfly over warp 0's lanes
            ff v0 = ff_make(0.0f), v1 = v0, v3 = v0;
            float v2 = 0.0f, v4 = 0.0f;
            if (lane < nwarps) {
                v0 = s_wsum[0][lane];
                v1 = s_wsum[1][lane];
                v3 = s_wsum[2][lane];
                v2 = s_wmax[0][lane];
                v4 = s_wmax[1][lane];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const ff w0{__shfl_xor_sync(0xffffffffu, v0.hi, o), __shfl_xor_sync(0xffffffffu, v0.lo, o)};
                const ff w1{__shfl_xor_sync(0xffffffffu, v1.hi, o), __shfl_xor_sync(0xffffffffu, v1.lo, o)};
                const ff w3{__shfl_xor_sync(0xffffffffu, v3.hi, o), __shfl_xor_sync(0xffffffffu, v3.lo, o)};
                v0 = ff_add(v0, w0);
                v1 = ff_add(v1, w1);
                v3 = ff_add(v3, w3);
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
                const float D = ff_f(v1) / d;
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
                const float a = ff_f(tot[CS_ASUM]) / (float)P.M;
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
            set_step_scalars(h, P.d, s_eps, s_c1, s_c2s);
            H = h;
            s_switch = sw_flag;
            s_now = now;
            }
        }
        __syncthreads();
        // the trace row (block 0), written by the last warp while the others go on
        if (blockIdx.x == 0 && tid == blockDim.x - 32 && H.iters < P.trace_cap) {
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
            r.time_ns = (double)(s_now - H.t0_ns);
            P.trace[H.iters] = r;
        }
        LAPS_PHASE_MARK(7);
        if (s_switch) {
            // Sec. 4: diagonal preconditioner y = x / Var[x]^{1/2}, fixed from now on
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int j = gl + LPC * k;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = 4 * j + c;
                    float s = 1.0f;
                    if (j < P.nblk && i < P.d) {
                        const float v = s_var[i];
                        s = v > 0.0f ? sqrtf(v) : 1.0f;
                    }
                    const int q = 4 * k + c;
                    sg[q] = s;
                    y[q] = y[q] / s;
                    g[q] = g[q] * s;
                }
            }
            if (blockIdx.x == 0)
                for (int i = tid; i < P.d; i += blockDim.x) {
                    const float v = s_var[i];
                    P.sigma[i] = v > 0.0f ? sqrtf(v) : 1.0f;
                }
        }
    }

    // ---- store the state and (block 0) the phase machine
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int j = gl + LPC * k;
        if (active && j < P.nblk) {
            const size_t off = (size_t)m * dp + 4 * j;
            *reinterpret_cast<float4*>(P.y + off) = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
            *reinterpret_cast<float4*>(P.u + off) = make_float4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
            *reinterpret_cast<float4*>(P.g + off) = make_float4(g[4 * k], g[4 * k + 1], g[4 * k + 2], g[4 * k + 3]);
        }
    }
    if (active && gl == 0) P.logp_ff[m] = make_float2(lp.hi, lp.lo);
    if (blockIdx.x == 0 && tid == 0) *P.hyper = H;
}

}  // namespace laps
