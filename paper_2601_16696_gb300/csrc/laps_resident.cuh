// laps_resident.cuh -- persistent, register-resident LAPS kernel (sm_103a).
//
// One cooperative launch runs many iterations of Algorithm 1.  Each chain is
// owned by a group of LPC lanes; lane `gl` of the group holds the coordinate
// blocks j = gl + LPC*k (k < CPL/4) of the chain's position y, velocity u and
// gradient g in registers for the whole launch.  An iteration is
//   1. the chain update: an unadjusted step O_{eps/2} Phi_eps O_{eps/2} with
//      leapfrog (App. E, Eq. "discrete update"), or a MAMS proposal of N such
//      steps with MN2/MN4 and the accept/reject test (App. F);
//   2. per-block sums of y, y^2, g, y g over the block's chains and of the
//      per-chain energy error / acceptance (compensated FP32), added into
//      global 128-bit fixed-point accumulators with integer atomics (exact,
//      so the totals do not depend on the order of the blocks);
//   3. one grid barrier;
//   4. every block reads the totals (Eq. ECA) and computes, identically, the
//      per-coordinate Var, V_ii (App. B), the window statistic
//      delta[x_i^2] (Eq. "relative fluctuations"), b^2 (Eq. "bias") and the
//      finalise (Sec. 3.1 controller, Eq. "L", the switch of Sec. 4, the
//      bisection of Sec. 5.1), so all blocks hold bit-identical
//      hyperparameters without a broadcast or a second barrier.
#pragma once
#include <cmath>

#include "laps_device.cuh"
#include "laps_params.h"

namespace laps {

constexpr int kMaxThreads = 512;

struct Coefs {  // integrator tables (Table "integrators"), copied to shared memory
    float b[3][8];
    float a[3][8];
    int K[3];
};

// ---------------------------------------------------------------- target
// log p at x = sigma o y and the gradient in y (sigma o grad_x).  Returns the
// group-wide log p as a compensated float-float.
template <int KIND, int LPC, int CPL>
__device__ __forceinline__ ff eval_target(const KParams& P, int gl, int lane,
                                          const float (&y)[CPL], float (&g)[CPL],
                                          const float (&pr)[CPL], const float (&sg)[CPL]) {
    if constexpr (KIND == TGT_GAUSS) {
        float part = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const float xt = sg[q] * y[q];
            const float gx = -pr[q] * xt;
            g[q] = sg[q] * gx;
            part = fmaf(0.5f * gx, xt, part);  // -1/2 prec x^2
        }
        return group_sum_ff<LPC>(ff_make(part));
    } else if constexpr (KIND == TGT_BANANA) {
        ff part = ff_make(0.0f);
#pragma unroll
        for (int q = 0; q < CPL; q += 2) {
            const float a = sg[q] * y[q], b = sg[q + 1] * y[q + 1];
            const float r = fmaf(-a, a, b);
            const float ris = r * P.inv_s2;
            part = ff_add(part, fmaf(-0.5f * a, a, -0.5f * r * ris));
            g[q] = sg[q] * fmaf(2.0f * a, ris, -a);
            g[q + 1] = sg[q + 1] * (-ris);
        }
        return group_sum_ff<LPC>(part);
    } else {  // TGT_FUNNEL: coordinate 0 is v (lane gl == 0, slot q == 0)
        float xt[CPL];
        float ss = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            xt[q] = sg[q] * y[q];
            if (!(gl == 0 && q == 0)) ss = fmaf(xt[q], xt[q], ss);
        }
        ss = group_sum<LPC>(ss);
        const float v = __shfl_sync(0xffffffffu, xt[0], lane & ~(LPC - 1));
        const float ev = expf(-v);
        const float n = (float)(P.d - 1);
        ff lp = ff_make(-0.5f * v * v * P.inv_sv2);
        lp = ff_add(lp, -0.5f * n * v);
        lp = ff_add(lp, -0.5f * ev * ss);
#pragma unroll
        for (int q = 0; q < CPL; ++q) g[q] = sg[q] * (-xt[q] * ev);
        if (gl == 0) g[0] = sg[0] * (fmaf(-v, P.inv_sv2, -0.5f * n) + 0.5f * ev * ss);
        return lp;
    }
}

// A map with the target: y <- y + ae u (App. E, "Position update"), the
// gradient at the new point, and the change log p(x') - log p(x) written in
// difference form (products of x' - x and x' + x), so that the energy error
// keeps its accuracy when |log p| is large and the change is small.
template <int KIND, int LPC, int CPL>
__device__ __forceinline__ ff a_step(const KParams& P, int gl, int lane, float ae,
                                     float (&y)[CPL], const float (&u)[CPL], float (&g)[CPL],
                                     const float (&pr)[CPL], const float (&sg)[CPL]) {
    if constexpr (KIND == TGT_GAUSS) {
        float part = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const float xo = sg[q] * y[q];
            const float yn = fmaf(ae, u[q], y[q]);
            const float xn = sg[q] * yn;
            part = fmaf(-0.5f * pr[q] * (xn - xo), xo + xn, part);
            y[q] = yn;
            g[q] = sg[q] * (-pr[q] * xn);
        }
        return group_sum_ff<LPC>(ff_make(part));
    } else if constexpr (KIND == TGT_BANANA) {
        ff part = ff_make(0.0f);
#pragma unroll
        for (int q = 0; q < CPL; q += 2) {
            const float ao = sg[q] * y[q], bo = sg[q + 1] * y[q + 1];
            const float ya = fmaf(ae, u[q], y[q]), yb = fmaf(ae, u[q + 1], y[q + 1]);
            const float an = sg[q] * ya, bn = sg[q + 1] * yb;
            const float da = an - ao, db = bn - bo, sa = ao + an;
            const float ro = fmaf(-ao, ao, bo), rn = fmaf(-an, an, bn);
            const float dr = fmaf(-da, sa, db);
            part = ff_add(part, -0.5f * da * sa);
            part = ff_add(part, -0.5f * P.inv_s2 * dr * (ro + rn));
            y[q] = ya;
            y[q + 1] = yb;
            const float ris = rn * P.inv_s2;
            g[q] = sg[q] * fmaf(2.0f * an, ris, -an);
            g[q + 1] = sg[q + 1] * (-ris);
        }
        return group_sum_ff<LPC>(part);
    } else {  // TGT_FUNNEL
        float xn[CPL];
        float so = 0.0f, ds = 0.0f;
        float vo = 0.0f, vn = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const float xo = sg[q] * y[q];
            const float yn = fmaf(ae, u[q], y[q]);
            xn[q] = sg[q] * yn;
            y[q] = yn;
            if (gl == 0 && q == 0) {
                vo = xo;
                vn = xn[q];
            } else {
                so = fmaf(xo, xo, so);
                ds = fmaf(xn[q] - xo, xo + xn[q], ds);
            }
        }
        so = group_sum<LPC>(so);
        ds = group_sum<LPC>(ds);
        const int src = lane & ~(LPC - 1);
        vo = __shfl_sync(0xffffffffu, vo, src);
        vn = __shfl_sync(0xffffffffu, vn, src);
        const float dv = vn - vo;
        const float evo = expf(-vo), evn = expf(-vn);
        const float sn = so + ds;
        const float n = (float)(P.d - 1);
        // -(v'^2 - v^2)/(2 sv^2) - (n/2)(v' - v) - 1/2 (e^-v' S' - e^-v S)
        ff lp = ff_make(-0.5f * P.inv_sv2 * dv * (vo + vn));
        lp = ff_add(lp, -0.5f * n * dv);
        lp = ff_add(lp, -0.5f * evn * ds);
        lp = ff_add(lp, -0.5f * so * evo * expm1f(-dv));
#pragma unroll
        for (int q = 0; q < CPL; ++q) g[q] = sg[q] * (-xn[q] * evn);
        if (gl == 0) g[0] = sg[0] * (fmaf(-vn, P.inv_sv2, -0.5f * n) + 0.5f * evn * sn);
        return lp;
    }
}

// ---------------------------------------------------------------- O, B, A maps
// App. E, Eq. "O update": u <- (c1 u + c2 Z) / |.|, Z ~ N(0, I/d) per coordinate
// (std 1/sqrt(d)); c2s = c2 / sqrt(d).
template <int LPC, int CPL>
__device__ __forceinline__ void o_update(const KParams& P, int gl, bool active, uint32_t m,
                                         uint32_t t, uint32_t tag, float c1, float c2s,
                                         float (&u)[CPL]) {
    float n2 = 0.0f;
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = gl + LPC * k;
        float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (active && j < P.nblk) normals4(j, m, t, tag | (P.pid << 8), P.seed_lo, P.seed_hi, z);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = (4 * j + c < P.d) ? fmaf(c1, u[4 * k + c], c2s * z[c]) : 0.0f;
            u[4 * k + c] = v;
            n2 = fmaf(v, v, n2);
        }
    }
    n2 = group_sum<LPC>(n2);
    const float inv = n2 > 0.0f ? 1.0f / sqrtf(n2) : 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) u[q] *= inv;
}

// App. E, Eq. "B MCHMC" in the overflow-free form with zeta = e^-delta:
// u' = [2 zeta u + (1-zeta)((1+zeta) + (e.u)(1-zeta)) e] / [(1+zeta^2) + (e.u)(1-zeta^2)],
// kinetic change (d-1)[delta + log(den / 2)], den/2 - 1 = -(1-zeta)(1+zeta)(1-e.u)/2.
template <int LPC, int CPL>
__device__ __forceinline__ void b_update(float beps, float inv_dm1, float dm1,
                                         const float (&g)[CPL], float (&u)[CPL], ff& dl) {
    float gg = 0.0f, gu = 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        gg = fmaf(g[q], g[q], gg);
        gu = fmaf(g[q], u[q], gu);
    }
    gg = group_sum<LPC>(gg);
    gu = group_sum<LPC>(gu);
    if (gg > 0.0f) {
        const float gn = sqrtf(gg);
        const float eu = gu / gn;
        const float delta = beps * gn * inv_dm1;
        const float zeta = expf(-delta);
        const float om = -expm1f(-delta);  // 1 - zeta
        const float opz = 1.0f + zeta;
        const float den = fmaf(eu, om * opz, fmaf(zeta, zeta, 1.0f));
        const float inv = 1.0f / den;
        const float cu = 2.0f * zeta * inv;
        const float ce = om * fmaf(eu, om, opz) * inv / gn;
#pragma unroll
        for (int q = 0; q < CPL; ++q) u[q] = fmaf(cu, u[q], ce * g[q]);
        const float kin = dm1 * (delta + log1pf(-0.5f * om * opz * (1.0f - eu)));
        dl = ff_add(dl, kin);
    }
}

// Eq. "integrator": B_{b1 eps} A_{a1 eps} ... B_{bK eps}; each A adds
// -log p(x') + log p(x) to the energy error.  g and lp are kept consistent
// with y on exit (first-same-as-last gradient reuse).
template <int KIND, int LPC, int CPL>
__device__ __forceinline__ void phi_step(const KParams& P, const Coefs& cf, int integ, float eps,
                                         int gl, int lane, float (&y)[CPL], float (&u)[CPL],
                                         float (&g)[CPL], ff& lp, ff& dl, const float (&pr)[CPL],
                                         const float (&sg)[CPL]) {
    const float dm1 = (float)(P.d - 1), inv_dm1 = 1.0f / (float)(P.d - 1);
    const int K = cf.K[integ];
    for (int k = 0; k < K; ++k) {
        b_update<LPC, CPL>(cf.b[integ][k] * eps, inv_dm1, dm1, g, u, dl);
        if (k < K - 1) {
            const float ae = cf.a[integ][k] * eps;
            const ff dlp = a_step<KIND, LPC, CPL>(P, gl, lane, ae, y, u, g, pr, sg);
            dl = ff_add(dl, ff_neg(dlp));  // -log p(x') + log p(x)
            lp = ff_add(lp, dlp);
        }
    }
}

__device__ __forceinline__ bool finite_f(float v) { return isfinite(v); }

// FP32 scalars of the next iteration: eps, and the O-map constants for a half
// step, c1 = exp(-(eps/2)/L), c2 = sqrt(1 - c1^2) = sqrt(-expm1(-eps/L)), the
// latter scaled by 1/sqrt(d).
__device__ __forceinline__ void set_step_scalars(const Hyper& H, int d, float& eps, float& c1,
                                                 float& c2s) {
    eps = H.eps;
    c1 = expf(-0.5f * H.eps / H.L);
    c2s = sqrtf(-expm1f(-H.eps / H.L)) / sqrtf((float)d);
}

// ---------------------------------------------------------------- float-float helpers
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
    const float s = p + e;
    return ff{s, e - (s - p)};
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) { return ff_mul(a, ff{b, 0.0f}); }
__device__ __forceinline__ ff ff_divf(ff a, float b) {
    const float q1 = a.hi / b;
    const ff r = ff_add(a, ff_neg(ff_mulf(ff{q1, 0.0f}, b)));
    const float q2 = r.hi / b;
    const float s = q1 + q2;
    return ff{s, q2 - (s - q1)};
}
__device__ __forceinline__ float ff_f(ff a) { return a.hi + a.lo; }

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

// ---------------------------------------------------------------- the kernel
template <int KIND, int LPC, int CPL>
__global__ void __launch_bounds__(kMaxThreads) laps_resident_kernel(const KParams P,
                                                                   const Coefs* __restrict__ coefs) {
    constexpr int NB = CPL / 4;
    constexpr int GPW = 32 / LPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Hyper H;
    __shared__ Coefs CF;
    __shared__ ff s_wsum[3][kMaxThreads / 32];    // per-warp sums: Var, (1 - V)^2, b^2
    __shared__ float s_wmax[2][kMaxThreads / 32];  // per-warp maxima: delta, b^2
    __shared__ ff s_tot[NCS];
    __shared__ ff s_sl[NSL];
    __shared__ int s_switch, s_bad;
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
    const size_t acc_set = (size_t)P.nacc * 4 * FX_STRIDE;  // u64 words per accumulator set

    // dynamic shared memory: per-warp column sums, per-chain scalars,
    // per-coordinate variance (for the switch), window sums
    float* sq = reinterpret_cast<float*>(smem_raw);                        // [qpp][nwarps][dp]
    float* s_cs = sq + (size_t)P.qpp * nwarps * dp;                         // [slots][NCSF]
    float* s_var = s_cs + (size_t)slots * NCSF;                             // [dp]
    float4* s_win = reinterpret_cast<float4*>(s_var + dp);                  // [dp] (s1, s2 as ff)

    if (tid == 0) {
        H = *P.hyper;
        set_step_scalars(H, P.d, s_eps, s_c1, s_c2s);
        s_bad = 0;
    }
    for (int i = tid; i < (int)(sizeof(Coefs) / 4); i += blockDim.x)
        reinterpret_cast<int*>(&CF)[i] = reinterpret_cast<const int*>(coefs)[i];
    for (int i = tid; i < dp; i += blockDim.x) {
        s_win[i] = P.win_sums[i];
        s_var[i] = 0.0f;
    }
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
        // ------------------------------------------------ 2. block sums -> fixed-point totals
        unsigned long long* acc = P.acc + (size_t)(it % 3) * acc_set;
        {   // clear this block's share of the set the next iteration adds into
            unsigned long long* nxt = P.acc + (size_t)((it + 1) % 3) * acc_set;
            const size_t per = (acc_set + G - 1) / G;
            const size_t b0 = (size_t)blockIdx.x * per, b1 = min(acc_set, b0 + per);
            for (size_t k = b0 + tid; k < b1; k += blockDim.x) nxt[k] = 0ull;
        }
        const int nq = (H.phase == 1 && P.mode == 1) ? 2 : NQ;  // g sums unused after the switch
        int fx_bad = 0;
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
                fx_atomic_add(acc + ((size_t)qd * dp + i) * (4 * FX_STRIDE), s, fx_bad);
            }
            __syncthreads();
        }
        if (gl == 0) {
            float* cs = s_cs + (size_t)slot * NCSF;
            cs[0] = c_d.hi; cs[1] = c_d.lo; cs[2] = c_d2; cs[3] = c_fin; cs[4] = c_bad; cs[5] = c_a;
        }
        __syncthreads();
        if (tid < NCS) {
            ff s = ff_make(0.0f);
            for (int sl = 0; sl < slots; ++sl) {
                const float* cs = s_cs + (size_t)sl * NCSF;
                if (tid == CS_DSUM) s = ff_add(s, ff{cs[0], cs[1]});
                else s = ff_add(s, cs[tid + 1]);
            }
            fx_atomic_add(acc + ((size_t)NQ * dp + tid) * (4 * FX_STRIDE), s, fx_bad);
        }
        if (fx_bad) atomicOr(&s_bad, 1);
        LAPS_PHASE_MARK(2);
        // ------------------------------------------------ 3. the one grid barrier
        if (!grid_sync_count(P.bar_count, P.status, (unsigned)(it + 1) * (unsigned)(G + P.bar_extra),
                             P.timeout_ns))
            return;
        LAPS_PHASE_MARK(3);
        // ------------------------------------------------ 4. statistics (every block)
        const bool push = (P.mode == 1 && H.phase == 0);
        const bool have_g = nq == NQ;
        const float iM = 1.0f / (float)P.M;
        const int win_n = H.win_n;
        const int slot_new = win_n % (P.T + 1), slot_old = (win_n + 1) % (P.T + 1);
        ff a_var = ff_make(0.0f), a_dv = ff_make(0.0f), a_b2 = ff_make(0.0f);
        float a_del = 0.0f, a_b2m = 0.0f;
        for (int i = tid; i < P.d; i += blockDim.x) {
            const ff sy = fx_read(acc + ((size_t)0 * dp + i) * (4 * FX_STRIDE));
            const ff syy = fx_read(acc + ((size_t)1 * dp + i) * (4 * FX_STRIDE));
            const ff mean = ff_mulf(sy, iM), ey2 = ff_mulf(syy, iM);
            const float var_y = ff_f(ff_add(ey2, ff_neg(ff_mul(mean, mean))));
            const float sgi = P.sigma[i];
            const float s2i = sgi * sgi;
            const ff ex2 = ff_mulf(ey2, s2i);
            a_var = ff_add(a_var, s2i * var_y);
            s_var[i] = var_y;
            if (have_g) {
                const ff sg_ = fx_read(acc + ((size_t)2 * dp + i) * (4 * FX_STRIDE));
                const ff syg = fx_read(acc + ((size_t)3 * dp + i) * (4 * FX_STRIDE));
                // V_ii = -(E[y g] - E[y] E[g])  (App. B, Eq. ECA)
                const float V = -ff_f(ff_add(ff_mulf(syg, iM), ff_neg(ff_mul(mean, ff_mulf(sg_, iM)))));
                a_dv = ff_add(a_dv, (1.0f - V) * (1.0f - V));
            }
            if (push) {
                // moving window of E[x_i^2]: running sums over the last T values
                float4 w = s_win[i];
                ff s1{w.x, w.y}, s2{w.z, w.w};
                if (win_n >= P.T) {
                    const float2 o = __ldcg(reinterpret_cast<const float2*>(P.ring) + (size_t)slot_old * dp + i);
                    const ff old{o.x, o.y};
                    s1 = ff_add(s1, ff_neg(old));
                    s2 = ff_add(s2, ff_neg(ff_mul(old, old)));
                }
                s1 = ff_add(s1, ex2);
                s2 = ff_add(s2, ff_mul(ex2, ex2));
                s_win[i] = make_float4(s1.hi, s1.lo, s2.hi, s2.lo);
                if (blockIdx.x == 0) P.ring[(size_t)slot_new * dp + i] = make_float2(ex2.hi, ex2.lo);
                if (win_n + 1 >= P.T) {
                    const float Tf = (float)P.T;
                    const ff mu = ff_divf(s1, Tf);
                    const float vv = ff_f(ff_add(s2, ff_neg(ff_mul(s1, mu)))) / (Tf - 1.0f);
                    const float del = sqrtf(vv > 0.0f ? vv : 0.0f) / ff_f(mu);
                    a_del = (del > a_del || del != del) ? del : a_del;
                }
            }
            if (P.Ex2) {
                const float2 e = P.Ex2[i];
                const float dd = ff_f(ff_add(ex2, ff_neg(ff{e.x, e.y})));
                const float b2 = dd * dd * P.inv_varx2[i];
                a_b2 = ff_add(a_b2, b2);
                a_b2m = (b2 > a_b2m || b2 != b2) ? b2 : a_b2m;
            }
        }
        {   // one fused block reduction in a fixed order: warp butterflies, then warps in order
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const ff w0{__shfl_xor_sync(0xffffffffu, a_var.hi, o), __shfl_xor_sync(0xffffffffu, a_var.lo, o)};
                const ff w1{__shfl_xor_sync(0xffffffffu, a_dv.hi, o), __shfl_xor_sync(0xffffffffu, a_dv.lo, o)};
                const ff w3{__shfl_xor_sync(0xffffffffu, a_b2.hi, o), __shfl_xor_sync(0xffffffffu, a_b2.lo, o)};
                const float w2 = __shfl_xor_sync(0xffffffffu, a_del, o);
                const float w4 = __shfl_xor_sync(0xffffffffu, a_b2m, o);
                a_var = ff_add(a_var, w0);
                a_dv = ff_add(a_dv, w1);
                a_b2 = ff_add(a_b2, w3);
                a_del = (w2 > a_del || w2 != w2) ? w2 : a_del;
                a_b2m = (w4 > a_b2m || w4 != w4) ? w4 : a_b2m;
            }
            if (lane == 0) {
                s_wsum[0][warp] = a_var;
                s_wsum[1][warp] = a_dv;
                s_wsum[2][warp] = a_b2;
                s_wmax[0][warp] = a_del;
                s_wmax[1][warp] = a_b2m;
            }
        }
        if (tid < NCS) s_tot[tid] = fx_read(acc + ((size_t)NQ * dp + tid) * (4 * FX_STRIDE));
        __syncthreads();
        if (tid == 0) {
            ff v0 = ff_make(0.0f), v1 = v0, v3 = v0;
            float v2 = 0.0f, v4 = 0.0f;
            for (int w = 0; w < nwarps; ++w) {
                v0 = ff_add(v0, s_wsum[0][w]);
                v1 = ff_add(v1, s_wsum[1][w]);
                v3 = ff_add(v3, s_wsum[2][w]);
                v2 = (s_wmax[0][w] > v2 || s_wmax[0][w] != s_wmax[0][w]) ? s_wmax[0][w] : v2;
                v4 = (s_wmax[1][w] > v4 || s_wmax[1][w] != s_wmax[1][w]) ? s_wmax[1][w] : v4;
            }
            s_sl[SL_VAR] = v0; s_sl[SL_DV] = v1; s_sl[SL_B2SUM] = v3;
            s_sl[SL_MAXDEL] = ff_make(v2); s_sl[SL_B2MAX] = ff_make(v4);
        }
        LAPS_PHASE_MARK(4);
        // ------------------------------------------------ 5. finalise (identical in every block)
        if (tid == 0) {
            const float d = (float)P.d;
            const float sum_var = ff_f(s_sl[SL_VAR]);
            s_switch = 0;
            if (P.mode == 0) {
                H.eps = P.fixed_eps > 0.0f ? P.fixed_eps : P.eps0;
                H.L = P.alpha * sqrtf(sum_var);
                H.t0_ns = global_ns();
            } else if (H.phase == 0) {
                // Sec. 3.1: EEVPD, D~, desired EEVPD, new step size; Eq. "L"
                const float nfin = ff_f(s_tot[CS_NFIN]), nbad = ff_f(s_tot[CS_NBAD]);
                float eevpd = NAN;
                if (nfin > 0.0f) {
                    const ff mean = ff_divf(s_tot[CS_DSUM], nfin);
                    const ff sq2 = ff_divf(s_tot[CS_DSQ], nfin);
                    eevpd = ff_f(P.eevpd_centered ? ff_add(sq2, ff_neg(ff_mul(mean, mean))) : sq2) / d;
                }
                const float D = ff_f(s_sl[SL_DV]) / d;
                const float cd = P.C * D, rt = sqrtf(cd);
                const float wanted = 4.0f * cd * rt / ((1.0f + rt) * (1.0f + rt));
                H.eps_used = H.eps;
                if (P.fixed_eps > 0.0f)
                    H.eps = P.fixed_eps;
                else if (nbad > 0.0f || !(eevpd > 0.0f) || !isfinite(eevpd) || !isfinite(wanted))
                    H.eps = 0.5f * H.eps;
                else
                    H.eps = H.eps * powf(wanted / eevpd, 1.0f / 6.0f);
                H.L = P.alpha * sqrtf(sum_var);
                H.t += 1;
                H.grads += 1;
                H.win_n += 1;
                H.eevpd = eevpd;
                H.eevpd_wanted = wanted;
                H.dtilde = D;
                H.max_delta = (H.win_n >= P.T) ? s_sl[SL_MAXDEL].hi : NAN;
                H.acc = NAN;
                H.nonfinite_last = (int)nbad;
                H.nonfinite_total += (int)nbad;
                bool sw = (H.win_n >= P.T) && (s_sl[SL_MAXDEL].hi < P.switch_tol);
                if (P.force_switch_at > 0) sw = H.t >= P.force_switch_at;
                if (sw && P.adjusted && H.t < P.n_total) {
                    s_switch = 1;
                    if (sum_var > 0.0f) H.eps *= sqrtf(d / sum_var);
                    H.integ = (P.d > P.mn4_min_dim) ? INTEG_MN4 : INTEG_MN2;
                    H.a_target = (H.integ == INTEG_MN4) ? P.a_target_mn4 : P.a_target_mn2;
                    H.L = P.adj_L_factor * P.N * H.eps;
                    H.lo = 0.0f;
                    H.hi = 0.0f;
                    H.adapting = 1;
                    H.p = 0;
                    H.phase = 1;
                    H.t_switch = H.t;
                    if (H.t + P.N > P.n_total) H.done = 1;
                } else if (H.t >= P.n_total) {
                    H.done = 1;
                }
            } else {
                // Sec. 5.1: mean acceptance, bisection until |a - a*| <= tol
                const float a = ff_f(s_tot[CS_ASUM]) / (float)P.M;
                const float nbad = ff_f(s_tot[CS_NBAD]);
                H.eps_used = H.eps;
                H.adapting = H.adapting && (fabsf(a - H.a_target) > P.acc_tol);
                if (H.adapting) {
                    if (a > H.a_target) {
                        H.lo = H.eps;
                        H.eps = (H.hi > 0.0f) ? 0.5f * (H.lo + H.hi) : 2.0f * H.eps;
                    } else {
                        H.hi = H.eps;
                        H.eps = (H.lo > 0.0f) ? 0.5f * (H.lo + H.hi) : 0.5f * H.eps;
                    }
                }
                H.L = P.adj_L_factor * P.N * H.eps;
                H.acc = a;
                H.eevpd = H.eevpd_wanted = H.dtilde = H.max_delta = NAN;
                H.t += P.N;
                H.p += 1;
                H.grads += (long long)P.N * (H.integ == INTEG_MN4 ? 5 : 2);
                H.nonfinite_last = (int)nbad;
                H.nonfinite_total += (int)nbad;
                if (H.t + P.N > P.n_total) H.done = 1;
            }
            if (P.mode == 1) H.iters += 1;
            if (s_bad) atomicCAS(P.status, ST_OK, ST_OVERFLOW);
            H.sum_var = sum_var;
            const uint64_t now = global_ns();
            if (P.Ex2) {
                H.b2_avg = ff_f(s_sl[SL_B2SUM]) / d;
                H.b2_max = s_sl[SL_B2MAX].hi;
                const float b2 = P.stop_b2_max ? H.b2_max : H.b2_avg;
                if (H.b2_first_t < 0 && b2 < 0.01f) {
                    H.b2_first_t = H.t;
                    H.b2_first_grads = H.grads;
                    H.b2_first_ns = (double)(now - H.t0_ns);
                }
                if (P.stop_b2 > 0.0f && b2 < P.stop_b2) H.done = 1;
            } else {
                H.b2_avg = H.b2_max = NAN;
            }
            set_step_scalars(H, P.d, s_eps, s_c1, s_c2s);
            s_now = now;
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
        LAPS_PHASE_MARK(5);
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

    // ---- store the state and (block 0) the phase machine and window sums
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
    if (blockIdx.x == 0) {
        for (int i = tid; i < dp; i += blockDim.x) {
            P.win_sums[i] = s_win[i];
            P.var_y[i] = s_var[i];
        }
        if (tid == 0) *P.hyper = H;
    }
}

}  // namespace laps
