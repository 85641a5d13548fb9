// laps_resident.cuh -- persistent, register-resident LAPS kernel (sm_103a).
//
// One cooperative launch runs many iterations of Algorithm 1.  Each chain is
// owned by a group of LPC lanes; lane `gl` of the group holds the coordinate
// blocks j = gl + LPC*k (k < CPL/4) of the chain's position y, velocity u and
// gradient g in registers for the whole launch.  An iteration is
//   1. the chain update: an unadjusted step O_{eps/2} Phi_eps O_{eps/2} with
//      leapfrog (App. E, Eq. "discrete update"), or a MAMS proposal of N such
//      steps with MN2/MN4 and the accept/reject test (App. F);
//   2. per-block sums of y, y^2, g, y g over the block's chains (compensated
//      FP32) and of the per-chain energy error / acceptance, written as FP64
//      block partials (Eq. ECA);
//   3. grid barrier; block b reduces the partials of its slice of coordinates
//      over all blocks in FP64, in block order, and derives Var, V_ii (App. B),
//      the window statistic delta[x_i^2] (Eq. "relative fluctuations") and
//      b^2 (Eq. "bias") for those coordinates;
//   4. grid barrier; every block reduces the slice scalars in the same order
//      and runs the same FP64 finalise (Sec. 3.1 controller, Eq. "L", the
//      switch of Sec. 4, the bisection of Sec. 5.1), so all blocks hold
//      bit-identical hyperparameters without a broadcast.
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
// step, c1 = exp(-(eps/2)/L), c2 = sqrt(1 - c1^2) scaled by 1/sqrt(d).
__device__ __forceinline__ void set_step_scalars(const Hyper& H, int d, float& eps, float& c1,
                                                 float& c2s) {
    eps = (float)H.eps;
    const double e = exp(-0.5 * H.eps / H.L);
    c1 = (float)e;
    c2s = (float)(sqrt(1.0 - e * e) / sqrt((double)d));
}

// ---------------------------------------------------------------- the kernel
template <int KIND, int LPC, int CPL>
__global__ void __launch_bounds__(kMaxThreads) laps_resident_kernel(const KParams P,
                                                                   const Coefs* __restrict__ coefs) {
    constexpr int NB = CPL / 4;
    constexpr int GPW = 32 / LPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Hyper H;
    __shared__ Coefs CF;
    __shared__ double s_fin[NCS + NSL];
    __shared__ int s_switch;
    __shared__ float s_eps, s_c1, s_c2s;  // step scalars of the next iteration (FP32)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int gl = lane & (LPC - 1), grp = lane / LPC;
    const int slot = warp * GPW + grp, slots = nwarps * GPW;
    const int G = P.G;
    const int m = blockIdx.x * slots + slot;
    const bool active = m < P.M;
    const int dp = P.d_pad;
    const unsigned gmask = ((LPC == 32) ? 0xffffffffu : ((1u << LPC) - 1u)) << (grp * LPC);

    float* sq = reinterpret_cast<float*>(smem_raw);                      // [nwarps][d_pad]
    double* s_cs = reinterpret_cast<double*>(sq + (size_t)nwarps * dp);  // [slots][NCS]
    const int i0 = (int)(((long long)blockIdx.x * P.d) / G);
    const int i1 = (int)(((long long)(blockIdx.x + 1) * P.d) / G);
    double* s_sl = s_cs + (size_t)slots * NCS;                           // [i1-i0][NSL]

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
        const double l = P.logp[m];
        lp.hi = (float)l;
        lp.lo = (float)(l - (double)lp.hi);
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
    }

    const int n_iter = (P.mode == 0) ? 1 : P.n_iters;

    for (int it = 0; it < n_iter; ++it) {
        if (P.mode == 1 && H.done) break;
        // ------------------------------------------------ 1. chain update
        double c_d = 0.0, c_d2 = 0.0, c_fin = 0.0, c_bad = 0.0, c_a = 0.0;
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
                const float logU = logf(u01(r.x));
                const ff s = ff_add(dl, logU);
                keep = !bad && (s.hi < 0.0f || (s.hi == 0.0f && s.lo < 0.0f));
                a_m = bad ? 0.0f : (dl.hi <= 0.0f ? 1.0f : expf(-(dl.hi + dl.lo)));
            }
            if (!keep) {
#pragma unroll
                for (int q = 0; q < CPL; ++q) { y[q] = y0[q]; g[q] = g0[q]; u[q] = u0[q]; }
                lp = lp0;
            }
            if (active && gl == 0) {  // one lane per chain does the FP64 bookkeeping
                if (H.phase == 0) {
                    if (bad) c_bad = 1.0;
                    else {
                        const double dd = ff_to_double(dl);
                        c_d = dd; c_d2 = dd * dd; c_fin = 1.0;
                    }
                } else {
                    c_a = a_m;
                    c_bad = bad ? 1.0 : 0.0;
                }
            }
        }
        // ------------------------------------------------ 2. block partials
        for (int qd = 0; qd < NQ; ++qd) {
            if (H.phase == 1 && P.mode == 1 && qd >= 2) break;  // g sums unused after the switch
#pragma unroll
            for (int k = 0; k < NB; ++k) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int q = 4 * k + c;
                    float v = qd == 0 ? y[q] : qd == 1 ? y[q] * y[q] : qd == 2 ? g[q] : y[q] * g[q];
                    v = active ? v : 0.0f;
                    v = across_groups<LPC>(v);
                    const int j = gl + LPC * k;
                    if (grp == 0 && j < P.nblk) sq[warp * dp + 4 * j + c] = v;
                }
            }
            __syncthreads();
            for (int col = tid; col < dp; col += blockDim.x) {
                ff s = ff_make(0.0f);
                for (int w = 0; w < nwarps; ++w) s = ff_add(s, sq[w * dp + col]);
                P.part_coord[((size_t)qd * dp + col) * G + blockIdx.x] = ff_to_double(s);
            }
            __syncthreads();
        }
        if (gl == 0) {
            double* cs = s_cs + (size_t)slot * NCS;
            cs[CS_DSUM] = c_d; cs[CS_DSQ] = c_d2; cs[CS_NFIN] = c_fin; cs[CS_NBAD] = c_bad;
            cs[CS_ASUM] = c_a;
        }
        __syncthreads();
        if (tid < NCS) {
            double s = 0.0;
            for (int sl = 0; sl < slots; ++sl) s += s_cs[(size_t)sl * NCS + tid];
            P.part_chain[(size_t)tid * G + blockIdx.x] = s;
        }
        // ------------------------------------------------ 3. slice reduction
        if (!grid_barrier(P.bar_count, P.bar_gen, P.status, G + P.bar_extra, P.timeout_ns)) return;
        const bool push = (P.mode == 1 && H.phase == 0);
        const bool have_g = !(P.mode == 1 && H.phase == 1);
        for (int i = i0 + warp; i < i1; i += nwarps) {
            double s[NQ];
#pragma unroll
            for (int qd = 0; qd < NQ; ++qd) {
                double a = 0.0;
                if (qd < 2 || have_g)
                    for (int c = lane; c < G; c += 32)
                        a += __ldcg(&P.part_coord[((size_t)qd * dp + i) * G + c]);
                s[qd] = warp_sum_d(a);
            }
            if (lane == 0) {
                const double iM = 1.0 / (double)P.M;
                const double mean = s[0] * iM, ey2 = s[1] * iM;
                const double var_y = ey2 - mean * mean;
                const double sgi = (double)P.sigma[i];
                const double var_x = sgi * sgi * var_y, ex2 = sgi * sgi * ey2;
                const double V = -(s[3] * iM - mean * (s[2] * iM));
                double del = 0.0;
                if (push) {
                    const int slotw = H.win_n % P.T;
                    const bool full = H.win_n >= P.T;
                    double* w = P.win + (size_t)slotw * dp + i;
                    const double old = full ? *w : 0.0;
                    *w = ex2;
                    const double s1 = P.win_s1[i] + ex2 - old;
                    const double s2 = P.win_s2[i] + ex2 * ex2 - old * old;
                    P.win_s1[i] = s1;
                    P.win_s2[i] = s2;
                    if (H.win_n + 1 >= P.T) {
                        const double mu = s1 / P.T;
                        const double vv = (s2 - s1 * s1 / P.T) / (P.T - 1);
                        del = sqrt(vv > 0.0 ? vv : 0.0) / mu;
                    }
                }
                double b2 = 0.0;
                if (P.Ex2) {
                    const double e = ex2 - P.Ex2[i];
                    b2 = e * e / P.Varx2[i];
                }
                P.var_y[i] = var_y;
                double* o = s_sl + (size_t)(i - i0) * NSL;
                o[SL_VAR] = var_x;
                o[SL_DV] = (1.0 - V) * (1.0 - V);
                o[SL_MAXDEL] = del;
                o[SL_B2SUM] = b2;
                o[SL_B2MAX] = b2;
            }
        }
        __syncthreads();
        if (tid < NSL) {
            double a = 0.0;  // sums start at 0; maxima too (all terms are >= 0)
            for (int i = i0; i < i1; ++i) {
                const double v = s_sl[(size_t)(i - i0) * NSL + tid];
                if (tid == SL_MAXDEL || tid == SL_B2MAX) a = (v > a || v != v) ? v : a;
                else a += v;
            }
            P.part_slice[(size_t)tid * G + blockIdx.x] = a;
        }
        // ------------------------------------------------ 4. finalise
        if (!grid_barrier(P.bar_count, P.bar_gen, P.status, G + P.bar_extra, P.timeout_ns)) return;
        for (int col = warp; col < NCS + NSL; col += nwarps) {
            const double* src = col < NCS ? P.part_chain + (size_t)col * G
                                          : P.part_slice + (size_t)(col - NCS) * G;
            const bool is_max = (col == NCS + SL_MAXDEL) || (col == NCS + SL_B2MAX);
            double a = 0.0;
            for (int c = lane; c < G; c += 32) {
                const double v = __ldcg(src + c);
                a = is_max ? ((v > a || v != v) ? v : a) : a + v;
            }
            s_fin[col] = is_max ? warp_max_d(a) : warp_sum_d(a);
        }
        __syncthreads();
        if (tid == 0) {
            const double d = (double)P.d;
            const double sum_var = s_fin[NCS + SL_VAR];
            s_switch = 0;
            if (P.mode == 0) {
                H.eps = P.eps0;
                H.L = P.alpha * sqrt(sum_var);
                H.t0_ns = global_ns();
            } else if (H.phase == 0) {
                // Sec. 3.1: EEVPD, D~, desired EEVPD, new step size; Eq. "L"
                const double nfin = s_fin[CS_NFIN], nbad = s_fin[CS_NBAD];
                double eevpd = NAN;
                if (nfin > 0) {
                    const double mean = s_fin[CS_DSUM] / nfin;
                    const double sq2 = s_fin[CS_DSQ] / nfin;
                    eevpd = (P.eevpd_centered ? sq2 - mean * mean : sq2) / d;
                }
                const double D = s_fin[NCS + SL_DV] / d;
                const double cd = P.C * D, rt = sqrt(cd);
                const double wanted = 4.0 * cd * rt / ((1.0 + rt) * (1.0 + rt));
                H.eps_used = H.eps;
                if (nbad > 0 || !(eevpd > 0) || !isfinite(eevpd) || !isfinite(wanted))
                    H.eps = 0.5 * H.eps;
                else
                    H.eps = H.eps * pow(wanted / eevpd, 1.0 / 6.0);
                H.L = P.alpha * sqrt(sum_var);
                H.t += 1;
                H.grads += 1;
                H.win_n += 1;
                H.eevpd = eevpd;
                H.eevpd_wanted = wanted;
                H.dtilde = D;
                H.max_delta = (H.win_n >= P.T) ? s_fin[NCS + SL_MAXDEL] : NAN;
                H.acc = NAN;
                H.nonfinite_last = (int)nbad;
                H.nonfinite_total += (int)nbad;
                bool sw = (H.win_n >= P.T) && (s_fin[NCS + SL_MAXDEL] < P.switch_tol);
                if (P.force_switch_at > 0) sw = H.t >= P.force_switch_at;
                if (sw && P.adjusted && H.t < P.n_total) {
                    s_switch = 1;
                    if (sum_var > 0) H.eps *= sqrt(d / sum_var);
                    H.integ = (P.d > P.mn4_min_dim) ? INTEG_MN4 : INTEG_MN2;
                    H.a_target = (H.integ == INTEG_MN4) ? P.a_target_mn4 : P.a_target_mn2;
                    H.L = P.adj_L_factor * P.N * H.eps;
                    H.lo = 0.0;
                    H.hi = 0.0;
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
                const double a = s_fin[CS_ASUM] / (double)P.M;
                const double nbad = s_fin[CS_NBAD];
                H.eps_used = H.eps;
                H.adapting = H.adapting && (fabs(a - H.a_target) > P.acc_tol);
                if (H.adapting) {
                    if (a > H.a_target) {
                        H.lo = H.eps;
                        H.eps = (H.hi > 0) ? 0.5 * (H.lo + H.hi) : 2.0 * H.eps;
                    } else {
                        H.hi = H.eps;
                        H.eps = (H.lo > 0) ? 0.5 * (H.lo + H.hi) : 0.5 * H.eps;
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
            H.sum_var = sum_var;
            const uint64_t now = global_ns();
            if (P.Ex2) {
                H.b2_avg = s_fin[NCS + SL_B2SUM] / d;
                H.b2_max = s_fin[NCS + SL_B2MAX];
                const double b2 = P.stop_b2_max ? H.b2_max : H.b2_avg;
                if (H.b2_first_t < 0 && b2 < 0.01) {
                    H.b2_first_t = H.t;
                    H.b2_first_grads = H.grads;
                    H.b2_first_ns = (double)(now - H.t0_ns);
                }
                if (P.stop_b2 > 0 && b2 < P.stop_b2) H.done = 1;
            } else {
                H.b2_avg = H.b2_max = NAN;
            }
            set_step_scalars(H, P.d, s_eps, s_c1, s_c2s);
            if (blockIdx.x == 0 && H.iters < P.trace_cap) {
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
                r.sum_var = sum_var;
                r.nonfinite = P.mode == 0 ? 0 : H.nonfinite_last;
                r.adapting = H.adapting;
                r.grads = H.grads;
                r.time_ns = (double)(now - H.t0_ns);
                P.trace[H.iters] = r;
            }
        }
        __syncthreads();
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
                        const double v = __ldcg(&P.var_y[i]);
                        s = v > 0.0 ? (float)sqrt(v) : 1.0f;
                    }
                    const int q = 4 * k + c;
                    sg[q] = s;
                    y[q] = y[q] / s;
                    g[q] = g[q] * s;
                }
            }
            for (int i = i0 + tid; i < i1; i += blockDim.x) {
                const double v = __ldcg(&P.var_y[i]);
                P.sigma[i] = v > 0.0 ? (float)sqrt(v) : 1.0f;
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
    if (active && gl == 0) P.logp[m] = ff_to_double(lp);
    if (blockIdx.x == 0 && tid == 0) *P.hyper = H;
}

// Host-side dispatch helpers, defined per target in laps_resident_<kind>.cu.
struct ResidentShape {
    int lpc, cpl;
};

}  // namespace laps
