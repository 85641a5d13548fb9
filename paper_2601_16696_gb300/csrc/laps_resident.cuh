// laps_resident.cuh -- the per-chain maps of the LAPS kernels (sm_103a):
// the targets' log p and gradient in the sampler's coordinates, the O, B and A
// maps of App. E on a chain held by a group of LPC lanes (CPL coordinates per
// lane, in registers), the integrator step of Eq. "integrator", the step
// scalars of an iteration, and float-float helpers.  The register-resident
// kernel (laps_resident_kernel.cuh) and the streamed path build on these.
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
// Dense-precision Gaussian (Sec. 6, the rotated ill-conditioned Gaussian): r = P x
// for the group's chain.  dsm holds P [d_pad][d_pad] then one [d_pad] row per chain
// slot of the block.  The lanes stage their coordinates of x in the slot's row;
// each lane then forms its coordinates of P x over the d columns, reading row j of
// the symmetric P for column j (float4 reads, consecutive across the group's
// lanes), every product entering a float-float accumulator exactly (the
// compensated dot product of Ogita, Rump and Oishi, 2005): at condition numbers
// near 1e5 a binary32 sum loses ~1e-4 of the gradient to cancellation.
template <int LPC, int CPL>
__device__ __forceinline__ void dense_px(const KParams& P, int gl, float* dsm, const float (&x)[CPL],
                                         float (&r)[CPL]) {
    const int dp = P.d_pad;
    const float* sP = dsm;
    float* sx = dsm + (size_t)dp * dp + (size_t)(threadIdx.x / LPC) * dp;
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = gl + LPC * k;
        if (j < P.nblk)
            *reinterpret_cast<float4*>(sx + 4 * j) = make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
    }
    __syncwarp();
    float hi[CPL], lo[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) hi[q] = lo[q] = 0.0f;
    for (int jj = 0; jj < P.d; ++jj) {
        const float xj = sx[jj];
#pragma unroll
        for (int k = 0; k < CPL / 4; ++k) {
            const int j = gl + LPC * k;
            if (j >= P.nblk) continue;
            const float4 p4 = *reinterpret_cast<const float4*>(sP + (size_t)jj * dp + 4 * j);
            const float pc[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int q = 4 * k + c;
                const float pv = xj * pc[c];
                const float er = fmaf(xj, pc[c], -pv);  // exact: x_j P_ji = pv + er
                float sh, sl;
                two_sum(hi[q], pv, sh, sl);
                hi[q] = sh;
                lo[q] += sl + er;
            }
        }
    }
    __syncwarp();  // the slot's row is rewritten by the next evaluation
#pragma unroll
    for (int q = 0; q < CPL; ++q) r[q] = hi[q] + lo[q];
}

// log p at x = sigma o y and the gradient in y (sigma o grad_x).  Returns the
// group-wide log p as a compensated float-float.  dsm: GAUSS_DENSE only.
template <int KIND, int LPC, int CPL>
__device__ __forceinline__ ff eval_target(const KParams& P, int gl, int lane, float* dsm,
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
    } else if constexpr (KIND == TGT_GAUSS_DENSE) {
        float xt[CPL], r[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) xt[q] = sg[q] * y[q];
        dense_px<LPC, CPL>(P, gl, dsm, xt, r);
        float part = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            g[q] = sg[q] * (-r[q]);
            part = fmaf(-0.5f * xt[q], r[q], part);  // -1/2 x (P x)
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
__device__ __forceinline__ ff a_step(const KParams& P, int gl, int lane, float* dsm, float ae,
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
    } else if constexpr (KIND == TGT_GAUSS_DENSE) {
        // log p(x') - log p(x) = -1/2 (x' - x)^T P (x' + x) = 1/2 (x' - x).(g_x' + g_x)
        //                      = 1/2 sum_i (y'_i - y_i)(g_y'_i + g_y_i)
        float xn[CPL], r[CPL], dy[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const float yn = fmaf(ae, u[q], y[q]);
            dy[q] = yn - y[q];
            y[q] = yn;
            xn[q] = sg[q] * yn;
        }
        dense_px<LPC, CPL>(P, gl, dsm, xn, r);
        float part = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const float gn = sg[q] * (-r[q]);
            part = fmaf(0.5f * dy[q], gn + g[q], part);
            g[q] = gn;
        }
        return group_sum_ff<LPC>(ff_make(part));
    } else if constexpr (KIND == TGT_BANANA) {
        // the lane's few terms of the change in binary32 (each is small, of the
        // order of the step), the group's total in float-float
        float part = 0.0f;
#pragma unroll
        for (int q = 0; q < CPL; q += 2) {
            const float ao = sg[q] * y[q], bo = sg[q + 1] * y[q + 1];
            const float ya = fmaf(ae, u[q], y[q]), yb = fmaf(ae, u[q + 1], y[q + 1]);
            const float an = sg[q] * ya, bn = sg[q + 1] * yb;
            const float da = an - ao, db = bn - bo, sa = ao + an;
            const float ro = fmaf(-ao, ao, bo), rn = fmaf(-an, an, bn);
            const float dr = fmaf(-da, sa, db);
            part = fmaf(-0.5f * da, sa, part);
            part = fmaf(-0.5f * P.inv_s2 * dr, ro + rn, part);
            y[q] = ya;
            y[q + 1] = yb;
            const float ris = rn * P.inv_s2;
            g[q] = sg[q] * fmaf(2.0f * an, ris, -an);
            g[q + 1] = sg[q + 1] * (-ris);
        }
        return group_sum_ff<LPC>(ff_make(part));
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
// The noise Z of one O map (this lane's coordinate blocks), apart from the map
// itself: it depends only on the counters, so a step can draw both of its O
// maps' noise up front and the generator's arithmetic overlaps the reductions.
template <int LPC, int CPL>
__device__ __forceinline__ void o_noise(const KParams& P, int gl, bool active, uint32_t m, uint32_t t,
                                        uint32_t tag, float (&z)[CPL]) {
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = gl + LPC * k;
        float w[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (active && j < P.nblk) normals4(j, m, t, tag | (P.pid << 8), P.seed_lo, P.seed_hi, w);
#pragma unroll
        for (int c = 0; c < 4; ++c) z[4 * k + c] = w[c];
    }
}
template <int LPC, int CPL>
__device__ __forceinline__ void o_apply(const KParams& P, int gl, float c1, float c2s, const float (&z)[CPL],
                                        float (&u)[CPL]) {
    float n2 = 0.0f;
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = gl + LPC * k;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = (4 * j + c < P.d) ? fmaf(c1, u[4 * k + c], c2s * z[4 * k + c]) : 0.0f;
            u[4 * k + c] = v;
            n2 = fmaf(v, v, n2);
        }
    }
    n2 = group_sum<LPC>(n2);
    const float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) u[q] *= inv;
}
template <int LPC, int CPL>
__device__ __forceinline__ void o_update(const KParams& P, int gl, bool active, uint32_t m,
                                         uint32_t t, uint32_t tag, float c1, float c2s,
                                         float (&u)[CPL]) {
    float z[CPL];
    o_noise<LPC, CPL>(P, gl, active, m, t, tag, z);
    o_apply<LPC, CPL>(P, gl, c1, c2s, z, u);
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
        // per-chain scalars, evaluated by every lane of the group: 1/|g| from one
        // reciprocal square root (~2 ulp), zeta from 1 - zeta (accurate for small
        // delta), the denominator (in [2 zeta^2, 2], > 0) inverted approximately
        const float rg = rsqrtf(gg);
        const float gn = gg * rg;
        const float eu = gu * rg;
        const float delta = beps * gn * inv_dm1;
        const float om = -expm1f(-delta);  // 1 - zeta
        const float zeta = 1.0f - om;
        const float opz = 1.0f + zeta;
        const float den = fmaf(eu, om * opz, fmaf(zeta, zeta, 1.0f));
        const float inv = __fdividef(1.0f, den);
        const float cu = 2.0f * zeta * inv;
        const float ce = om * fmaf(eu, om, opz) * inv * rg;
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
                                         int gl, int lane, float* dsm, float (&y)[CPL], float (&u)[CPL],
                                         float (&g)[CPL], ff& lp, ff& dl, const float (&pr)[CPL],
                                         const float (&sg)[CPL]) {
    const float dm1 = (float)(P.d - 1), inv_dm1 = 1.0f / (float)(P.d - 1);
    const int K = cf.K[integ];
    for (int k = 0; k < K; ++k) {
        b_update<LPC, CPL>(cf.b[integ][k] * eps, inv_dm1, dm1, g, u, dl);
        if (k < K - 1) {
            const float ae = cf.a[integ][k] * eps;
            const ff dlp = a_step<KIND, LPC, CPL>(P, gl, lane, dsm, ae, y, u, g, pr, sg);
            dl = ff_add(dl, ff_neg(dlp));  // -log p(x') + log p(x)
            lp = ff_add(lp, dlp);
        }
    }
}

// the same with the number of B maps known at compile time (LF: 2, MN2: 3), so
// that the maps of one step are scheduled together
template <int KIND, int LPC, int CPL, int K>
__device__ __forceinline__ void phi_step_k(const KParams& P, const Coefs& cf, int integ, float eps,
                                           int gl, int lane, float* dsm, float (&y)[CPL], float (&u)[CPL],
                                           float (&g)[CPL], ff& lp, ff& dl, const float (&pr)[CPL],
                                           const float (&sg)[CPL]) {
    const float dm1 = (float)(P.d - 1), inv_dm1 = 1.0f / (float)(P.d - 1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        b_update<LPC, CPL>(cf.b[integ][k] * eps, inv_dm1, dm1, g, u, dl);
        if (k < K - 1) {
            const float ae = cf.a[integ][k] * eps;
            const ff dlp = a_step<KIND, LPC, CPL>(P, gl, lane, dsm, ae, y, u, g, pr, sg);
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

}  // namespace laps
