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
#include "laps_finalise.cuh"

namespace laps {

// ---------------------------------------------------------------- phase timing
// Built only with -DLAPS_PHASE_TIMING (a diagnostic build): block
// LAPS_PHASE_BLOCK (default 0) adds the %globaltimer time spent between
// consecutive marks to P.phase_ns[k].
#ifdef LAPS_PHASE_TIMING
#define LAPS_PHASE_MARK(k)                                                              \
    do {                                                                                \
        __syncthreads();                                                                \
        if (blockIdx.x == LAPS_PHASE_BLOCK && threadIdx.x == 0 && P.phase_ns) {         \
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

// ---------------------------------------------------------------- full-rank proxy
// ±1 with the sign of bit `sh` of w (set: +1), as a float: the bit moved to the
// sign position and flipped against -1.0f
__device__ __forceinline__ float pm_one(uint32_t w, uint32_t sh) {
    return __int_as_float(((w >> sh) << 31) ^ 0xBF800000u);
}

// App. B "Full rank", the block's share: with z_k the K Rademacher vectors of
// step t and the common shifts ybar', gbar' (the ensemble means of the previous
// iteration, read from the per-coordinate results), the block's records
// Q_ik = sum_m y'_mi s'_mk and sum_m s'_mk of y' = y - ybar', s'_k = (g - gbar') . z_k
// (see fr_stride()).  The slice owners add the blocks' records and correct
// for the shift with the current means, so no product of uncentred values
// enters a covariance.  Both products are register-tiled, four chains (or
// coordinates) by four vectors per thread, on shared memory.
// Step one, inlined: the chains' y and g into shared memory (padding as zeros).
template <int LPC, int CPL>
__device__ __forceinline__ void fullrank_stage(const KParams& P, const float (&y)[CPL], const float (&g)[CPL],
                                               bool active, int slot, int gl, float* f_y, float* f_g) {
    const int dp = P.d_pad;
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = gl + LPC * k;
        if (j < P.nblk) {
            float4 vy, vg;
            float* py = &vy.x;
            float* pg = &vg.x;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const bool in = active && 4 * j + c < P.d;
                py[c] = in ? y[4 * k + c] : 0.0f;
                pg[c] = in ? g[4 * k + c] : 0.0f;
            }
            *reinterpret_cast<float4*>(f_y + (size_t)slot * dp + 4 * j) = vy;
            *reinterpret_cast<float4*>(f_g + (size_t)slot * dp + 4 * j) = vg;
        }
    }
}

// Diagnostic build only: the timed block adds the time of the full-rank
// sub-steps to P.phase_ns[8 + k].
#ifdef LAPS_PHASE_TIMING
#define FR_MARK(k)                                                    \
    do {                                                              \
        __syncthreads();                                              \
        if (blockIdx.x == LAPS_PHASE_BLOCK && threadIdx.x == 0 && P.phase_ns) { \
            const unsigned long long now_ = global_ns();              \
            P.phase_ns[8 + (k)] += now_ - fr_t_;                      \
            fr_t_ = now_;                                             \
        }                                                             \
    } while (0)
#else
#define FR_MARK(k) \
    do {           \
    } while (0)
#endif

// Step two, the products; all threads of the block call it after the staging.
// Only the kernels built with the full-rank proxy contain it, so its register
// tiles do not raise the pressure of the diagonal kernels' chain update.
// my, mg: thread tid's coordinate of the shifts (tid < d; threads >= d_pad).
__device__ __forceinline__ void fullrank_products(const KParams& P, const Hyper& H, int slots, int K, int K4,
                                               int nzw, float my, float mg, float* f_y, float* f_g, float* f_s,
                                               float* f_my, float* f_mg, uint32_t* f_z) {
    const int tid = threadIdx.x, dp = P.d_pad, G = P.G, b = blockIdx.x;
    const int nb = min(slots, P.M - b * slots);
#ifdef LAPS_PHASE_TIMING
    unsigned long long fr_t_ = global_ns();
#endif
    if (tid < dp) {
        f_my[tid] = my;
        f_mg[tid] = mg;
    }
    const int n128 = nzw / 4;
    for (int w = tid; w < K * n128; w += blockDim.x) {
        const int blk = w % n128, k = w / n128;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)k, (uint32_t)H.t, TAG_Z | (P.pid << 8)),
                                      P.seed_lo, P.seed_hi);
        f_z[(size_t)(4 * blk + 0) * K4 + k] = r.x;
        f_z[(size_t)(4 * blk + 1) * K4 + k] = r.y;
        f_z[(size_t)(4 * blk + 2) * K4 + k] = r.z;
        f_z[(size_t)(4 * blk + 3) * K4 + k] = r.w;
    }
    if (K4 > K)
        for (int w = tid; w < nzw * (K4 - K); w += blockDim.x)
            f_z[(size_t)(w / (K4 - K)) * K4 + K + w % (K4 - K)] = 0u;
    __syncthreads();
    // centre the block's chains (padding coordinates stay zero, idle slots stay zero)
    for (int o = tid; o < nb * dp; o += blockDim.x) {
        const int i = o % dp;
        f_y[o] -= f_my[i];
        f_g[o] -= f_mg[i];
    }
    __syncthreads();
    FR_MARK(0);
    // s' = G' Z over the block's slots: z multiplies exactly (±1).  Task (js, tile)
    // adds coordinate blocks [js nblk / JS, (js + 1) nblk / JS) into buffer js.
    const int ntk = K4 / 4, nts = (slots + 3) / 4, ntile = nts * ntk;
    const int JS = fr_jsplit(dp, slots, K, blockDim.x);
    float* f_sp = reinterpret_cast<float*>(f_z + (size_t)nzw * K4);  // [JS - 1][slots][K4]
    for (int task = tid; task < JS * ntile; task += blockDim.x) {
        const int js = task / ntile, tile = task - js * ntile;
        const int s0 = 4 * (tile / ntk), k0 = 4 * (tile - (tile / ntk) * ntk);
        const int j0 = (js * P.nblk) / JS, j1 = ((js + 1) * P.nblk) / JS;
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = 0.0f;
        for (int j = j0; j < j1; ++j) {
            const uint4 w = *reinterpret_cast<const uint4*>(f_z + (size_t)(j >> 3) * K4 + k0);
            float4 gv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
                gv[a] = s0 + a < slots ? *reinterpret_cast<const float4*>(f_g + (size_t)(s0 + a) * dp + 4 * j)
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t sh = (uint32_t)((4 * j + c) & 31);
                const float z[4] = {pm_one(w.x, sh), pm_one(w.y, sh), pm_one(w.z, sh), pm_one(w.w, sh)};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float gc = c == 0 ? gv[a].x : c == 1 ? gv[a].y : c == 2 ? gv[a].z : gv[a].w;
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[a][q] = fmaf(gc, z[q], acc[a][q]);
                }
            }
        }
        float* dst = js == 0 ? f_s : f_sp + (size_t)(js - 1) * slots * K4;
#pragma unroll
        for (int a = 0; a < 4; ++a)
            if (s0 + a < slots)
                *reinterpret_cast<float4*>(dst + (size_t)(s0 + a) * K4 + k0) =
                    make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
    }
    if (JS > 1) {
        __syncthreads();
        for (int o = tid; o < slots * K4; o += blockDim.x) {
            float v = f_s[o];
            for (int js = 1; js < JS; ++js) v += f_sp[(size_t)(js - 1) * slots * K4 + o];
            f_s[o] = v;
        }
    }
    __syncthreads();
    FR_MARK(1);
    float* R = reinterpret_cast<float*>(reinterpret_cast<char*>(P.part) + fr_offset(dp, G)) +
               (size_t)b * fr_stride(dp, K);
    for (int k = tid; k < K4; k += blockDim.x) {
        float ss = 0.0f;
        for (int sl = 0; sl < nb; ++sl) ss += f_s[(size_t)sl * K4 + k];
        R[(size_t)dp * K4 + k] = ss;
    }
    FR_MARK(2);
    // Q = Y'^T S' over the block's chains, rows of K4 floats (coalesced float4 stores)
    const int nti = (P.d + 3) / 4;
    for (int tile = tid; tile < nti * ntk; tile += blockDim.x) {
        const int i0 = 4 * (tile / ntk), k0 = 4 * (tile - (tile / ntk) * ntk);
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = 0.0f;
        for (int sl = 0; sl < nb; ++sl) {
            const float4 yv = *reinterpret_cast<const float4*>(f_y + (size_t)sl * dp + i0);
            const float4 sv = *reinterpret_cast<const float4*>(f_s + (size_t)sl * K4 + k0);
            const float ya[4] = {yv.x, yv.y, yv.z, yv.w}, sa[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[a][q] = fmaf(ya[a], sa[q], acc[a][q]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
            *reinterpret_cast<float4*>(R + (size_t)(i0 + a) * K4 + k0) =
                make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
    }
    FR_MARK(3);
}

// ---------------------------------------------------------------- the kernel
template <int KIND, int LPC, int CPL, bool FR>
__global__ void __launch_bounds__(kMaxThreads) laps_resident_kernel(const KParams P,
                                                                   const Coefs* __restrict__ coefs) {
    constexpr int NB = CPL / 4;
    constexpr int GPW = 32 / LPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Hyper H;
    __shared__ Coefs CF;
    __shared__ FinShared FS;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int gl = lane & (LPC - 1), grp = lane / LPC;
    const int slot = warp * GPW + grp, slots = nwarps * GPW;
    const int G = P.G;
    const int m = blockIdx.x * slots + slot;
    const bool active = m < P.M;
    const int dp = P.d_pad;
    const unsigned gmask = ((LPC == 32) ? 0xffffffffu : ((1u << LPC) - 1u)) << (grp * LPC);

    // dynamic shared memory
    float* sq = reinterpret_cast<float*>(smem_raw);                  // [qpp][nwarps][dp]
    float* s_cs = sq + (size_t)P.qpp * nwarps * dp;                   // [slots][NCSF]
    float* s_var = s_cs + (size_t)slots * NCSF;                       // [dp] Var y (switch)
    ff* s_q = reinterpret_cast<ff*>(s_var + dp);                      // [NQ][smax] + [NCS]
    // full-rank bias proxy only (App. B "Full rank", K Rademacher vectors); the
    // layout is the one fullrank_smem() sizes
    const int KF = FR ? P.dfull_K : 0, K4 = (KF + 3) & ~3, nzw = ((dp + 127) / 128) * 4;
    ff* s_fr = s_q + (size_t)NQ * P.smax + NCS;  // [3 threads] + [smax K]: the slice owners' partials
    float* f_y = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(s_fr + (size_t)P.smax * KF + 3 * blockDim.x) + 15) & ~(uintptr_t)15);  // [slots][dp]
    float* f_g = f_y + (size_t)slots * dp;                   // [slots][dp]
    float* f_s = f_g + (size_t)slots * dp;                   // [slots][K4]
    float* f_my = f_s + (size_t)slots * K4;                  // [dp] shift ybar'
    float* f_mg = f_my + dp;                                 // [dp] shift gbar'
    uint32_t* f_z = reinterpret_cast<uint32_t*>(f_mg + dp);  // [nzw][K4] Rademacher words
    // dense-precision Gaussian only: P [dp][dp], then one row of x per chain slot,
    // after the reduction's rows (dense_smem() sizes it)
    float* dsm = nullptr;
    if constexpr (KIND == TGT_GAUSS_DENSE) {
        dsm = reinterpret_cast<float*>(
            (reinterpret_cast<uintptr_t>(s_q + (size_t)NQ * P.smax + NCS) + 15) & ~(uintptr_t)15);
        for (int o = tid; o < dp * dp / 4; o += blockDim.x)
            reinterpret_cast<float4*>(dsm)[o] = reinterpret_cast<const float4*>(P.prec)[o];
    }

    if (tid == 0) {
        H = *P.hyper;
        set_step_scalars(H, P.d, FS.eps, FS.c1, FS.c2s);
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
        lp = eval_target<KIND, LPC, CPL>(P, gl, lane, dsm, y, g, pr, sg);
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
    // the O maps' noise of an unadjusted step depends only on its counters, so the
    // next step's is drawn while this iteration's grid barriers are outstanding
    // (z_o1 in the first, z_o2 in the second); z_t names the step it belongs to
    float z_o1[CPL], z_o2[CPL];
    bool z_pre = false;
    uint32_t z_t = 0u;
    // likewise a MAMS proposal's first step's O-map noise (z_o1, z_o2), drawn inside the
    // previous proposal's barriers; a_t names the step it belongs to
    bool a_pre = false;
    uint32_t a_t = 0u;
#ifdef LAPS_PHASE_TIMING
    unsigned long long phase_t_ = 0;
#endif
    for (int it = 0; it < n_iter; ++it) {
        if (P.mode == 1 && H.done) break;
        LAPS_PHASE_MARK(0);
        // full-rank proxy: the previous iteration's means (the block products' shift),
        // loaded now so that their latency hides behind the chain update
        float fr_my = 0.0f, fr_mg = 0.0f;
        if (FR && KF > 0 && P.mode == 1 && H.phase == 0 && tid < P.d) {
            fr_my = __ldcg(P.cstat + (size_t)tid * NCO + CO_MY);
            fr_mg = __ldcg(P.cstat + (size_t)tid * NCO + CO_MG);
        }
        // ------------------------------------------------ 1. chain update
        ff c_d = ff_make(0.0f);
        float c_d2 = 0.0f, c_fin = 0.0f, c_bad = 0.0f, c_a = 0.0f;
        if (P.mode == 1) {
            const float eps = FS.eps, c1 = FS.c1, c2s = FS.c2s;
            float y0[CPL], g0[CPL], u0[CPL];
            const ff lp0 = lp;
#pragma unroll
            for (int q = 0; q < CPL; ++q) { y0[q] = y[q]; g0[q] = g[q]; u0[q] = u[q]; }
            ff dl = ff_make(0.0f);
            if (H.phase == 0) {
                const uint32_t t = (uint32_t)H.t;
                if (!(z_pre && z_t == t)) {
                    o_noise<LPC, CPL>(P, gl, active, m, t, TAG_O1, z_o1);
                    o_noise<LPC, CPL>(P, gl, active, m, t, TAG_O2, z_o2);
                }
                o_apply<LPC, CPL>(P, gl, c1, c2s, z_o1, u);
                phi_step_k<KIND, LPC, CPL, 2>(P, CF, INTEG_LF, eps, gl, lane, dsm, y, u, g, lp, dl, pr, sg);
                o_apply<LPC, CPL>(P, gl, c1, c2s, z_o2, u);
            } else {
                // App. F step 2: u uniform on the sphere
                const uint32_t pidx = (uint32_t)H.p;
                const uint32_t t0 = (uint32_t)H.t;
                const bool pre = a_pre && a_t == t0;
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
                for (int n = 0; n < P.N; ++n) {
                    if (n > 0 || !pre) {
                        o_noise<LPC, CPL>(P, gl, active, m, t0 + n, TAG_O1, z_o1);
                        o_noise<LPC, CPL>(P, gl, active, m, t0 + n, TAG_O2, z_o2);
                    }
                    o_apply<LPC, CPL>(P, gl, c1, c2s, z_o1, u);
                    if (H.integ == INTEG_MN2)
                        phi_step_k<KIND, LPC, CPL, 3>(P, CF, INTEG_MN2, eps, gl, lane, dsm, y, u, g, lp, dl, pr,
                                                      sg);
                    else
                        phi_step<KIND, LPC, CPL>(P, CF, H.integ, eps, gl, lane, dsm, y, u, g, lp, dl, pr, sg);
                    o_apply<LPC, CPL>(P, gl, c1, c2s, z_o2, u);
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
        const int nq = ens_nq(P, H);
        if (nq == NQ && P.qpp >= NQ) {
            // all four quantities in one pass (the usual case): y, y^2, g, y g of each
            // coordinate formed together; the same values and summation order as below
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int j = gl + LPC * k;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int q = 4 * k + c;
                    const float yv = active ? y[q] : 0.0f, gv = active ? g[q] : 0.0f;
                    const float v0 = across_groups<LPC>(yv), v1 = across_groups<LPC>(yv * yv);
                    const float v2 = across_groups<LPC>(gv), v3 = across_groups<LPC>(yv * gv);
                    if (grp == 0 && j < P.nblk) {
                        float* row = sq + (size_t)warp * dp + 4 * j + c;
                        row[0] = v0;
                        row[(size_t)nwarps * dp] = v1;
                        row[(size_t)2 * nwarps * dp] = v2;
                        row[(size_t)3 * nwarps * dp] = v3;
                    }
                }
            }
            __syncthreads();
            for (int col = tid; col < NQ * dp; col += blockDim.x) {
                const int qd = col / dp, i = col - qd * dp;
                if (i >= P.d) continue;
                ff s = ff_make(0.0f);
                const float* src = sq + (size_t)qd * nwarps * dp + i;
                for (int w = 0; w < nwarps; ++w) s = ff_add(s, src[(size_t)w * dp]);
                P.part[((size_t)qd * dp + i) * G + blockIdx.x] = make_float2(s.hi, s.lo);
            }
            __syncthreads();
        } else
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
        if (FR && KF > 0 && P.mode == 1 && H.phase == 0) {
            fullrank_stage<LPC, CPL>(P, y, g, active, slot, gl, f_y, f_g);
            fullrank_products(P, H, slots, KF, K4, nzw, fr_my, fr_mg, f_y, f_g, f_s, f_my, f_mg, f_z);
        }
        LAPS_PHASE_MARK(3);
        // ------------------------------------------------ 3. barrier, then this block's slice
        // an unadjusted iteration that is not the launch's last draws the next step's
        // noise (step t + 1 if this iteration stays unadjusted) inside its barriers
        // (not with the full-rank proxy or 16 coordinates per lane, whose kernels have
        // no registers to spare)
        const bool z_next = !FR && CPL <= 8 && P.mode == 1 && H.phase == 0 && it + 1 < n_iter;
        const uint32_t t_next = (uint32_t)H.t + 1u;
        // a proposal that is not the launch's last draws the next one's first step's O-map
        // noise (step t + N) the same way
        const bool a_next = !FR && CPL <= 8 && P.mode == 1 && H.phase == 1 && it + 1 < n_iter;
        const uint32_t t0_next = (uint32_t)H.t + (uint32_t)P.N;
        n_bar += 1;
        grid_arrive(P.bar_count);
        if (z_next) o_noise<LPC, CPL>(P, gl, active, m, t_next, TAG_O1, z_o1);
        if (a_next) o_noise<LPC, CPL>(P, gl, active, m, t0_next, TAG_O1, z_o1);
        if (!grid_wait(P.bar_count, P.status, n_bar * (unsigned)(G + P.bar_extra), P.timeout_ns)) return;
        LAPS_PHASE_MARK(4);
        ens_slice(P, H, s_q, blockIdx.x, G, FR ? s_fr : nullptr);
        LAPS_PHASE_MARK(5);
        // ------------------------------------------------ 4. barrier, then every block gathers
        n_bar += 1;
        grid_arrive(P.bar_count);
        if (z_next) o_noise<LPC, CPL>(P, gl, active, m, t_next, TAG_O2, z_o2);
        if (a_next) o_noise<LPC, CPL>(P, gl, active, m, t0_next, TAG_O2, z_o2);
        if (!grid_wait(P.bar_count, P.status, n_bar * (unsigned)(G + P.bar_extra), P.timeout_ns)) return;
        z_pre = z_next;
        z_t = t_next;
        a_pre = a_next;
        a_t = t0_next;
        LAPS_PHASE_MARK(6);
        ens_gather(P, H, s_var, FS);
        // the trace row (block 0), written by the last warp while the others go on
        if (blockIdx.x == 0 && tid == blockDim.x - 32) ens_trace_row(P, H, FS.now);
        LAPS_PHASE_MARK(7);
        if (FS.sw) {
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
