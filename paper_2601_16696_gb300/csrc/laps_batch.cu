// laps_batch.cu -- many independent LAPS problems (diagonal Gaussians of
// uneven dimension and ensemble size) in one persistent cooperative launch.
//
// The batch is too large for register residency (a d = 10^4 problem with
// 16384 chains alone is 1.3 GB of y and u), so the state streams from HBM:
// an unadjusted step reads and writes y and u once (16 bytes per coordinate);
// g and the energy error are recomputed from y (g = -prec o x, Eq. ECA's
// statistics need only sums of y and y^2 per coordinate for this target).
//
// A launch runs iterations of Algorithm 1 for every live problem in lockstep:
//   1. chain phase: a problem's chains are split evenly over a range of
//      blocks (host-side schedule, batch_schedule): every block when the
//      problem has at least one group-round of chains per block, else just
//      enough blocks for one round each, placed where the blocks carry the
//      least work, so that no block runs a round with most of its groups idle.
//      A chain is processed by a group of L lanes (4, 8 or 16 lanes of a warp
//      shared with other chains, or 1..16 whole warps; chosen per problem from
//      its d), with its coordinates in registers (CPL per lane) and group
//      reductions by butterflies over the group's lanes plus, across the
//      group's warps, shared memory and a named barrier.  Per-coordinate sums of y
//      and y^2 accumulate in shared memory per thread; the block writes one
//      float-float column per problem (the register-resident kernel's layout);
//   2. grid barrier; slice tasks (problem, block of coordinates) spread over
//      the blocks run ens_slice;
//   3. grid barrier; the finalise of problem p runs on block p mod G;
//   4. grid barrier.
// All sums have fixed orders; a result depends on the launch shape (the block
// and group counts fix the order of the column sums), not on timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "laps_internal.h"

namespace laps {

constexpr int kBT = 512;          // threads per block
constexpr int kBW = kBT / 32;     // warps per block
constexpr int kMaxGrp = kBT / 4;   // chain groups of a block at 4 lanes per chain
constexpr int kRed = 128;         // reduction scratch floats per group: 2 buffers x 4 values x 16 warps

struct BatchArgs {
    const KParams* probs;  // [n]
    const int* gw;         // [n] lanes per chain: 4, 8, 16 (chains share a warp) or 32 x warps
    const int2* sched;     // [n] (first block, blocks) that hold the problem's chains; P.G = blocks
    const Coefs* coefs;
    int n;                 // problems
    int mode;              // 0: initialise, 1: iterate
    int n_iters;
    int SL;                // coordinates per slice task
    int cap_pad;           // shared capacity of the per-coordinate constants (>= every d_pad)
    unsigned* bar_count;
    int* status;
    long long timeout_ns;
    int bar_extra;
    PhiloxKeys keys;       // round keys of the batch seed (every problem draws with it)
};

// ---------------------------------------------------------------- chain groups
struct Grp {
    int gw;      // warps in the group (1 for a group of 4, 8, 16 or 32 lanes)
    int grp;     // group index in the block
    int wig;     // warp in the group
    int gl;      // lane in the group (0 .. lpc - 1)
    int lpc;     // lanes per chain: 4, 8, 16 (part of a warp) or 32 gw
    float* red;  // this group's reduction scratch
    int flip;    // scratch buffer in use
};

__device__ __forceinline__ void grp_bar(const Grp& G) {
    if (G.gw > 1) asm volatile("bar.sync %0, %1;" ::"r"(1 + G.grp), "r"(32 * G.gw) : "memory");
}

// The group's warps' partials of value k sit at s[16 k + w] (w the warp in the
// group, gw in {1, 2, 4, 8, 16}).  Lane l < gw of every warp reads partial l and
// a butterfly over the warp adds them (the other lanes add zeros, exactly): every
// lane of the group ends with the same bits, with one load and five shuffle-adds a lane in
// place of gw sequential additions.
__device__ __forceinline__ float part_sum(const float* s, int gw) {
    const int lane = threadIdx.x & 31;
    float t = lane < gw ? s[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}
// float-float partials: high words at hi[w], low words at lo[w]
__device__ __forceinline__ ff part_sum_ff(const float* hi, const float* lo, int gw) {
    const int lane = threadIdx.x & 31;
    ff t = lane < gw ? ff{hi[lane], lo[lane]} : ff_make(0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        t = ff_add(t, ff{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)});
    return t;
}

// Sum of NV values over the group: warp butterfly, then a butterfly over the
// group's warp partials.  Two scratch buffers alternate, so one barrier per call suffices (a
// warp cannot run two calls ahead of the others).  Every lane gets the same bits.
template <int NV>
__device__ __forceinline__ void gsum(Grp& G, float (&v)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            if (o < G.lpc) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (G.gw == 1) return;
    float* s = G.red + G.flip * 64;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) s[16 * k + G.wig] = v[k];
    grp_bar(G);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = part_sum(s + 16 * k, G.gw);
    G.flip ^= 1;
}
__device__ __forceinline__ float gsum1(Grp& G, float v) {
    float a[1] = {v};
    gsum<1>(G, a);
    return a[0];
}
__device__ __forceinline__ ff gsum_ff(Grp& G, ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        if (o < G.lpc) v = ff_add(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    if (G.gw == 1) return v;
    float* s = G.red + G.flip * 64;
    if ((threadIdx.x & 31) == 0) {
        s[G.wig] = v.hi;
        s[16 + G.wig] = v.lo;
    }
    grp_bar(G);
    const ff t = part_sum_ff(s, s + 16, G.gw);
    G.flip ^= 1;
    return t;
}

// bytes (a multiple of 16) at a 16-byte aligned global address into L2
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes)
                 : "memory");
}

// ---------------------------------------------------------------- maps on a group
// App. E, Eq. "O update" (Z ~ N(0, I/d) per coordinate; c2s = c2 / sqrt(d))
template <int CPL>
__device__ __forceinline__ void g_o(const KParams& P, const PhiloxKeys& K, Grp& G, uint32_t m, uint32_t t,
                                    uint32_t tag, float c1, float c2s, float (&u)[CPL]) {
    float n2 = 0.0f;
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = G.gl + G.lpc * k;
        float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (j < P.nblk) normals4(j, m, t, tag | (P.pid << 8), K, z);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = (4 * j + c < P.d) ? fmaf(c1, u[4 * k + c], c2s * z[c]) : 0.0f;
            u[4 * k + c] = v;
            n2 = fmaf(v, v, n2);
        }
    }
    n2 = gsum1(G, n2);
    const float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) u[q] *= inv;
}

// The gradient in y of the diagonal Gaussian, g_y = sigma o (-prec o (sigma o y))
// = -c o y with c_i = prec_i sigma_i^2 (kept in shared memory per coordinate),
// for this thread's coordinate block k (recomputed where needed: one multiply,
// cheaper than keeping it in registers)
template <int CPL>
__device__ __forceinline__ void g_blk(const Grp& G, const KParams& P, const float (&y)[CPL], int k,
                                      const float4* s_c4, float (&g)[4]) {
    const int j = G.gl + G.lpc * k;
    if (j >= P.nblk) {
        g[0] = g[1] = g[2] = g[3] = 0.0f;
        return;
    }
    const float4 c = s_c4[j];
    g[0] = -c.x * y[4 * k];
    g[1] = -c.y * y[4 * k + 1];
    g[2] = -c.z * y[4 * k + 2];
    g[3] = -c.w * y[4 * k + 3];
}

// ---------------------------------------------------------------- fused step
// One step O_{eps/2} Phi_eps O_{eps/2} with fewer group reductions than maps:
// the first O map's |v|^2 is reduced together with g.v and |g|^2 (the first
// B's g.u is (g.v)/|v|); each A map's reduction carries the next B's |g'|^2
// and g'.u, while the A maps' log p changes stay per lane until the step's
// (or the proposal's) end, where they are reduced with the last O map's |v|^2
// and the non-finite flag of the chain update (`check`).  Each map is App. E's:
// O as g_o, B in the overflow-free zeta = e^-delta form, A with the log p
// change in difference form -1/2 prec (x' - x)(x' + x).

// one float-float and NV (<= 2) floats summed over the group in one pass
template <int NV>
__device__ __forceinline__ void gsum_mix(Grp& G, ff& a, float (&v)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (o >= G.lpc) continue;  // uniform: every group of the block has lpc lanes
        a = ff_add(a, ff{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if (G.gw == 1) return;
    float* s = G.red + G.flip * 64;
    if ((threadIdx.x & 31) == 0) {
        s[G.wig] = a.hi;
        s[16 + G.wig] = a.lo;
#pragma unroll
        for (int k = 0; k < NV; ++k) s[16 * (2 + k) + G.wig] = v[k];
    }
    grp_bar(G);
    a = part_sum_ff(s, s + 16, G.gw);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = part_sum(s + 16 * (2 + k), G.gw);
    G.flip ^= 1;
}

// u <- c1 u + c2s Z, not yet normalised; thread partials of |v|^2 (and, with
// WITH_G, of g.v and |g|^2 with g the gradient at y) into s
template <int CPL, bool WITH_G>
__device__ __forceinline__ void g_o_mix(const KParams& P, const PhiloxKeys& K, const Grp& G, uint32_t m,
                                        uint32_t t, uint32_t tag,
                                        float c1, float c2s, float (&u)[CPL], const float (&y)[CPL],
                                        const float4* s_c4, float (&s)[3]) {
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        const int j = G.gl + G.lpc * k;
        float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (j < P.nblk) normals4(j, m, t, tag | (P.pid << 8), K, z);
        float g[4];
        if (WITH_G) g_blk<CPL>(G, P, y, k, s_c4, g);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = (4 * j + c < P.d) ? fmaf(c1, u[4 * k + c], c2s * z[c]) : 0.0f;
            u[4 * k + c] = v;
            s[0] = fmaf(v, v, s[0]);
            if (WITH_G) {
                s[1] = fmaf(g[c], v, s[1]);
                s[2] = fmaf(g[c], g[c], s[2]);
            }
        }
    }
}

// B with its sums |g|^2 and g.u already reduced
template <int CPL>
__device__ __forceinline__ void g_b_apply(const Grp& G, const KParams& P, float beps, float inv_dm1, float dm1,
                                          float gg, float gu, const float (&y)[CPL], float (&u)[CPL], ff& dl,
                                          const float4* s_c4) {
    if (!(gg > 0.0f)) return;
    // per-chain scalars as in the resident kernel's B: 1/|g| from one reciprocal
    // square root, zeta from 1 - zeta, the positive denominator inverted approximately
    const float rg = rsqrtf(gg);
    const float gn = gg * rg;
    const float eu = gu * rg;
    const float delta = beps * gn * inv_dm1;
    const float om = -expm1f(-delta);
    const float zeta = 1.0f - om;
    const float opz = 1.0f + zeta;
    const float den = fmaf(eu, om * opz, fmaf(zeta, zeta, 1.0f));
    const float inv = __fdividef(1.0f, den);
    const float cu = 2.0f * zeta * inv;
    const float ce = om * fmaf(eu, om, opz) * inv * rg;
#pragma unroll
    for (int k = 0; k < CPL / 4; ++k) {
        float g[4];
        g_blk<CPL>(G, P, y, k, s_c4, g);
#pragma unroll
        for (int c = 0; c < 4; ++c) u[4 * k + c] = fmaf(cu, u[4 * k + c], ce * g[c]);
    }
    dl = ff_add(dl, dm1 * (delta + log1pf(-0.5f * om * opz * (1.0f - eu))));
}

// dl collects the B maps' kinetic-energy changes (per chain, the same on every
// lane); dlA each lane's part of the A maps' log-p changes, reduced over the
// group only when the energy error is read (check: the step's or the
// proposal's end), together with the last O map's norm.
template <int CPL>
__device__ __forceinline__ void g_step(const KParams& P, const PhiloxKeys& RK, Grp& G, const Coefs& CF, int integ,
                                       float eps, float c1, float c2s, uint32_t m, uint32_t t, float (&y)[CPL],
                                       float (&u)[CPL], ff& dl, ff& dlA, float inv_dm1, float dm1,
                                       const float4* s_c4, bool check, bool& bad) {
    const int K = CF.K[integ];
    float s[3] = {0.0f, 0.0f, 0.0f};
    g_o_mix<CPL, true>(P, RK, G, m, t, TAG_O1, c1, c2s, u, y, s_c4, s);
    gsum<3>(G, s);
    float inv = s[0] > 0.0f ? rsqrtf(s[0]) : 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) u[q] *= inv;
    float gg = s[2], gu = s[1] * inv;
    for (int k = 0; k < K; ++k) {
        g_b_apply<CPL>(G, P, CF.b[integ][k] * eps, inv_dm1, dm1, gg, gu, y, u, dl, s_c4);
        if (k < K - 1) {
            // A map, its log p change (difference form) and the next B's sums
            const float ae = CF.a[integ][k] * eps;
            float part = 0.0f, v2[2] = {0.0f, 0.0f};
#pragma unroll
            for (int kb = 0; kb < CPL / 4; ++kb) {
                const int j = G.gl + G.lpc * kb;
                if (j >= P.nblk) continue;
                const float4 c4 = s_c4[j];
                const float cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // log p(y') - log p(y) = -1/2 c (y' - y)(y' + y)
                    const int q = 4 * kb + c;
                    const float yo = y[q];
                    const float yn = fmaf(ae, u[q], yo);
                    part = fmaf(-0.5f * cs[c] * (yn - yo), yo + yn, part);
                    y[q] = yn;
                    const float g = -cs[c] * yn;
                    v2[0] = fmaf(g, g, v2[0]);
                    v2[1] = fmaf(g, u[q], v2[1]);
                }
            }
            gsum<2>(G, v2);
            dlA = ff_add(dlA, -part);
            gg = v2[0];
            gu = v2[1];
        }
    }
    float s2[3] = {0.0f, 0.0f, 0.0f};
    g_o_mix<CPL, false>(P, RK, G, m, t, TAG_O2, c1, c2s, u, y, s_c4, s2);
    if (check) {
        float f = (isfinite(dl.hi) && isfinite(dlA.hi)) ? 0.0f : 1.0f;
#pragma unroll
        for (int q = 0; q < CPL; ++q)
            if (!(isfinite(y[q]) && isfinite(u[q]))) f = 1.0f;
        float r[2] = {s2[0], f};
        gsum_mix<2>(G, dlA, r);  // the A maps' log-p change of the chain, with the O map's norm
        dl = ff_add(dl, dlA);
        dlA = ff_make(0.0f);
        s2[0] = r[0];
        bad = r[1] > 0.0f;
    } else {
        s2[0] = gsum1(G, s2[0]);
    }
    inv = s2[0] > 0.0f ? rsqrtf(s2[0]) : 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) u[q] *= inv;
}

// ---------------------------------------------------------------- the kernel
template <int CPL>
__global__ void __launch_bounds__(kBT, 1) batch_kernel(const __grid_constant__ BatchArgs B) {
    constexpr int NB = CPL / 4;
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ KParams sP;
    __shared__ Hyper sH;
    __shared__ Coefs CF;
    __shared__ FinShared FS;
    __shared__ float s_eps, s_c1, s_c2s;
    __shared__ int s_live;
    float* qbuf = reinterpret_cast<float*>(bsm);   // [2][ng][lpc CPL]: per-thread column sums
    float* s_c = qbuf + 2 * kBT * CPL;             // [cap_pad] prec_i sigma_i^2 (0 past d)
    float* s_sg = s_c + B.cap_pad;                 // [cap_pad] preconditioner
    float* s_red = s_sg + B.cap_pad;               // [kBW][kRed]
    ff* s_cs = reinterpret_cast<ff*>(s_red + kBW * kRed);  // [kMaxGrp][NCS]
    ff* s_q = s_cs + kMaxGrp * NCS;                // [NQ SL + NCS]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    for (int i = tid; i < (int)(sizeof(Coefs) / 4); i += kBT)
        reinterpret_cast<int*>(&CF)[i] = reinterpret_cast<const int*>(B.coefs)[i];

    // the problem's parameters and phase machine into shared memory
    auto load_prob = [&](int p) {
        __syncthreads();
        const int* src = reinterpret_cast<const int*>(B.probs + p);
        for (int i = tid; i < (int)(sizeof(KParams) / 4); i += kBT) reinterpret_cast<int*>(&sP)[i] = src[i];
        __syncthreads();
        if (tid == 0) {
            sP.mode = B.mode;
            sH = *sP.hyper;
            set_step_scalars(sH, sP.d, s_eps, s_c1, s_c2s);
        }
        __syncthreads();
    };

    unsigned n_bar = 0;
    const int n_iter = B.mode == 0 ? 1 : B.n_iters;
    for (int it = 0; it < n_iter; ++it) {
        if (tid == 0) {
            int live = 0;
            for (int p = 0; p < B.n; ++p) live |= (B.mode == 0 || !B.probs[p].hyper->done) ? 1 : 0;
            // a latched error ends the launch (a replayed graph launch after a failure is empty)
            if (*reinterpret_cast<volatile int*>(B.status) != ST_OK) live = 0;
            s_live = live;
        }
        __syncthreads();
        if (!s_live) break;  // uniform: every block reads the same phase machines
        // ------------------------------------------------ 1. chain phase
        for (int p = 0; p < B.n; ++p) {
            const int2 sc = B.sched[p];  // the same for every thread: a uniform branch
            const int slot = b - sc.x;
            if (slot < 0 || slot >= sc.y) continue;
            load_prob(p);
            if (B.mode == 1 && sH.done) continue;
            const KParams& P = sP;
            for (int i = tid; i < P.d_pad; i += kBT) {
                const float sg = P.sigma[i];
                s_c[i] = i < P.d ? P.prec[i] * (sg * sg) : 0.0f;
                s_sg[i] = sg;
            }
            // lanes per chain: 4, 8 or 16 (several chains share a warp) or a multiple of 32
            const int Lp = B.gw[p], ng = kBT / Lp;
            Grp Gc;
            if (Lp >= 32) {
                const int gw = Lp / 32;
                Gc = Grp{gw, warp / gw, warp % gw, (warp % gw) * 32 + lane, Lp, s_red + (warp / gw) * kRed, 0};
            } else {
                Gc = Grp{1, warp * (32 / Lp) + lane / Lp, 0, lane % Lp, Lp, nullptr, 0};
            }
            const int cap = Gc.lpc * CPL;
            // this thread's column slots, one float4 per coordinate block (conflict-free)
            float4* q0 = reinterpret_cast<float4*>(qbuf + (size_t)(0 * ng + Gc.grp) * cap);
            float4* q1 = reinterpret_cast<float4*>(qbuf + (size_t)(1 * ng + Gc.grp) * cap);
            const float4* s_c4 = reinterpret_cast<const float4*>(s_c);
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int j = Gc.gl + Gc.lpc * k;
                q0[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                q1[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            ff cs[NCS];
#pragma unroll
            for (int k = 0; k < NCS; ++k) cs[k] = ff_make(0.0f);
            __syncthreads();
            const float eps = s_eps, c1 = s_c1, c2s = s_c2s;
            const float dm1 = (float)(P.d - 1), inv_dm1 = 1.0f / (float)(P.d - 1);
            const bool pend = (B.mode == 1 && sH.phase == 1 && sH.p == 0);  // y still in x (switch)
            const int64_t m0 = (int64_t)slot * P.M / sc.y, m1 = (int64_t)(slot + 1) * P.M / sc.y;
            // the same number of rounds for every group of the block (the groups of a
            // warp share its shuffles); a group past its share's last chain runs on
            // zeros and writes nothing
            for (int64_t base = m0; base < m1; base += ng) {
                const int64_t mm = base + Gc.grp;
                const bool act = mm < m1;
                const uint32_t m = (uint32_t)mm;
                // unadjusted phase: the next round's rows of y and u into L2 while this
                // round's single step runs (one bulk prefetch per row from the group's
                // first lane; a hint, no wait).  A MAMS round is long enough without it.
                if (B.mode == 1 && sH.phase == 0 && Gc.gl == 0 && mm + ng < m1) {
                    const size_t row = (size_t)(mm + ng) * P.d_pad;
                    l2_prefetch(P.y + row, (uint32_t)P.d_pad * 4u);
                    l2_prefetch(P.u + row, (uint32_t)P.d_pad * 4u);
                }
                float y[CPL], u[CPL];
                auto load = [&](const float* src, float(&v)[CPL]) {
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        const int j = Gc.gl + Gc.lpc * k;
                        float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (act && j < P.nblk) a = *reinterpret_cast<const float4*>(src + (size_t)mm * P.d_pad + 4 * j);
                        v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
                    }
                };
                auto store = [&](float* dst, const float(&v)[CPL]) {
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        const int j = Gc.gl + Gc.lpc * k;
                        if (act && j < P.nblk)
                            *reinterpret_cast<float4*>(dst + (size_t)mm * P.d_pad + 4 * j) =
                                make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    }
                };
                if (B.mode == 0) {
                    // Alg. 1 input and App. C "Initialization"
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        const int j = Gc.gl + Gc.lpc * k;
                        float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                        if (j < P.nblk && P.x0 == nullptr)
                            normals4(j, m, 0u, TAG_X0 | (P.pid << 8), B.keys, z);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int i = 4 * j + c;
                            y[4 * k + c] = (act && j < P.nblk && i < P.d)
                                               ? (P.x0 ? P.x0[(size_t)mm * P.d + i] : P.x0_scale * z[c])
                                               : 0.0f;
                        }
                    }
                    float n2 = 0.0f;
                    bool bad = false;
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        float g[4];
                        g_blk<CPL>(Gc, P, y, k, s_c4, g);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            n2 = fmaf(g[c], g[c], n2);
                            bad = bad || !(isfinite(y[4 * k + c]) && isfinite(g[c]));
                        }
                    }
                    n2 = gsum1(Gc, n2);
#pragma unroll
                    for (int q = 0; q < CPL; ++q) u[q] = 0.0f;
                    g_o<CPL>(P, B.keys, Gc, m, 0xFFFFFFFFu, TAG_O1, 0.0f, 1.0f, u);
                    if (n2 > 0.0f) {
                        const float inv = 1.0f / sqrtf(n2);
#pragma unroll
                        for (int k = 0; k < NB; ++k) {
                            float g[4];
                            g_blk<CPL>(Gc, P, y, k, s_c4, g);
#pragma unroll
                            for (int c = 0; c < 4; ++c) u[4 * k + c] = g[c] * inv;
                        }
                    }
                    if (bad && act) atomicCAS(P.status, ST_OK, ST_NONFINITE);
                    store(P.y, y);
                    store(P.u, u);
                } else {
                    load(P.y, y);
                    load(P.u, u);
                    if (pend)  // Sec. 4: the preconditioner fixed at the switch, y = x / sigma
#pragma unroll
                        for (int k = 0; k < NB; ++k) {
                            const int j = Gc.gl + Gc.lpc * k;
                            if (j < P.nblk)
#pragma unroll
                                for (int c = 0; c < 4; ++c) y[4 * k + c] = y[4 * k + c] / s_sg[4 * j + c];
                        }
                    ff dl = ff_make(0.0f), dlA = ff_make(0.0f);
                    const int integ = sH.phase == 0 ? INTEG_LF : sH.integ;
                    bool bad = false;
                    if (sH.phase == 0) {
                        g_step<CPL>(P, B.keys, Gc, CF, integ, eps, c1, c2s, m, (uint32_t)sH.t, y, u, dl, dlA, inv_dm1, dm1,
                                    s_c4, true, bad);
                    } else {
                        // App. F step 2: u uniform on the sphere, then N steps
                        float n2 = 0.0f;
#pragma unroll
                        for (int k = 0; k < NB; ++k) {
                            const int j = Gc.gl + Gc.lpc * k;
                            float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                            if (j < P.nblk)
                                normals4(j, m, (uint32_t)sH.p, TAG_REFRESH | (P.pid << 8), B.keys, z);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float v = (4 * j + c < P.d) ? z[c] : 0.0f;
                                u[4 * k + c] = v;
                                n2 = fmaf(v, v, n2);
                            }
                        }
                        n2 = gsum1(Gc, n2);
                        const float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
#pragma unroll
                        for (int q = 0; q < CPL; ++q) u[q] *= inv;
                        const uint32_t t0 = (uint32_t)sH.t;
                        for (int n = 0; n < P.N; ++n)
                            g_step<CPL>(P, B.keys, Gc, CF, integ, eps, c1, c2s, m, t0 + n, y, u, dl, dlA, inv_dm1, dm1, s_c4,
                                        n == P.N - 1, bad);
                    }
                    bool keep = !bad;
                    float a_m = 0.0f;
                    if (sH.phase == 1) {
                        // App. F step 5: accept with probability min(1, e^-Delta)
                        const uint4 r = philox4x32_10(
                            make_uint4(0u, m, (uint32_t)sH.p, TAG_MH | (P.pid << 8)), B.keys);
                        const ff s = ff_add(dl, logf(u01(r.x)));
                        keep = !bad && (s.hi < 0.0f || (s.hi == 0.0f && s.lo < 0.0f));
                        a_m = bad ? 0.0f : (dl.hi <= 0.0f ? 1.0f : expf(-(dl.hi + dl.lo)));
                    }
                    if (keep) {
                        store(P.y, y);
                        store(P.u, u);
                    } else {
                        load(P.y, y);  // the accepted state stays and enters the sums
                        if (pend)
#pragma unroll
                            for (int k = 0; k < NB; ++k) {
                                const int j = Gc.gl + Gc.lpc * k;
                                if (j < P.nblk)
#pragma unroll
                                    for (int c = 0; c < 4; ++c) y[4 * k + c] = y[4 * k + c] / s_sg[4 * j + c];
                            }
                        if (pend) store(P.y, y);  // keep the accepted point in the new coordinates
                    }
                    if (!act) {
                    } else if (sH.phase == 0) {
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
                // per-coordinate sums of y and y^2 (this thread's own slots)
                if (act)
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const int j = Gc.gl + Gc.lpc * k;
                    float4 a = q0[j], s = q1[j];
                    const float* v = y + 4 * k;
                    a.x += v[0]; a.y += v[1]; a.z += v[2]; a.w += v[3];
                    s.x = fmaf(v[0], v[0], s.x); s.y = fmaf(v[1], v[1], s.y);
                    s.z = fmaf(v[2], v[2], s.z); s.w = fmaf(v[3], v[3], s.w);
                    q0[j] = a;
                    q1[j] = s;
                }
            }
            if (Gc.gl == 0)
#pragma unroll
                for (int k = 0; k < NCS; ++k) s_cs[Gc.grp * NCS + k] = cs[k];
            __syncthreads();
            // this block's column of the problem: groups in order, float-float
            const int G2 = P.G, dp = P.d_pad;
            for (int i = tid; i < P.d; i += kBT)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float* src = qbuf + (size_t)q * ng * cap + i;
                    ff s = ff_make(src[0]);
                    for (int gg = 1; gg < ng; ++gg) s = ff_add(s, src[(size_t)gg * cap]);
                    P.part[((size_t)q * dp + i) * G2 + slot] = make_float2(s.hi, s.lo);
                }
            if (tid < NCS) {
                ff s = s_cs[tid];
                for (int gg = 1; gg < ng; ++gg) s = ff_add(s, s_cs[gg * NCS + tid]);
                P.part[((size_t)NQ * dp + tid) * G2 + slot] = make_float2(s.hi, s.lo);
            }
        }
        // ------------------------------------------------ 2. slices
        n_bar += 1;
        if (!grid_sync_count(B.bar_count, B.status, n_bar * (unsigned)(G + B.bar_extra), B.timeout_ns)) return;
        {
            int task = 0;
            for (int p = 0; p < B.n; ++p) {
                const int d = B.probs[p].d;
                const int nsl = (d + B.SL - 1) / B.SL;
                for (int s = 0; s < nsl; ++s, ++task) {
                    if (task % G != b) continue;
                    load_prob(p);
                    if (B.mode == 1 && sH.done) continue;
                    ens_slice(sP, sH, s_q, s, nsl);
                }
            }
        }
        // ------------------------------------------------ 3. finalise per problem
        n_bar += 1;
        if (!grid_sync_count(B.bar_count, B.status, n_bar * (unsigned)(G + B.bar_extra), B.timeout_ns)) return;
        for (int p = b; p < B.n; p += G) {
            load_prob(p);
            if (B.mode == 1 && sH.done) continue;
            ens_gather(sP, sH, qbuf, FS);
            if (tid == 0) {
                *sP.hyper = sH;
                ens_trace_row(sP, sH, FS.now);
            }
            if (FS.sw)  // Sec. 4: the diagonal preconditioner, applied to y at the next load
                for (int i = tid; i < sP.d; i += kBT) {
                    const float v = qbuf[i];
                    sP.sigma[i] = v > 0.0f ? sqrtf(v) : 1.0f;
                }
        }
        n_bar += 1;
        if (!grid_sync_count(B.bar_count, B.status, n_bar * (unsigned)(G + B.bar_extra), B.timeout_ns)) return;
    }
}

// ---------------------------------------------------------------- host
const void* batch_fn(int cpl) {
    switch (cpl) {
    case 8: return (const void*)batch_kernel<8>;
    case 12: return (const void*)batch_kernel<12>;
    case 16: return (const void*)batch_kernel<16>;
    case 20: return (const void*)batch_kernel<20>;
    }
    return nullptr;
}

size_t batch_smem(int cpl, int cap_pad, int SL) {
    return (size_t)2 * kBT * cpl * 4 + (size_t)2 * cap_pad * 4 + (size_t)kBW * kRed * 4 +
           (size_t)kMaxGrp * NCS * sizeof(ff) + ((size_t)NQ * SL + NCS) * sizeof(ff);
}

int batch_threads() { return kBT; }

// lanes per chain for dimension d with cpl coordinates per lane: the fewest of
// 4, 8, 16, 32, 64, ..., 512 that hold d (a chain of small d shares a warp with
// others, a chain of large d spans warps), doubled `widen` times; 0 if none does
int batch_gw(int64_t d, int cpl, int widen) {
    const int64_t dp = ((d + 3) / 4) * 4;
    int L = 4;
    while ((int64_t)L * cpl < dp && L < kBT) L *= 2;
    if ((int64_t)L * cpl < dp) return 0;
    for (int k = 0; k < widen && L < kBT; ++k) L *= 2;
    return L;
}

cudaError_t batch_launch(int cpl, int G, const KParams* probs, const int* gw, const int2* sched,
                         const Coefs* coefs, int n, int mode, int n_iters, int SL, int cap_pad, unsigned* bar,
                         int* status, long long timeout_ns, int bar_extra, uint64_t seed, cudaStream_t st) {
    BatchArgs a;
    a.keys = philox_keys((uint32_t)seed, (uint32_t)(seed >> 32));
    a.probs = probs;
    a.gw = gw;
    a.sched = sched;
    a.coefs = coefs;
    a.n = n;
    a.mode = mode;
    a.n_iters = n_iters;
    a.SL = SL;
    a.cap_pad = cap_pad;
    a.bar_count = bar;
    a.status = status;
    a.timeout_ns = timeout_ns;
    a.bar_extra = bar_extra;
    const void* fn = batch_fn(cpl);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = batch_smem(cpl, cap_pad, SL);
    cudaError_t e = ensure_dyn_smem(fn, smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone)
        return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBT), args, smem, st);
    // inside a stream capture: the launch-attribute form records a cooperative kernel node
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// A block runs one problem at a time with all its ng = 512 / L chain groups of
// L lanes; a round (ng chains side by side) costs about ceil(nblk / L) passes
// over the lanes' coordinate blocks whatever L is, so that is a problem's cost
// per round.  A problem with at least ng chains per block is spread over every
// block (rounds = ceil(ceil(M / G) / ng) each).  Any other problem gets
// ceil(M / ng) blocks, one round each, at the place where the most loaded of
// those blocks carries the least work so far (larger problems placed first).
void batch_schedule(const int64_t* d, const int64_t* M, int n, int cpl, int widen, int G, int2* sched) {
    std::vector<double> load(G, 0.0);
    std::vector<int> order;
    auto cost = [&](int k, int& ng) {
        const int L = std::max(batch_gw(d[k], cpl, widen), 4);  // lanes per chain
        ng = kBT / L;
        const int64_t nblk = (d[k] + 3) / 4;
        return (double)((nblk + L - 1) / L);
    };
    for (int k = 0; k < n; ++k) {
        int ng = 1;
        const double c = cost(k, ng);
        if (M[k] >= (int64_t)G * ng) {
            sched[k] = make_int2(0, G);
            const double rounds = (double)((((M[k] + G - 1) / G) + ng - 1) / ng);
            for (int b = 0; b < G; ++b) load[b] += rounds * c;
        } else {
            order.push_back(k);
        }
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        int na = 1, nb = 1;
        const double ca = cost(a, na), cb = cost(b, nb);
        return ca * (double)((M[a] + na - 1) / na) > cb * (double)((M[b] + nb - 1) / nb);
    });
    for (int k : order) {
        int ng = 1;
        const double c = cost(k, ng);
        const int nb = (int)std::min<int64_t>(G, std::max<int64_t>(1, (M[k] + ng - 1) / ng));
        int best = 0;
        double best_max = 1e300;
        for (int b0 = 0; b0 + nb <= G; ++b0) {
            double mx = 0.0;
            for (int b = b0; b < b0 + nb; ++b) mx = std::max(mx, load[b]);
            if (mx < best_max) {
                best_max = mx;
                best = b0;
            }
        }
        sched[k] = make_int2(best, nb);
        for (int b = best; b < best + nb; ++b) load[b] += c;
    }
}

int batch_blocks_per_sm(int cpl, int cap_pad, int SL) {
    const void* fn = batch_fn(cpl);
    const size_t smem = batch_smem(cpl, cap_pad, SL);
    if (!fn || ensure_dyn_smem(fn, smem) != cudaSuccess)
        return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBT, smem) != cudaSuccess) return 0;
    return bps;
}

}  // namespace laps
