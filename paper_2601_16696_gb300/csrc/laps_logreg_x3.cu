// laps_logreg_x3.cu -- the logistic-regression ensemble gradient at FP32
// accuracy on the 5th-generation tensor cores: every FP32 operand is split
// into three BF16 terms, v = v0 + v1 + v2 (exact for normal-range binary32:
// 8 + 8 + 8 significand bits), and of the nine cross products the six of
// order <= 2^-16 are formed (v_i w_j with i + j <= 2); the three dropped ones
// are of order 2^-24 relative, the rounding unit of binary32.  This is the
// split-precision technique of Henry, Tang and Heinecke (ARITH 2019), here
// with FP32 accumulation in tensor memory.
//
// A CTA owns 128 chains (one MMA M tile) and one range of data rows, walked
// in chunks of 64 rows:
//   Z_c  = sum_{i+j<=2} W_i X_{c,j}^T     128 x 64 (TMEM)
//   R_c  = y_c - sigmoid(Z_c)             FP32 epilogue, split into R_0 + R_1 + R_2
//   G   += sum_{i+j<=2} R_{c,i} X_{c,j}   128 x kp, 6 products of K = 64 (TMEM)
// A tensor-core instruction costs about the same whether its N is 64 or 128,
// so the Z products are issued as three wide ones per K step: the chunk's
// three X terms lie one after another along N, and W_0 [X_0; X_1; X_2]
// (N = 192), W_1 [X_0; X_1] (N = 128) and W_2 X_0 (N = 64) accumulate into
// three 64-column blocks whose sum, formed by the epilogue, is Z_c.  The
// tensor cores round each accumulation toward zero relative to the running
// sum, so the products go smallest first (W_2 X_0, then W_1 [...], then
// W_0 [...]; for G likewise): the small ones accumulate at their own scale.
// The epilogue clears the Z blocks after reading them, so that every Z product
// accumulates and the order is free.
//
// Storage: the three terms of the points W live in tensor memory (the A
// operand of the Z products; one chain per lane, two BF16 per column), so
// shared memory holds only the data ring and the residual buffers.  One copy
// of each X chunk, laid out [feature atom][term][64 rows][128 bytes], serves
// both contractions: K-major as the B operand of Z, MN-major as the B operand
// of G.
//
// Roles (640 threads): warp 0 streams the three terms of each X chunk with
// TMA (128-byte swizzle); warp 1 issues the MMAs from one thread; warps 4..19
// write the points' terms into tensor memory, then run the epilogue (warp w
// reads TMEM lanes 32 (w % 4) .. +31, i.e. chains, and a quarter of the
// columns).  All waits are bounded: on expiry the CTA records ST_TIMEOUT in
// the status word, drains what it issued and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "laps_device.cuh"
#include "laps_logreg.cuh"
#include "laps_tc.cuh"

namespace laps {

namespace {

using namespace tc;

constexpr int MT = 128;       // chains per CTA (MMA M)
constexpr int TNR = 64;       // data rows per chunk (MMA N of Z, K of G)
constexpr int NTHR = 640;
constexpr int EPI_WARP0 = 4;  // first epilogue warp
constexpr int NEPI = 16;      // epilogue warps: 4 lane quarters x 4 column quarters

// the six products of G (term of R, term of X), smallest first
__device__ constexpr int kPairA[6] = {0, 1, 2, 0, 1, 0};
__device__ constexpr int kPairX[6] = {2, 1, 0, 1, 0, 0};

struct X3Args {
    int64_t M;           // chains
    int n;               // data rows
    int n_pad;           // rows of one term of the split data
    int rps;             // rows per split, a multiple of 64
    float inv_v;         // 1 / prior variance
    const float* W32;    // [M][kp] FP32 points
    const float* y;      // [n] labels
    float* gpart;        // [S][M][kp]
    float2* lpart;       // [S][M]
    int* status;
    long long timeout_ns;
    const int* guard;    // nullable: 0 there means the iteration no longer runs
};

template <int KP>
struct SmemX3 {
    static constexpr int NA = KP / 64;                          // 64-wide feature atoms
    // X ring depth and residual buffers: three stages keep the next chunk's
    // load ahead of the tensor pipe; at kp = 128 that leaves room for one
    // residual buffer (its writer waits for the previous G products instead)
    static constexpr int NST = KP == 64 ? 4 : 3;
    static constexpr int NRB = KP == 64 ? 2 : 1;
    static constexpr uint32_t TERM = (uint32_t)TNR * 128;       // one term of one feature atom
    static constexpr uint32_t ATOM = 3 * TERM;                  // the three terms of one atom
    static constexpr uint32_t STAGE = NA * ATOM;
    static constexpr uint32_t RTERM = MT * 128;                 // one term of R: 128 chains x 64 rows
    static constexpr uint32_t RBUF = 3 * RTERM;
    static constexpr uint32_t OFF_X = 0;
    static constexpr uint32_t OFF_R = OFF_X + NST * STAGE;
    static constexpr uint32_t OFF_BAR = OFF_R + NRB * RBUF;
    static constexpr uint32_t OFF_LP = OFF_BAR + 256;           // [4][MT] float-float
    static constexpr uint32_t TOTAL = OFF_LP + 4 * MT * 8 + 1024;  // + alignment slack
    // tensor memory: the Z blocks [0, 192), G [192, 192 + KP), W terms [320, 320 + 3 KP / 2)
    static constexpr uint32_t T_G = 3 * TNR, T_W = 320, TMEM_COLS = 512;
    static_assert(T_G + KP <= T_W && T_W + 3 * KP / 2 <= TMEM_COLS, "tensor memory columns");
    static_assert(TOTAL <= 227 * 1024, "shared memory");
};

template <int KP>
struct Bars {
    static constexpr int NST = SmemX3<KP>::NST, NRB = SmemX3<KP>::NRB;
    static constexpr int WFULL = 0, XFULL = 1, XEMPTY = XFULL + NST, ZFULL = XEMPTY + NST,
                         ZEMPTY = ZFULL + 1, RFULL = ZEMPTY + 1, REMPTY = RFULL + NRB, GDONE = REMPTY + NRB,
                         DRAIN = GDONE + 1, N = DRAIN + 1;
    static_assert(N * 8 <= 256, "barrier space");
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
// v = t0 + t1 + t2 in BF16 (each remainder is exact in binary32)
__device__ __forceinline__ void split3(float v, __nv_bfloat16& t0, __nv_bfloat16& t1, __nv_bfloat16& t2) {
    t0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(t0);
    t1 = __float2bfloat16_rn(r1);
    t2 = __float2bfloat16_rn(r1 - __bfloat162float(t1));
}
__device__ constexpr uint32_t kZero16[16] = {};
__device__ __forceinline__ uint32_t bits2(__nv_bfloat162 h) { return *reinterpret_cast<const uint32_t*>(&h); }
// the same for a pair (a, b): packed terms, a in the low half
__device__ __forceinline__ void split3x2(float a, float b, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b);
    const float2 f0 = __bfloat1622float2(h0);
    const float ra = a - f0.x, rb = b - f0.y;
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(ra, rb);
    const float2 f1 = __bfloat1622float2(h1);
    p0 = bits2(h0);
    p1 = bits2(h1);
    p2 = bits2(__floats2bfloat162_rn(ra - f1.x, rb - f1.y));
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int KP>
__global__ void __launch_bounds__(NTHR, 1)
logreg_grad_x3_kernel(const __grid_constant__ CUtensorMap tmX3, const X3Args A) {
    if (A.guard != nullptr && *A.guard == 0) return;  // uniform: before any barrier or allocation
    using S = SmemX3<KP>;
    using B = Bars<KP>;
    constexpr int NST = S::NST, NRB = S::NRB;
    extern __shared__ __align__(1024) unsigned char x3_smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const uint32_t raw = smem_u32(x3_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned for the swizzle atoms
    unsigned char* gbase = x3_smem_raw + (base - raw);
    const uint32_t sX = base + S::OFF_X, sR = base + S::OFF_R;
    const uint32_t bars = base + S::OFF_BAR;
    ff* s_lp = reinterpret_cast<ff*>(gbase + S::OFF_LP);
    auto bar = [&](int k) { return bars + 8u * (uint32_t)k; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * MT;
    const int split = blockIdx.y;
    const int r_begin = split * A.rps;
    const int r_end = min(A.n, r_begin + A.rps);
    const int nc = r_end > r_begin ? (r_end - r_begin + TNR - 1) / TNR : 0;
    const unsigned long long deadline = global_ns() + (unsigned long long)A.timeout_ns;

    if (tid == 32) {
        mbar_init(bar(B::WFULL), NEPI);
        for (int s = 0; s < NST; ++s) {
            mbar_init(bar(B::XFULL + s), 1);
            mbar_init(bar(B::XEMPTY + s), 1);
        }
        mbar_init(bar(B::ZFULL), 1);
        mbar_init(bar(B::ZEMPTY), NEPI);
        for (int b = 0; b < NRB; ++b) {
            mbar_init(bar(B::RFULL + b), NEPI);
            mbar_init(bar(B::REMPTY + b), 1);
        }
        mbar_init(bar(B::GDONE), 1);
        mbar_init(bar(B::DRAIN), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tZ = tmem, tG = tmem + S::T_G, tW = tmem + S::T_W;

    if (warp == 0) {
      if (lane == 0) {
        // ------------------------------------------------ TMA producer: the three terms of each chunk
        bool ok = true;
        int issued = 0;
        for (int c = 0; c < nc && ok; ++c) {
            const int st = c % NST;
            if (!mbar_wait(bar(B::XEMPTY + st), ((c / NST) & 1) ^ 1, deadline)) { ok = false; break; }
            const uint32_t dst = sX + (uint32_t)st * S::STAGE;
            mbar_expect_tx(bar(B::XFULL + st), S::STAGE);
            const int row = r_begin + c * TNR;
            for (int a = 0; a < S::NA; ++a)
                for (int t = 0; t < 3; ++t)
                    tma_load_2d(dst + (uint32_t)a * S::ATOM + (uint32_t)t * S::TERM, &tmX3, 64 * a,
                                t * A.n_pad + row, bar(B::XFULL + st));
            issued = c + 1;
        }
        if (!ok) {
            atomicExch(&s_fail, 1);
            // wait (bounded) for the copies this thread issued
            const unsigned long long d2 = global_ns() + drain_ns(A.timeout_ns);
            for (int c = max(0, issued - NST); c < issued; ++c)
                mbar_wait(bar(B::XFULL + c % NST), (c / NST) & 1, d2);
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      if (lane == 0) {
        // ------------------------------------------------ MMA issuer
        constexpr uint32_t ID_G = idesc_bf16(MT, KP, true);
        // descriptors at the ring's base; an operand's descriptor is its base's
        // plus its byte offset / 16 (the start-address field, 14 bits, cannot
        // carry: shared-memory offsets stay below 256 KB)
        const uint64_t dX = sw128_desc(sX), dXmn = sw128_mn_desc(sX, S::ATOM), dR = sw128_desc(sR);
        bool ok = mbar_wait(bar(B::WFULL), 0, deadline);
        tc_fence_after();
        auto gemm2 = [&](int cc) -> bool {
            const int rb = cc % NRB, st = cc % NST;
            if (!mbar_wait(bar(B::RFULL + rb), (cc / NRB) & 1, deadline)) return false;
            tc_fence_after();
            const uint64_t aR = dR + (uint64_t)((uint32_t)rb * S::RBUF >> 4);
            const uint64_t bX = dXmn + (uint64_t)((uint32_t)st * S::STAGE >> 4);
#pragma unroll
            for (int p = 0; p < 6; ++p)
#pragma unroll
                for (int kk = 0; kk < TNR / 16; ++kk)
                    tc_mma(tG, aR + (((uint32_t)kPairA[p] * S::RTERM + 32u * kk) >> 4),
                           bX + (((uint32_t)kPairX[p] * S::TERM + 2048u * kk) >> 4), ID_G,
                           (cc > 0 || p > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bar(B::REMPTY + rb));
            tc_commit(bar(B::XEMPTY + st));
            return true;
        };
        constexpr uint32_t ID_Z3 = idesc_bf16(MT, 3 * TNR), ID_Z2 = idesc_bf16(MT, 2 * TNR),
                           ID_Z1 = idesc_bf16(MT, TNR);
        for (int c = 0; c <= nc && ok; ++c) {
            if (c < nc) {
                const int st = c % NST;
                if (!mbar_wait(bar(B::XFULL + st), (c / NST) & 1, deadline) ||
                    !mbar_wait(bar(B::ZEMPTY), (c & 1) ^ 1, deadline)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t bX = dX + (uint64_t)((uint32_t)st * S::STAGE >> 4);
                // rows of X_0, X_1, X_2 follow one another along N; the blocks
                // were cleared by the epilogue, so every product accumulates
#pragma unroll
                for (int kk = 0; kk < KP / 16; ++kk)
                    tc_mma_ts(tZ, tW + (uint32_t)KP + 8u * kk,
                              bX + (((uint32_t)(kk / 4) * S::ATOM + 32u * (kk % 4)) >> 4), ID_Z1, 1u);
#pragma unroll
                for (int kk = 0; kk < KP / 16; ++kk)
                    tc_mma_ts(tZ, tW + (uint32_t)(KP / 2) + 8u * kk,
                              bX + (((uint32_t)(kk / 4) * S::ATOM + 32u * (kk % 4)) >> 4), ID_Z2, 1u);
#pragma unroll
                for (int kk = 0; kk < KP / 16; ++kk)
                    tc_mma_ts(tZ, tW + 8u * kk,
                              bX + (((uint32_t)(kk / 4) * S::ATOM + 32u * (kk % 4)) >> 4), ID_Z3, 1u);
                tc_commit(bar(B::ZFULL));
            }
            if (c >= 1 && !gemm2(c - 1)) { ok = false; break; }
        }
        if (ok) {
            tc_commit(bar(B::GDONE));
        } else {
            atomicExch(&s_fail, 1);
            tc_commit(bar(B::DRAIN));  // everything issued so far has completed once this arrives
            mbar_wait(bar(B::DRAIN), 0, global_ns() + drain_ns(A.timeout_ns));
        }
      }
      __syncwarp();
    } else if (warp >= EPI_WARP0 && warp < EPI_WARP0 + NEPI) {
        // ------------------------------------------------ points into tensor memory, then the epilogue
        constexpr int FH = KP / 4;  // features of one column quarter
        constexpr int CH = FH / 2;  // TMEM columns of one term in one column quarter
        const int q = warp & 3;                 // TMEM lane quarter: chains 32q .. 32q+31
        const int h = (warp - EPI_WARP0) >> 2;  // column quarter
        const int rt = 32 * q + lane;           // this thread's chain in the tile
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        const int64_t m = m0 + rt;
        {
            float wv[FH];
            if (m < A.M) {
                const float4* src = reinterpret_cast<const float4*>(A.W32 + (size_t)m * KP + h * FH);
#pragma unroll
                for (int j4 = 0; j4 < FH / 4; ++j4) {
                    const float4 v = src[j4];
                    wv[4 * j4] = v.x; wv[4 * j4 + 1] = v.y; wv[4 * j4 + 2] = v.z; wv[4 * j4 + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < FH; ++j) wv[j] = 0.0f;
            }
            uint32_t pk[3][CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                __nv_bfloat16 a0, a1, a2, b0, b1, b2;
                split3(wv[2 * c], a0, a1, a2);
                split3(wv[2 * c + 1], b0, b1, b2);
                pk[0][c] = pack2(a0, b0);
                pk[1][c] = pack2(a1, b1);
                pk[2][c] = pack2(a2, b2);
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const uint32_t ta = tW + lane_off + (uint32_t)(t * (KP / 2) + h * CH);
                if constexpr (CH == 16) tmem_st16(ta, pk[t]);
                else tmem_st8(ta, pk[t]);
            }
#pragma unroll
            for (int b = 0; b < 3; ++b) tmem_st16(tZ + lane_off + (uint32_t)(b * TNR + 16 * h), kZero16);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B::WFULL));
        }
        ff lp = ff_make(0.0f);
        bool ok = true;
        for (int c = 0; c < nc; ++c) {
            // the labels of data rows row0 .. row0 + 15, loaded before waiting for Z
            const int row0 = r_begin + c * TNR + 16 * h;
            const int nlive = min(16, r_end - row0);
            float yy[16];
            if (nlive >= 16) {
#pragma unroll
                for (int j4 = 0; j4 < 4; ++j4) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(A.y + row0) + j4);
                    yy[4 * j4] = v.x; yy[4 * j4 + 1] = v.y; yy[4 * j4 + 2] = v.z; yy[4 * j4 + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) yy[j] = j < nlive ? A.y[row0 + j] : 0.0f;
            }
            if (!mbar_wait(bar(B::ZFULL), c & 1, deadline)) { ok = false; break; }
            tc_fence_after();
            // Z = D_0 + (D_1 + D_2): the products with X_0, X_1 and X_2
            float z[16], z1[16], z2[16];
            tmem_ld16(tZ + lane_off + (uint32_t)(16 * h), z);
            tmem_ld16(tZ + lane_off + (uint32_t)(TNR + 16 * h), z1);
            tmem_ld16(tZ + lane_off + (uint32_t)(2 * TNR + 16 * h), z2);
#pragma unroll
            for (int b = 0; b < 3; ++b) tmem_st16(tZ + lane_off + (uint32_t)(b * TNR + 16 * h), kZero16);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B::ZEMPTY));
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] += z1[j] + z2[j];
            // residuals and log-likelihood terms in binary32: t = e^{-|z|}
            // (expf), sigmoid from 1 / (1 + t) by the hardware's approximate
            // reciprocal refined with one Newton-Raphson step (within about one
            // ulp; 1 + t lies in [1, 2]), softplus = max(z, 0) + ln 2 log2(1 + t).
            // Log p enters the Metropolis test only through sums of these terms,
            // so its per-row error is an absolute one: about 2^-22 from the
            // base-2 logarithm, next to the binary32 rounding of 1 + t itself.
            float r[16];
            float lsum = 0.0f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float zz = z[j];
                const float t = expf(-fabsf(zz));
                const float opt = 1.0f + t;
                float inv = rcp_approx(opt);
                inv = fmaf(inv, fmaf(-opt, inv, 1.0f), inv);
                const float sp = fmaf(0.6931471805599453f, lg2_approx(opt), fmaxf(zz, 0.0f));
                const float sig = zz >= 0.0f ? inv : t * inv;
                const bool live = j < nlive;
                r[j] = live ? yy[j] - sig : 0.0f;
                lsum += live ? fmaf(yy[j], zz, -sp) : 0.0f;
            }
            lp = ff_add(lp, lsum);
            const int rb = c % NRB;
            if (!mbar_wait(bar(B::REMPTY + rb), ((c / NRB) & 1) ^ 1, deadline)) { ok = false; break; }
            // the three terms of R row rt, 16-byte chunks 2h, 2h+1 of each 128-byte row, 128-byte swizzle
            unsigned char* rrow = gbase + S::OFF_R + (size_t)rb * S::RBUF + (size_t)rt * 128;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int chunk = (2 * h + i) ^ (rt & 7);
                uint32_t w[3][4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    split3x2(r[8 * i + 2 * e], r[8 * i + 2 * e + 1], w[0][e], w[1][e], w[2][e]);
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    *reinterpret_cast<uint4*>(rrow + (size_t)t * S::RTERM + 16 * chunk) =
                        make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B::RFULL + rb));
        }
        if (ok && !mbar_wait(bar(B::GDONE), 0, deadline)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        const float* wrow = A.W32 + (size_t)(m < A.M ? m : 0) * KP;
        if (!ok) atomicExch(&s_fail, 1);
        if (ok) {
            tc_fence_after();
            // G columns [h kp/4, (h+1) kp/4) of chain m, plus the prior on split 0
            float* gout = A.gpart + ((size_t)split * A.M + (m < A.M ? m : 0)) * KP;
#pragma unroll
            for (int piece = 0; piece < KP / 64; ++piece) {
                float g[16];
                const int col = h * (KP / 4) + 16 * piece;
                tmem_ld16(tG + lane_off + (uint32_t)col, g);
                if (nc == 0)
#pragma unroll
                    for (int k = 0; k < 16; ++k) g[k] = 0.0f;  // no chunk: G was never written
                if (m < A.M) {
#pragma unroll
                    for (int j4 = 0; j4 < 4; ++j4) {
                        float4 v = make_float4(g[4 * j4], g[4 * j4 + 1], g[4 * j4 + 2], g[4 * j4 + 3]);
                        if (split == 0) {
                            const float4 w = *reinterpret_cast<const float4*>(wrow + col + 4 * j4);
                            v.x = fmaf(-w.x, A.inv_v, v.x);
                            v.y = fmaf(-w.y, A.inv_v, v.y);
                            v.z = fmaf(-w.z, A.inv_v, v.z);
                            v.w = fmaf(-w.w, A.inv_v, v.w);
                        }
                        *reinterpret_cast<float4*>(gout + col + 4 * j4) = v;
                    }
                }
            }
            // log p: the four column quarters of a chain meet in shared memory
            s_lp[h * MT + rt] = lp;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NEPI * 32) : "memory");  // every epilogue warp
        if (ok) {
            if (h == 0 && m < A.M) {
                ff l = s_lp[rt];
#pragma unroll
                for (int k = 1; k < 4; ++k) l = ff_add(l, s_lp[k * MT + rt]);
                if (split == 0) {
                    float w2 = 0.0f;
                    for (int k = 0; k < KP; k += 4) {
                        const float4 w = *reinterpret_cast<const float4*>(wrow + k);
                        w2 = fmaf(w.x, w.x, fmaf(w.y, w.y, fmaf(w.z, w.z, fmaf(w.w, w.w, w2))));
                    }
                    l = ff_add(l, -0.5f * A.inv_v * w2);
                }
                A.lpart[(size_t)split * A.M + m] = make_float2(l.hi, l.lo);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail && tid == 0) atomicExch(A.status, ST_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS)
                     : "memory");
    }
}

// the data X [n][kp] (FP32) -> its three BF16 terms [3][n_pad][kp], rows past n zero
__global__ void split_data_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ X3, int n, int n_pad,
                                  int kp) {
    const int64_t tot = (int64_t)n_pad * kp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(k / kp);
        const float v = r < n ? X[k] : 0.0f;
        __nv_bfloat16 t0, t1, t2;
        split3(v, t0, t1, t2);
        X3[k] = t0;
        X3[tot + k] = t1;
        X3[2 * tot + k] = t2;
    }
}

template <int KP>
cudaError_t launch_x3(const LogregData& D, const X3Args& a, int S, cudaStream_t st) {
    using Sm = SmemX3<KP>;
    cudaError_t e = cudaFuncSetAttribute(logreg_grad_x3_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Sm::TOTAL);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((a.M + MT - 1) / MT), (unsigned)S);
    logreg_grad_x3_kernel<KP><<<grid, NTHR, Sm::TOTAL, st>>>(*reinterpret_cast<const CUtensorMap*>(D.tmX3), a);
    return cudaGetLastError();
}

}  // namespace

bool logreg_x3_supported(int kp) { return kp == 64 || kp == 128; }

cudaError_t logreg_x3_prepare(LogregData& D) {
    if (!logreg_x3_supported(D.kp)) return cudaErrorInvalidValue;
    D.n_pad = (D.n + TNR - 1) / TNR * TNR;
    const size_t nb = (size_t)3 * D.n_pad * D.kp * sizeof(__nv_bfloat16);
    cudaError_t e = cudaMalloc(&D.X3b, nb);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)D.n_pad * D.kp + 255) / 256);
    split_data_kernel<<<std::max(blocks, 1), 256>>>(D.X, reinterpret_cast<__nv_bfloat16*>(D.X3b), D.n, D.n_pad,
                                                    D.kp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // [3 n_pad][kp], boxes of 64 features x 64 rows
    if (!encode_bf16_2d(D.tmX3, D.X3b, (uint64_t)D.kp, (uint64_t)3 * D.n_pad, 64, TNR))
        return cudaErrorInvalidValue;
    return cudaDeviceSynchronize();
}

cudaError_t logreg_grad_x3(const LogregData& D, const float* W32, int64_t M, int S, int rps, float* gpart,
                           float2* lpart, int* status, long long timeout_ns, cudaStream_t st, const int* guard) {
    if (M <= 0) return cudaSuccess;
    if (D.X3b == nullptr) return cudaErrorInvalidValue;
    X3Args a;
    a.M = M;
    a.n = D.n;
    a.n_pad = D.n_pad;
    a.rps = rps;
    a.inv_v = D.inv_v;
    a.W32 = W32;
    a.y = D.y;
    a.gpart = gpart;
    a.lpart = lpart;
    a.status = status;
    a.timeout_ns = timeout_ns;
    a.guard = guard;
    if (D.kp == 64) return launch_x3<64>(D, a, S, st);
    if (D.kp == 128) return launch_x3<128>(D, a, S, st);
    return cudaErrorInvalidValue;
}

size_t logreg_x3_smem(int kp) { return kp == 64 ? SmemX3<64>::TOTAL : SmemX3<128>::TOTAL; }

// Data splits: about three waves of one CTA per SM.  The tensor cores round
// each accumulation into G toward zero, so the error of a G partial grows with
// the number of rows it sums; more, shorter splits (added in order in FP32 by
// the consumer) keep it at the FP32 form's level and use every SM.
int logreg_x3_splits(const LogregData& D, int64_t M, int nsm, int* rps_out) {
    const int64_t tiles = (M + MT - 1) / MT;
    int S = (int)std::max<int64_t>(1, 3 * (int64_t)nsm / std::max<int64_t>(1, tiles));
    const int chunks = (D.n + TNR - 1) / TNR;
    S = std::max(1, std::min(S, chunks));
    int rps = ((D.n + S - 1) / S + TNR - 1) / TNR * TNR;
    S = (D.n + rps - 1) / rps;
    if (rps_out) *rps_out = rps;
    return S;
}

}  // namespace laps
