// laps_logreg_mma.cu -- the logistic-regression ensemble gradient on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory), for the unadjusted phase of the mixed-precision form.
//
// A CTA owns 128 chains (one MMA M tile) and one range of data rows, which it
// walks in chunks of 64 rows:
//   Z_c  = [W_hi | W_lo] [X_c | X_c]^T     128 x 64, K = 2 kp   (TMEM, two buffers)
//   R_c  = y_c - sigmoid(Z_c)  (BF16, written into tensor memory by the epilogue)
//   G   += R_c X_c                          128 x kp, K = 64     (TMEM; R read from TMEM)
// W = x is split into two BF16 terms (hi + lo carries ~16 significant bits),
// so the logits are those of the BF16-rounded data at nearly FP32 accuracy in
// x and log p stays smooth along a trajectory; R is a single BF16 term.
//
// Roles (640 threads): warp 0 loads W once and X / X^T chunks through a
// 4-stage ring with TMA (128-byte swizzle); warp 1 issues the MMAs from one
// thread; warps 4..19 are the epilogue (warp w reads TMEM lanes 32 (w % 4) ..
// +31, i.e. chains, and a quarter of the columns).  All waits are bounded: on
// expiry the CTA records ST_TIMEOUT in the status word, drains what it
// issued and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "laps_device.cuh"
#include "laps_logreg.cuh"
#include "laps_tc.cuh"

namespace laps {

namespace {

constexpr int MT = 128;      // chains per CTA (MMA M)
constexpr int TNR = 64;      // data rows per chunk (MMA N of Z, K of G)
constexpr int NSTAGE = 4;    // X / X^T ring depth
constexpr int NTHR = 640;
constexpr int EPI_WARP0 = 4;  // first epilogue warp
constexpr int NEPI = 16;      // epilogue warps: 4 lane quarters x 4 column quarters

using namespace tc;

// SFU approximations in their flush-to-zero forms (the epilogue's arguments
// are never subnormal: 1 + t lies in [1, 2]; e^{-|z|} below 2^-126 flushes to 0)
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_ftz(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_ftz(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

struct MmaArgs {
    int64_t M;           // chains
    int n;               // data rows
    int rps;             // rows per split, a multiple of 64
    float inv_v;         // 1 / prior variance
    const float* W32;    // [M][kp] FP32 x (for the prior terms)
    const float* y;      // [n] labels
    float* gpart;        // [S][M][kp]
    float2* lpart;       // [S][M]
    int* status;
    long long timeout_ns;
    const int* guard;    // nullable: 0 there means the iteration no longer runs
};

template <int KP>
struct Smem {
    static constexpr int NA = KP / 64;                    // 64-wide K atoms of one W term
    static constexpr uint32_t W_BYTES = 2u * NA * MT * 128;  // hi and lo
    static constexpr uint32_t X_BYTES = (uint32_t)NA * TNR * 128;
    static constexpr uint32_t XT_BYTES = (uint32_t)KP * 128;
    static constexpr uint32_t STAGE = X_BYTES + XT_BYTES;
    static constexpr uint32_t OFF_W = 0;
    static constexpr uint32_t OFF_X = OFF_W + W_BYTES;
    static constexpr uint32_t OFF_BAR = OFF_X + NSTAGE * STAGE;
    static constexpr uint32_t OFF_LP = OFF_BAR + 256;      // [4][MT] float-float
    static constexpr uint32_t TOTAL = OFF_LP + 4 * MT * 8 + 1024;  // + alignment slack
    // tensor memory: Z buffers [0, 128), G [128, 128 + kp), R buffers (64 BF16 rows
    // per chain = 32 columns each) after G
    static constexpr uint32_t T_R = 2 * TNR + KP, TMEM_COLS = T_R + 2 * (TNR / 2) <= 256 ? 256 : 512;
    static_assert(T_R + TNR <= TMEM_COLS, "tensor memory columns");
};

enum { B_WFULL = 0, B_XFULL = 1, B_XEMPTY = B_XFULL + NSTAGE, B_ZFULL = B_XEMPTY + NSTAGE,
       B_ZEMPTY = B_ZFULL + 2, B_RFULL = B_ZEMPTY + 2, B_REMPTY = B_RFULL + 2,
       B_GDONE = B_REMPTY + 2, B_DRAIN = B_GDONE + 1, NBAR = B_DRAIN + 1 };

template <int KP>
__global__ void __launch_bounds__(NTHR, 1)
logreg_grad_mma_kernel(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmX,
                       const __grid_constant__ CUtensorMap tmXt, const MmaArgs A) {
    if (A.guard != nullptr && *A.guard == 0) return;  // uniform: before any barrier or allocation
    using S = Smem<KP>;
    extern __shared__ __align__(1024) unsigned char mma_smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const uint32_t raw = smem_u32(mma_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned for the swizzle atoms
    unsigned char* gbase = mma_smem_raw + (base - raw);
    const uint32_t sW = base + S::OFF_W, sX = base + S::OFF_X;
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
        mbar_init(bar(B_WFULL), 1);
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(bar(B_XFULL + s), 1);
            mbar_init(bar(B_XEMPTY + s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar(B_ZFULL + b), 1);
            mbar_init(bar(B_ZEMPTY + b), NEPI);
            mbar_init(bar(B_RFULL + b), NEPI);
            mbar_init(bar(B_REMPTY + b), 1);
        }
        mbar_init(bar(B_GDONE), 1);
        mbar_init(bar(B_DRAIN), 1);
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
    const uint32_t tZ = tmem, tG = tmem + 2 * TNR, tR = tmem + S::T_R;

    if (warp == 0) {
      if (lane == 0) {
        // ------------------------------------------------ TMA producer
        bool ok = true;
        mbar_expect_tx(bar(B_WFULL), S::W_BYTES);
        for (int a = 0; a < 2 * S::NA; ++a)  // hi atoms then lo atoms: columns 64a of [hi | lo]
            tma_load_2d(sW + (uint32_t)a * (MT * 128), &tmW, 64 * a, (int)m0, bar(B_WFULL));
        int issued = 0;
        for (int c = 0; c < nc && ok; ++c) {
            const int st = c % NSTAGE;
            if (!mbar_wait(bar(B_XEMPTY + st), ((c / NSTAGE) & 1) ^ 1, deadline)) { ok = false; break; }
            const uint32_t dst = sX + (uint32_t)st * S::STAGE;
            mbar_expect_tx(bar(B_XFULL + st), S::STAGE);
            const int row = r_begin + c * TNR;
            for (int a = 0; a < S::NA; ++a)
                tma_load_2d(dst + (uint32_t)a * (TNR * 128), &tmX, 64 * a, row, bar(B_XFULL + st));
            tma_load_2d(dst + S::X_BYTES, &tmXt, row, 0, bar(B_XFULL + st));
            issued = c + 1;
        }
        if (!ok) {
            atomicExch(&s_fail, 1);
            // wait (bounded) for the copies this thread issued
            const unsigned long long d2 = global_ns() + drain_ns(A.timeout_ns);
            mbar_wait(bar(B_WFULL), 0, d2);
            for (int c = max(0, issued - NSTAGE); c < issued; ++c)
                mbar_wait(bar(B_XFULL + c % NSTAGE), (c / NSTAGE) & 1, d2);
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      if (lane == 0) {
        // ------------------------------------------------ MMA issuer
        constexpr uint32_t ID_Z = idesc_bf16(MT, TNR), ID_G = idesc_bf16(MT, KP);
        bool ok = mbar_wait(bar(B_WFULL), 0, deadline);
        tc_fence_after();
        auto gemm2 = [&](int cc) -> bool {
            const int rb = cc & 1, st = cc % NSTAGE;
            if (!mbar_wait(bar(B_RFULL + rb), (cc >> 1) & 1, deadline)) return false;
            tc_fence_after();
            const uint32_t aR = tR + (uint32_t)rb * (TNR / 2);
            const uint32_t bXt = sX + (uint32_t)st * S::STAGE + S::X_BYTES;
#pragma unroll
            for (int kk = 0; kk < TNR / 16; ++kk)
                tc_mma_ts(tG, aR + 8u * kk, sw128_desc(bXt + 32u * kk), ID_G,
                       (cc > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bar(B_REMPTY + rb));
            tc_commit(bar(B_XEMPTY + st));
            return true;
        };
        for (int c = 0; c <= nc && ok; ++c) {
            if (c < nc) {
                const int st = c % NSTAGE, zb = c & 1;
                if (!mbar_wait(bar(B_XFULL + st), (c / NSTAGE) & 1, deadline) ||
                    !mbar_wait(bar(B_ZEMPTY + zb), ((c >> 1) & 1) ^ 1, deadline)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t bX = sX + (uint32_t)st * S::STAGE;
                const uint32_t dZ = tZ + (uint32_t)zb * TNR;
                int k = 0;
#pragma unroll
                for (int part = 0; part < 2; ++part)
#pragma unroll
                    for (int kk = 0; kk < KP / 16; ++kk, ++k) {
                        const uint32_t aW = sW + (uint32_t)(part * S::NA + kk / 4) * (MT * 128) + 32u * (kk % 4);
                        const uint32_t bx = bX + (uint32_t)(kk / 4) * (TNR * 128) + 32u * (kk % 4);
                        tc_mma(dZ, sw128_desc(aW), sw128_desc(bx), ID_Z, k > 0 ? 1u : 0u);
                    }
                tc_commit(bar(B_ZFULL + zb));
            }
            if (c >= 1 && !gemm2(c - 1)) { ok = false; break; }
        }
        if (ok) {
            tc_commit(bar(B_GDONE));
        } else {
            atomicExch(&s_fail, 1);
            tc_commit(bar(B_DRAIN));  // everything issued so far has completed once this arrives
            mbar_wait(bar(B_DRAIN), 0, global_ns() + drain_ns(A.timeout_ns));
        }
      }
      __syncwarp();
    } else if (warp >= EPI_WARP0 && warp < EPI_WARP0 + NEPI) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;                 // TMEM lane quarter: chains 32q .. 32q+31
        const int h = (warp - EPI_WARP0) >> 2;  // column quarter: Z columns 16h .. 16h+15
        const int rt = 32 * q + lane;           // this thread's chain in the tile
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        ff lp = ff_make(0.0f);
        bool ok = true;
        for (int c = 0; c < nc; ++c) {
            const int zb = c & 1;
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
            if (!mbar_wait(bar(B_ZFULL + zb), (c >> 1) & 1, deadline)) { ok = false; break; }
            tc_fence_after();
            float z[16];
            tmem_ld16(tZ + lane_off + (uint32_t)(zb * TNR + 16 * h), z);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_ZEMPTY + zb));
            // residuals and log-likelihood terms.  Fast SFU approximations (this
            // form serves the unadjusted phase only): t = e^{-|z|}, sigmoid from
            // 1 / (1 + t), softplus = max(z, 0) + log(1 + t)
            float r[16];
            float lsum = 0.0f;
            auto body = [&](auto full) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float zz = z[j];
                    const float t = ex2_ftz(-1.4426950408889634f * fabsf(zz));  // e^{-|z|}
                    const float opt = 1.0f + t;
                    const float inv = rcp_ftz(opt);
                    const float sig = zz >= 0.0f ? inv : t * inv;
                    const float sp = fmaf(0.6931471805599453f, lg2_ftz(opt), fmaxf(zz, 0.0f));
                    const float term = fmaf(yy[j], zz, -sp);
                    if (decltype(full)::value) {
                        r[j] = yy[j] - sig;
                        lsum += term;
                    } else {
                        r[j] = j < nlive ? yy[j] - sig : 0.0f;
                        lsum += j < nlive ? term : 0.0f;
                    }
                }
            };
            if (nlive >= 16) body(std::true_type{});
            else body(std::false_type{});
            lp = ff_add(lp, lsum);
            const int rb = zb;
            if (!mbar_wait(bar(B_REMPTY + rb), ((c >> 1) & 1) ^ 1, deadline)) { ok = false; break; }
            // R row rt, data rows 16h .. 16h+15: columns 8h .. 8h+7 of this lane's R buffer
            uint32_t pr[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) pr[e] = pack_bf16(r[2 * e], r[2 * e + 1]);
            tmem_st8(tR + lane_off + (uint32_t)(rb * (TNR / 2) + 8 * h), pr);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_RFULL + rb));
        }
        if (ok && !mbar_wait(bar(B_GDONE), 0, deadline)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        const int64_t m = m0 + rt;
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

// ------------------------------------------------------------------ host
__global__ void to_bf16_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ Xb,
                               __nv_bfloat16* __restrict__ Xtb, int n, int n_pad, int kp) {
    const int64_t tot = (int64_t)n_pad * kp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(k / kp), i = (int)(k - (int64_t)r * kp);
        const __nv_bfloat16 v = __float2bfloat16_rn(r < n ? X[(size_t)r * kp + i] : 0.0f);
        Xb[k] = v;
        Xtb[(size_t)i * n_pad + r] = v;
    }
}

// caller's points [M][d] -> the FP32 [M][kp] copy and the BF16 hi | lo [M_pad][2 kp] copy
__global__ void pack_points_kernel(const float* __restrict__ x, int64_t M, int d, int kp,
                                   float* __restrict__ W32, __nv_bfloat16* __restrict__ Wb) {
    const int64_t n = M * kp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k / kp;
        const int i = (int)(k - m * kp);
        const float v = i < d ? x[m * d + i] : 0.0f;
        W32[k] = v;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        Wb[m * 2 * kp + i] = hi;
        Wb[m * 2 * kp + kp + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

}  // namespace

cudaError_t logreg_pack_points(const float* x, int64_t M, int d, int kp, float* W32, void* Wb,
                               cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((M * kp + 255) / 256, 4096);
    pack_points_kernel<<<std::max(blocks, 1), 256, 0, st>>>(x, M, d, kp, W32,
                                                          reinterpret_cast<__nv_bfloat16*>(Wb));
    return cudaGetLastError();
}

bool logreg_mma_supported(int kp) { return kp == 64 || kp == 128; }

size_t logreg_mma_smem(int kp) { return kp == 64 ? Smem<64>::TOTAL : Smem<128>::TOTAL; }

cudaError_t logreg_mma_prepare(LogregData& D) {
    if (!logreg_mma_supported(D.kp)) return cudaErrorInvalidValue;
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    D.n_pad = (D.n + TNR - 1) / TNR * TNR;
    const size_t nb = (size_t)D.n_pad * D.kp * sizeof(__nv_bfloat16);
    cudaError_t e = cudaMalloc(&D.Xb, nb);
    if (e == cudaSuccess) e = cudaMalloc(&D.Xtb, nb);
    if (e != cudaSuccess) return e;
    to_bf16_kernel<<<std::min(4096, (int)((D.n_pad * (int64_t)D.kp + 255) / 256)), 256>>>(
        D.X, reinterpret_cast<__nv_bfloat16*>(D.Xb), reinterpret_cast<__nv_bfloat16*>(D.Xtb), D.n, D.n_pad, D.kp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const cuuint32_t es[2] = {1, 1};
    {   // X: [n_pad][kp], boxes of 64 features x 64 rows
        const cuuint64_t dims[2] = {(cuuint64_t)D.kp, (cuuint64_t)D.n_pad};
        const cuuint64_t strides[1] = {(cuuint64_t)D.kp * 2};
        const cuuint32_t box[2] = {64, TNR};
        if (enc(reinterpret_cast<CUtensorMap*>(D.tmX), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, D.Xb, dims, strides,
                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {   // X^T: [kp][n_pad], boxes of 64 rows x kp features
        const cuuint64_t dims[2] = {(cuuint64_t)D.n_pad, (cuuint64_t)D.kp};
        const cuuint64_t strides[1] = {(cuuint64_t)D.n_pad * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)D.kp};
        if (enc(reinterpret_cast<CUtensorMap*>(D.tmXt), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, D.Xtb, dims, strides,
                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    return cudaDeviceSynchronize();
}

cudaError_t logreg_mma_wmap(void* tmW, const void* Wb, int64_t M_pad, int kp) {
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint32_t es[2] = {1, 1};
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * kp), (cuuint64_t)M_pad};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * kp) * 2};
    const cuuint32_t box[2] = {64, MT};
    if (enc(reinterpret_cast<CUtensorMap*>(tmW), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(Wb), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

int logreg_mma_splits(const LogregData& D, int64_t M, int nsm, int* rps_out) {
    const int64_t tiles = (M + MT - 1) / MT;
    int S = (int)std::max<int64_t>(1, nsm / std::max<int64_t>(1, tiles));
    const int chunks = (D.n + TNR - 1) / TNR;
    S = std::max(1, std::min(S, chunks));
    int rps = ((D.n + S - 1) / S + TNR - 1) / TNR * TNR;
    S = (D.n + rps - 1) / rps;
    if (rps_out) *rps_out = rps;
    return S;
}

cudaError_t logreg_grad_mma(const LogregData& D, const void* tmW, const float* W32, int64_t M, int S,
                            int rps, float* gpart, float2* lpart, int* status, long long timeout_ns,
                            cudaStream_t st, const int* guard) {
    if (M <= 0) return cudaSuccess;
    MmaArgs a;
    a.M = M;
    a.n = D.n;
    a.rps = rps;
    a.inv_v = D.inv_v;
    a.W32 = W32;
    a.y = D.y;
    a.gpart = gpart;
    a.lpart = lpart;
    a.status = status;
    a.timeout_ns = timeout_ns;
    a.guard = guard;
    const dim3 grid((unsigned)((M + MT - 1) / MT), (unsigned)S);
    const CUtensorMap& mw = *reinterpret_cast<const CUtensorMap*>(tmW);
    const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(D.tmX);
    const CUtensorMap& mt = *reinterpret_cast<const CUtensorMap*>(D.tmXt);
    cudaError_t e;
    if (D.kp == 64) {
        e = cudaFuncSetAttribute(logreg_grad_mma_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<64>::TOTAL);
        if (e != cudaSuccess) return e;
        logreg_grad_mma_kernel<64><<<grid, NTHR, Smem<64>::TOTAL, st>>>(mw, mx, mt, a);
    } else if (D.kp == 128) {
        e = cudaFuncSetAttribute(logreg_grad_mma_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<128>::TOTAL);
        if (e != cudaSuccess) return e;
        logreg_grad_mma_kernel<128><<<grid, NTHR, Smem<128>::TOTAL, st>>>(mw, mx, mt, a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace laps
