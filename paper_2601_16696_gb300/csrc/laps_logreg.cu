// laps_logreg.cu -- FP32 SIMT gradient of the logistic-regression target for
// an ensemble of points (the all-FP32 form; also the adjusted phase of the
// mixed-precision form).
//
// A block owns a tile of 64 chains and one range of data rows.  Its 64 x kp
// slice of W stays in shared memory; the data rows stream through shared
// memory 64 at a time.  Per chunk:
//   Z  = W_tile X_chunk^T      (64 x 64, thread tile 4 chains x 4 rows)
//   R  = y - sigmoid(Z), log p terms y z - softplus(z)   (registers)
//   G += R^T-tile X_chunk      (64 x kp, thread tile 4 chains x 4 NG coords)
// so Z and R live only in registers and a 17 KB shared tile.
#include <cuda_runtime.h>

#include <algorithm>

#include "laps_device.cuh"
#include "laps_logreg.cuh"

namespace laps {

namespace {

constexpr int TM = 64;    // chains per block
constexpr int TN = 64;    // data rows per chunk
constexpr int NT = 256;   // threads
constexpr int RTS = TM + 4;  // row stride of the transposed R tile

template <int KP>
__global__ void __launch_bounds__(NT, KP <= 128 ? 2 : 1)
logreg_grad_f32_kernel(const float* __restrict__ W, int64_t M, const float* __restrict__ X,
                       const float* __restrict__ yv, int n, int rps, float inv_v,
                       float* __restrict__ gpart, float2* __restrict__ lpart, const int* __restrict__ guard) {
    if (guard != nullptr && *guard == 0) return;  // the iteration no longer runs
    constexpr int LD = KP + 4;   // padded row stride (floats) of the W and X tiles
    constexpr int NG = KP / 64;  // float4 column groups per thread in the G phase
    extern __shared__ __align__(16) float sm[];
    float* Ws = sm;                 // [TM][LD]
    float* Xs = Ws + TM * LD;       // [TN][LD]
    float* Rt = Xs + TN * LD;       // [TN][RTS]  R transposed: Rt[row][chain]
    float* wsq = Rt + TN * RTS;     // [TM] |w|^2

    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int s = blockIdx.y;
    const int r_begin = s * rps;
    const int r_end = min(n, r_begin + rps);

    // W tile (rows beyond M are zero)
    for (int k = tid; k < TM * (KP / 4); k += NT) {
        const int r = k / (KP / 4), c4 = k - r * (KP / 4);
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (m0 + r < M) v = *reinterpret_cast<const float4*>(W + (m0 + r) * KP + 4 * c4);
        *reinterpret_cast<float4*>(Ws + r * LD + 4 * c4) = v;
    }
    __syncthreads();
    if (s == 0) {  // |w|^2 for the prior term: 4 lanes per chain
        const int r = tid >> 2, q = tid & 3;
        float a = 0.0f;
        for (int k = q; k < KP; k += 4) a = fmaf(Ws[r * LD + k], Ws[r * LD + k], a);
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (q == 0) wsq[r] = a;
    }

    const int cr = tid >> 4;  // chains 4cr .. 4cr+3 of the tile
    const int dc = tid & 15;  // Z phase: rows dc + 16e;  G phase: columns 64q + 4dc .. +3
    float gacc[4][4 * NG];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 4 * NG; ++k) gacc[c][k] = 0.0f;
    ff lacc[4] = {ff_make(0.0f), ff_make(0.0f), ff_make(0.0f), ff_make(0.0f)};

    for (int row0 = r_begin; row0 < r_end; row0 += TN) {
        // ---- the chunk's data rows (rows past the range are zero and masked below)
        __syncthreads();
        for (int k = tid; k < TN * (KP / 4); k += NT) {
            const int r = k / (KP / 4), c4 = k - r * (KP / 4);
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (row0 + r < r_end) v = *reinterpret_cast<const float4*>(X + (size_t)(row0 + r) * KP + 4 * c4);
            *reinterpret_cast<float4*>(Xs + r * LD + 4 * c4) = v;
        }
        __syncthreads();
        // ---- Z = W X^T on the 4 x 4 thread tile
        float z[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) z[c][e] = 0.0f;
#pragma unroll 4
        for (int k = 0; k < KP; k += 4) {
            float4 wv[4], xv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) wv[c] = *reinterpret_cast<const float4*>(Ws + (4 * cr + c) * LD + k);
#pragma unroll
            for (int e = 0; e < 4; ++e) xv[e] = *reinterpret_cast<const float4*>(Xs + (dc + 16 * e) * LD + k);
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    z[c][e] = fmaf(wv[c].x, xv[e].x, z[c][e]);
                    z[c][e] = fmaf(wv[c].y, xv[e].y, z[c][e]);
                    z[c][e] = fmaf(wv[c].z, xv[e].z, z[c][e]);
                    z[c][e] = fmaf(wv[c].w, xv[e].w, z[c][e]);
                }
        }
        // ---- epilogue: residuals and log-likelihood terms
        float lsum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = row0 + dc + 16 * e;
            const bool ok = row < r_end;
            const float yn = ok ? yv[row] : 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float zz = z[c][e];
                const float t = expf(-fabsf(zz));               // e^{-|z|} in (0, 1]
                const float sp = fmaxf(zz, 0.0f) + log1pf(t);   // softplus(z)
                const float inv = 1.0f / (1.0f + t);
                const float sig = zz >= 0.0f ? inv : t * inv;   // sigmoid(z)
                Rt[(dc + 16 * e) * RTS + 4 * cr + c] = ok ? yn - sig : 0.0f;
                lsum[c] += ok ? fmaf(yn, zz, -sp) : 0.0f;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) lacc[c] = ff_add(lacc[c], lsum[c]);
        __syncthreads();
        // ---- G += R^T X over the chunk's rows
#pragma unroll 4
        for (int r = 0; r < TN; ++r) {
            const float4 rv = *reinterpret_cast<const float4*>(Rt + r * RTS + 4 * cr);
            const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                const float4 xv = *reinterpret_cast<const float4*>(Xs + r * LD + 64 * q + 4 * dc);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    gacc[c][4 * q + 0] = fmaf(rr[c], xv.x, gacc[c][4 * q + 0]);
                    gacc[c][4 * q + 1] = fmaf(rr[c], xv.y, gacc[c][4 * q + 1]);
                    gacc[c][4 * q + 2] = fmaf(rr[c], xv.z, gacc[c][4 * q + 2]);
                    gacc[c][4 * q + 3] = fmaf(rr[c], xv.w, gacc[c][4 * q + 3]);
                }
            }
        }
    }
    __syncthreads();  // wsq is visible (written before the loop; the loop may be empty)

    // ---- outputs: gradient partial (plus the prior on range 0) and log p partial
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t m = m0 + 4 * cr + c;
        // log p: the 16 threads of this chain group add their partials in a fixed order
        ff l = group_sum_ff<16>(lacc[c]);
        if (m >= M) continue;
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            const int col = 64 * q + 4 * dc;
            float4 v = make_float4(gacc[c][4 * q], gacc[c][4 * q + 1], gacc[c][4 * q + 2], gacc[c][4 * q + 3]);
            if (s == 0) {
                const float4 w = *reinterpret_cast<const float4*>(Ws + (4 * cr + c) * LD + col);
                v.x = fmaf(-w.x, inv_v, v.x);
                v.y = fmaf(-w.y, inv_v, v.y);
                v.z = fmaf(-w.z, inv_v, v.z);
                v.w = fmaf(-w.w, inv_v, v.w);
            }
            *reinterpret_cast<float4*>(gpart + ((size_t)s * M + m) * KP + col) = v;
        }
        if (dc == 0) {
            if (s == 0) l = ff_add(l, -0.5f * inv_v * wsq[4 * cr + c]);
            lpart[(size_t)s * M + m] = make_float2(l.hi, l.lo);
        }
    }
}

template <int KP>
size_t f32_smem() {
    return ((size_t)TM * (KP + 4) + (size_t)TN * (KP + 4) + (size_t)TN * RTS + TM) * sizeof(float);
}

template <int KP>
cudaError_t launch_f32(const LogregData& D, const float* W, int64_t M, int S, float* gpart,
                       float2* lpart, cudaStream_t st, const int* guard) {
    const size_t smem = f32_smem<KP>();
    cudaError_t e = cudaFuncSetAttribute(logreg_grad_f32_kernel<KP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int rps = (D.n + S - 1) / S;
    const dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)S);
    logreg_grad_f32_kernel<KP><<<grid, NT, smem, st>>>(W, M, D.X, D.y, D.n, rps, D.inv_v, gpart, lpart, guard);
    return cudaGetLastError();
}

}  // namespace

namespace {
template <int KP>
int f32_blocks_per_sm() {
    int n = 0;
    if (cudaFuncSetAttribute(logreg_grad_f32_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)f32_smem<KP>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, logreg_grad_f32_kernel<KP>, NT, f32_smem<KP>()) !=
            cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return std::max(n, 1);
}
}  // namespace

int logreg_f32_splits(const LogregData& D, int64_t M, int nsm) {
    int bps = 1;
    switch (D.kp) {
    case 64: bps = f32_blocks_per_sm<64>(); break;
    case 128: bps = f32_blocks_per_sm<128>(); break;
    case 192: bps = f32_blocks_per_sm<192>(); break;
    case 256: bps = f32_blocks_per_sm<256>(); break;
    }
    const int64_t tiles = (M + TM - 1) / TM, slots = (int64_t)bps * std::max(nsm, 1);
    const int chunks = std::max(1, (D.n + TN - 1) / TN);
    // a block's time ~ its rows plus about one chunk of fixed work (the W tile in,
    // the partials out); the run's time ~ waves x that
    int best = 1;
    int64_t best_cost = -1;
    for (int S = 1; S <= std::min(16, chunks); ++S) {
        const int64_t waves = (tiles * S + slots - 1) / slots;
        const int64_t cost = waves * ((D.n + S - 1) / S + TN);
        if (best_cost < 0 || cost < best_cost) {
            best = S;
            best_cost = cost;
        }
    }
    return best;
}

cudaError_t logreg_grad_f32(const LogregData& D, const float* W, int64_t M, int S, float* gpart,
                            float2* lpart, cudaStream_t st, const int* guard) {
    if (M <= 0) return cudaSuccess;
    if (S < 1 || S > 65535 || (M + TM - 1) / TM > 0x7fffffff) return cudaErrorInvalidValue;
    switch (D.kp) {
    case 64: return launch_f32<64>(D, W, M, S, gpart, lpart, st, guard);
    case 128: return launch_f32<128>(D, W, M, S, gpart, lpart, st, guard);
    case 192: return launch_f32<192>(D, W, M, S, gpart, lpart, st, guard);
    case 256: return launch_f32<256>(D, W, M, S, gpart, lpart, st, guard);
    }
    return cudaErrorInvalidValue;
}

}  // namespace laps
