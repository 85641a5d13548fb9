// laps_gauss_dense.cu -- log p and gradient of a Gaussian given by a dense
// precision matrix P (the rotated ill-conditioned Gaussian of the paper's
// Sec. 6):  log p = -1/2 x^T P x,  grad log p = -P x,  for the ensemble's
// points as one chains-by-coordinates contraction G = -W P.
//
// A block owns 8 CW chains: their points stay in shared memory, P streams
// through shared memory 32 rows at a time (rows up to d only), warp w accumulates chains
// CW w .. CW w + CW - 1 and lane l the columns l, l + 32, ... (conflict-free row
// reads of P, broadcast reads of the points).
//
// The target is ill-conditioned (condition number ~1e5 in the paper's
// experiment), so -P x cancels: a binary32 dot product loses ~1e-4 of max|g|.
// Each product therefore enters exactly (fma residual) into a float-float
// accumulator, the compensated dot product of Ogita, Rump and Oishi ("Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005): the result is as
// accurate as a dot product in twice the working precision, rounded once.
// log p sums x_o (P x)_o the same way, one warp butterfly per chain.
#include <cuda_runtime.h>

#include "laps_internal.h"

namespace laps {

namespace {
constexpr int kThreads = 256, kRows = 32;

// W [M][dp] points (zero padded), P [dp][dp] symmetric (zero padded), dp = 32 Q.
// G [M][dp] receives -P x (zeros in the padding), LP [M] log p as float-float.
template <int Q, int CW>
__global__ void __launch_bounds__(kThreads) gauss_dense_grad_kernel(const float* __restrict__ P, int d,
                                                                     const float* __restrict__ W, int64_t M,
                                                                     float* __restrict__ G,
                                                                     float2* __restrict__ LP,
                                                                     const int* __restrict__ guard) {
    if (guard != nullptr && *guard == 0) return;  // the iteration no longer runs
    constexpr int dp = 32 * Q, nch = 8 * CW;
    extern __shared__ __align__(16) float sm[];
    float* Xs = sm;                 // [nch][dp]
    float* Ps = sm + nch * dp;      // [kRows][dp]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t m0 = (int64_t)blockIdx.x * nch;
    const int nc = (int)(M - m0 < nch ? M - m0 : nch);
    for (int o = tid; o < nch * dp / 4; o += kThreads) {
        const int c = o / (dp / 4), j = o - c * (dp / 4);
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (c < nc) v = reinterpret_cast<const float4*>(W + (m0 + c) * dp)[j];
        reinterpret_cast<float4*>(Xs)[o] = v;
    }
    float hi[CW][Q], lo[CW][Q];
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int q = 0; q < Q; ++q) hi[c][q] = lo[c][q] = 0.0f;
    for (int k0 = 0; k0 < d; k0 += kRows) {
        __syncthreads();  // the points are staged; the previous rows are consumed
        for (int o = tid; o < kRows * dp / 4; o += kThreads)
            reinterpret_cast<float4*>(Ps)[o] = reinterpret_cast<const float4*>(P + (size_t)k0 * dp)[o];
        __syncthreads();
        // rows past d of P are zero: they would add exact zeros, so stop at d
        const int kn = d - k0 < kRows ? d - k0 : kRows;
#pragma unroll 2
        for (int kk = 0; kk < kn; ++kk) {
            float p[Q], x[CW];
#pragma unroll
            for (int q = 0; q < Q; ++q) p[q] = Ps[kk * dp + lane + 32 * q];
#pragma unroll
            for (int c = 0; c < CW; ++c) x[c] = Xs[(CW * warp + c) * dp + k0 + kk];
#pragma unroll
            for (int c = 0; c < CW; ++c)
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float pr = x[c] * p[q];
                    const float er = fmaf(x[c], p[q], -pr);  // exact: x p = pr + er
                    float sh, sl;
                    two_sum(hi[c][q], pr, sh, sl);
                    hi[c][q] = sh;
                    lo[c][q] += sl + er;
                }
        }
    }
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int ch = CW * warp + c;
        ff l = ff_make(0.0f);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int o = lane + 32 * q;
            const float xo = Xs[ch * dp + o], r = hi[c][q] + lo[c][q];
            const float pr = xo * r;
            l = ff_add(l, ff{pr, fmaf(xo, r, -pr)});
            if (ch < nc) G[(m0 + ch) * dp + o] = o < d ? -r : 0.0f;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const ff w{__shfl_xor_sync(0xffffffffu, l.hi, off), __shfl_xor_sync(0xffffffffu, l.lo, off)};
            l = ff_add(l, w);
        }
        if (lane == 0 && ch < nc) LP[m0 + ch] = make_float2(-0.5f * l.hi, -0.5f * l.lo);
    }
}

template <int Q>
cudaError_t launch_q(const float* P, int d, const float* W, int64_t M, float* G, float2* LP, cudaStream_t st,
                     const int* guard) {
    // accumulators: 2 CW Q registers; 8 CW chains per block, so that the ensembles
    // of a few thousand chains give every SM a block or more
    constexpr int CW = Q <= 8 ? 2 : 1;
    const size_t smem = (size_t)(8 * CW + kRows) * 32 * Q * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(gauss_dense_grad_kernel<Q, CW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (M + 8 * CW - 1) / (8 * CW);
    gauss_dense_grad_kernel<Q, CW><<<(unsigned)blocks, kThreads, smem, st>>>(P, d, W, M, G, LP, guard);
    return cudaGetLastError();
}
}  // namespace

cudaError_t gauss_dense_grad(const float* P, int d_pad, int d, const float* W, int64_t M, float* G,
                             float2* LP, cudaStream_t st, const int* guard) {
    if (M <= 0) return cudaSuccess;
    if (d_pad % 32 || d_pad < 32 || d_pad > kDenseMaxDim || M > (1LL << 30)) return cudaErrorInvalidValue;
    switch (d_pad / 32) {
#define LAPS_Q(n) \
    case n: return launch_q<n>(P, d, W, M, G, LP, st, guard);
        LAPS_Q(1) LAPS_Q(2) LAPS_Q(3) LAPS_Q(4) LAPS_Q(5) LAPS_Q(6) LAPS_Q(7) LAPS_Q(8)
        LAPS_Q(9) LAPS_Q(10) LAPS_Q(11) LAPS_Q(12) LAPS_Q(13) LAPS_Q(14) LAPS_Q(15) LAPS_Q(16)
#undef LAPS_Q
    }
    return cudaErrorInvalidValue;
}

}  // namespace laps
