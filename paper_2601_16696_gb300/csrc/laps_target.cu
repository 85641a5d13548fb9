// laps_target.cu -- stand-alone log-density + gradient of the built-in targets
// (the forward and hand-written backward used by the sampler), for M points in
// the caller's [M][d] layout.  One warp per point; log p is summed with
// compensated float-float arithmetic and rounded to FP32 at the end.
#include <cuda_runtime.h>

#include <algorithm>

#include "laps_internal.h"

namespace laps {

__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

__global__ void target_logp_grad_kernel(int kind, const float* __restrict__ x, int64_t M, int d,
                                        const float* __restrict__ prec, float inv_s2, float inv_sv2,
                                        float* __restrict__ logp, float* __restrict__ grad) {
    const int lane = threadIdx.x & 31;
    const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (m >= M) return;  // whole warps exit together
    const float* xm = x + m * d;
    float* gm = grad + m * d;
    ff part = ff_make(0.0f);
    if (kind == TGT_GAUSS) {
        for (int i = lane; i < d; i += 32) {
            const float gx = -prec[i] * xm[i];
            gm[i] = gx;
            part = ff_add(part, 0.5f * gx * xm[i]);
        }
        part = warp_sum_ff(part);
    } else if (kind == TGT_BANANA) {
        for (int k = lane; 2 * k + 1 < d; k += 32) {
            const float a = xm[2 * k], b = xm[2 * k + 1];
            const float r = fmaf(-a, a, b);
            const float ris = r * inv_s2;
            part = ff_add(part, fmaf(-0.5f * a, a, -0.5f * r * ris));
            gm[2 * k] = fmaf(2.0f * a, ris, -a);
            gm[2 * k + 1] = -ris;
        }
        part = warp_sum_ff(part);
    } else {  // funnel
        float ss = 0.0f;
        for (int i = 1 + lane; i < d; i += 32) ss = fmaf(xm[i], xm[i], ss);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float v = xm[0];
        const float ev = expf(-v);
        const float n = (float)(d - 1);
        part = ff_make(-0.5f * v * v * inv_sv2);
        part = ff_add(part, -0.5f * n * v);
        part = ff_add(part, -0.5f * ev * ss);
        for (int i = 1 + lane; i < d; i += 32) gm[i] = -xm[i] * ev;
        if (lane == 0) gm[0] = fmaf(-v, inv_sv2, -0.5f * n) + 0.5f * ev * ss;
    }
    if (lane == 0) logp[m] = part.hi + part.lo;
}

// LOGREG: the caller's [M][d] points padded to the contraction layout and back
__global__ void logreg_pack_kernel(const float* __restrict__ x, float* __restrict__ W, int64_t M,
                                   int d, int kp) {
    const int64_t n = M * kp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k / kp;
        const int i = (int)(k - m * kp);
        W[k] = i < d ? x[m * d + i] : 0.0f;
    }
}
// the S partials of the gradient kernel summed in order, back to the caller's [M][d]
__global__ void logreg_unpack_kernel(const float* __restrict__ G, const float2* __restrict__ lp,
                                     float* __restrict__ grad, float* __restrict__ logp, int64_t M,
                                     int d, int kp, int S) {
    const int64_t n = M * d;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = k / d;
        const int i = (int)(k - m * d);
        float g = 0.0f;
        for (int s = 0; s < S; ++s) g += G[((size_t)s * M + m) * kp + i];
        grad[k] = g;
        if (i == 0) {
            ff l = ff_make(0.0f);
            for (int s = 0; s < S; ++s) l = ff_add(l, ff{lp[(size_t)s * M + m].x, lp[(size_t)s * M + m].y});
            logp[m] = l.hi + l.lo;
        }
    }
}

// USER targets: the callback's FP32 log p as the float-float partial the chain
// updates read, and the gradient's padding columns cleared (the sampler's norms
// and dot products run over the padded rows)
__global__ void user_after_kernel(const float* __restrict__ lp, float2* __restrict__ LP, float* __restrict__ G,
                                  int64_t M, int d, int ld) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        LP[m] = make_float2(lp[m], 0.0f);
        for (int i = d; i < ld; ++i) G[m * ld + i] = 0.0f;
    }
}

laps_status user_grad(const laps_target* tg, const float* W, int64_t M, int ld, float* G, float* lp32,
                      float2* LP, cudaStream_t st) {
    const int r = tg->desc.user_fn(W, M, ld, lp32, G, (void*)st, tg->desc.user_data);
    if (r != 0) return fail(LAPS_ERR_CUDA, "user_fn returned " + std::to_string(r));
    const int blocks = (int)std::min<int64_t>((M + 255) / 256, 4096);
    user_after_kernel<<<blocks, 256, 0, st>>>(lp32, LP, G, M, tg->d, ld);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "user_after_kernel");
}

// targets evaluated by an ensemble contraction (LOGREG, GAUSS_DENSE): the points
// packed to the contraction's padded rows, its partials back to [M][d]
static laps_status streamed_logp_grad(const laps_target* tg, const float* x, int64_t M, float* logp,
                                      float* grad, cudaStream_t st) {
    const int kp = tg->d_pad, d = tg->d;
    const int S = streamed_target_splits(tg, M);
    float *W = nullptr, *G = nullptr;
    float2* lp = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&W, (size_t)M * kp * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&G, (size_t)S * M * kp * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&lp, (size_t)S * M * 8, st);
    laps_status rs = LAPS_OK;
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<int64_t>((M * kp + 255) / 256, 4096);
        logreg_pack_kernel<<<blocks, 256, 0, st>>>(x, W, M, d, kp);
        rs = streamed_target_grad(tg, W, M, S, G, lp, st);
        if (rs == LAPS_OK) {
            logreg_unpack_kernel<<<blocks, 256, 0, st>>>(G, lp, grad, logp, M, d, kp, S);
            e = cudaGetLastError();
        }
    }
    if (W) cudaFreeAsync(W, st);
    if (G) cudaFreeAsync(G, st);
    if (lp) cudaFreeAsync(lp, st);
    if (rs != LAPS_OK) return rs;
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "logp_grad of a contraction target");
}

// LOGREG on the tensor cores (the mixed-precision form's unadjusted-phase
// arithmetic: BF16-rounded data, points as two BF16 terms); stream-ordered, a
// bounded wait that expired is latched in the target's status word
static laps_status logreg_logp_grad_mixed(const laps_target* tg, const float* x, int64_t M, float* logp,
                                          float* grad, cudaStream_t st) {
    const LogregData& L = tg->lr;
    if (!L.Xb) return fail(LAPS_ERR_UNSUPPORTED, "mixed precision is built for LOGREG with d <= 128");
    const int kp = L.kp, d = tg->d;
    const int64_t M_pad = (M + 127) / 128 * 128;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int rps = 64;
    const int S = logreg_mma_splits(L, M, nsm, &rps);
    float *W32 = nullptr, *G = nullptr;
    void* Wb = nullptr;
    float2* lp = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&W32, (size_t)M * kp * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&Wb, (size_t)M_pad * 2 * kp * 2, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&G, (size_t)S * M * kp * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&lp, (size_t)S * M * 8, st);
    alignas(64) unsigned char tmW[128];
    if (e == cudaSuccess && M_pad > M)  // the last tile's rows past M stay zero
        e = cudaMemsetAsync(static_cast<char*>(Wb) + (size_t)M * 2 * kp * 2, 0,
                            (size_t)(M_pad - M) * 2 * kp * 2, st);
    if (e == cudaSuccess) e = logreg_pack_points(x, M, d, kp, W32, Wb, st);
    if (e == cudaSuccess) e = logreg_mma_wmap(tmW, Wb, M_pad, kp);
    if (e == cudaSuccess) e = logreg_grad_mma(L, tmW, W32, M, S, rps, G, lp, tg->status, 2000000000LL, st);
    if (e == cudaSuccess) {
        const int blocks = (int)std::min<int64_t>((M * d + 255) / 256, 4096);
        logreg_unpack_kernel<<<std::max(blocks, 1), 256, 0, st>>>(G, lp, grad, logp, M, d, kp, S);
        e = cudaGetLastError();
    }
    if (W32) cudaFreeAsync(W32, st);
    if (Wb) cudaFreeAsync(Wb, st);
    if (G) cudaFreeAsync(G, st);
    if (lp) cudaFreeAsync(lp, st);
    if (e != cudaSuccess) return cuda_fail(e, "LOGREG logp_grad (tensor cores)");
    return LAPS_OK;
}

// LOGREG on the tensor cores at FP32 accuracy (points, data and residuals
// each as three BF16 terms); stream-ordered, a bounded wait that expired is
// latched in the target's status word
static laps_status logreg_logp_grad_x3(const laps_target* tg, const float* x, int64_t M, float* logp,
                                       float* grad, cudaStream_t st) {
    const LogregData& L = tg->lr;
    if (!L.X3b) return fail(LAPS_ERR_UNSUPPORTED, "the three-term tensor-core form is built for LOGREG with d <= 128");
    const int kp = L.kp, d = tg->d;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int rps = 64;
    const int S = logreg_x3_splits(L, M, nsm, &rps);
    float *W32 = nullptr, *G = nullptr;
    float2* lp = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&W32, (size_t)M * kp * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&G, (size_t)S * M * kp * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&lp, (size_t)S * M * 8, st);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((M * kp + 255) / 256, 4096));
    if (e == cudaSuccess) {
        logreg_pack_kernel<<<blocks, 256, 0, st>>>(x, W32, M, d, kp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = logreg_grad_x3(L, W32, M, S, rps, G, lp, tg->status, 2000000000LL, st);
    if (e == cudaSuccess) {
        logreg_unpack_kernel<<<blocks, 256, 0, st>>>(G, lp, grad, logp, M, d, kp, S);
        e = cudaGetLastError();
    }
    if (W32) cudaFreeAsync(W32, st);
    if (G) cudaFreeAsync(G, st);
    if (lp) cudaFreeAsync(lp, st);
    if (e != cudaSuccess) return cuda_fail(e, "LOGREG logp_grad (tensor cores, three-term split)");
    return LAPS_OK;
}

}  // namespace laps

using namespace laps;

extern "C" laps_status laps_target_status(laps_target* tg) {
    if (!tg) return fail(LAPS_ERR_INVALID_ARG, "null target");
    if (!tg->status) return LAPS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    int s = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&s, tg->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(tg->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "laps_target_status");
    return status_error(s);
}

extern "C" laps_status laps_target_logp_grad_prec(const laps_target* tg, const float* x, int64_t M,
                                                  float* logp, float* grad, int precision, void* stream) {
    if (!tg || M < 0 || (M > 0 && (!x || !logp || !grad))) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if (precision == LAPS_FP32) return laps_target_logp_grad(tg, x, M, logp, grad, stream);
    if (precision != LAPS_MIXED && precision != LAPS_BF16X3) return fail(LAPS_ERR_INVALID_ARG, "unknown precision");
    if (tg->kind != TGT_LOGREG) return fail(LAPS_ERR_UNSUPPORTED, "mixed precision applies to LOGREG only");
    if (M == 0) return LAPS_OK;
    if (precision == LAPS_BF16X3) return logreg_logp_grad_x3(tg, x, M, logp, grad, (cudaStream_t)stream);
    return logreg_logp_grad_mixed(tg, x, M, logp, grad, (cudaStream_t)stream);
}

extern "C" laps_status laps_target_logp_grad(const laps_target* tg, const float* x, int64_t M,
                                             float* logp, float* grad, void* stream) {
    if (!tg || M < 0 || (M > 0 && (!x || !logp || !grad))) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if (M == 0) return LAPS_OK;
    if (tg->kind == TGT_USER) {
        const int r = tg->desc.user_fn(x, M, tg->d, logp, grad, stream, tg->desc.user_data);
        return r == 0 ? LAPS_OK : fail(LAPS_ERR_CUDA, "user_fn returned " + std::to_string(r));
    }
    if (streamed_kind(tg->kind)) return streamed_logp_grad(tg, x, M, logp, grad, (cudaStream_t)stream);
    const int threads = 256;
    const int64_t blocks = (M * 32 + threads - 1) / threads;
    if (blocks > 0x7fffffff) return fail(LAPS_ERR_INVALID_ARG, "M too large");
    const laps_target_desc& dsc = tg->desc;
    target_logp_grad_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        tg->kind, x, M, tg->d, tg->prec_pad, (float)(1.0 / (dsc.banana_sb * dsc.banana_sb)),
        (float)(1.0 / (dsc.funnel_sv * dsc.funnel_sv)), logp, grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "target_logp_grad_kernel");
    return LAPS_OK;
}

// ---------------------------------------------------------------- random stream
namespace laps {
__global__ void philox_kernel(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                              uint4* __restrict__ out, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = philox4x32_10(ctr[k], k0, k1);
}
__global__ void normals_kernel(uint32_t k0, uint32_t k1, uint32_t m0, int64_t nm, uint32_t t,
                               uint32_t tagpid, int64_t d, float* __restrict__ out) {
    const int64_t nblk = (d + 3) / 4;
    const int64_t n = nm * nblk;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mm = k / nblk, j = k - mm * nblk;
        float z[4];
        normals4((uint32_t)j, m0 + (uint32_t)mm, t, tagpid, k0, k1, z);
        for (int c = 0; c < 4; ++c)
            if (4 * j + c < d) out[mm * d + 4 * j + c] = z[c];
    }
}
}  // namespace laps

extern "C" laps_status laps_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n,
                                   void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) % 16)
        return fail(LAPS_ERR_INVALID_ARG, "ctr and out must be 16-byte aligned");
    if (n == 0) return LAPS_OK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    philox_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const uint4*>(ctr), (uint32_t)seed, (uint32_t)(seed >> 32),
        reinterpret_cast<uint4*>(out), n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "philox_kernel");
}

extern "C" laps_status laps_normals(uint64_t seed, uint32_t m0, int64_t nm, uint32_t t,
                                    uint32_t tag, uint32_t pid, int64_t d, float* out,
                                    void* stream) {
    if (nm < 0 || d < 1 || (nm > 0 && !out) || tag > 255 || pid >= (1u << 24))
        return fail(LAPS_ERR_INVALID_ARG, "bad argument");
    if (nm == 0) return LAPS_OK;
    const int64_t n = nm * ((d + 3) / 4);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    normals_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), m0, nm, t, tag | (pid << 8), d, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LAPS_OK : cuda_fail(e, "normals_kernel");
}
