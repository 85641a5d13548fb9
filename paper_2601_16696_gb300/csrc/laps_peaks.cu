// laps_peaks.cu -- throughput probes of this GPU: the denominators of the
// kernels' roofline fractions that no vendor table states for the clock the
// GPU actually runs at.  FP32 and FP64 fused multiply-add throughput, the
// special-function unit's base-2 exponential, and the latency of the grid
// barrier the persistent kernels use (laps_device.cuh), each timed with CUDA
// events; the SM clock is read inside the probes (cycle counter against the
// global nanosecond timer).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "laps_device.cuh"
#include "laps_internal.h"

namespace laps {
namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// clock of the SM running block 0, measured over the probe: cycles and ns
__device__ __forceinline__ void clock_mark(unsigned long long* clk, int slot) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[2 * slot] = (unsigned long long)clock64();
        clk[2 * slot + 1] = global_ns();
    }
}

__global__ void fma32_kernel(float* out, int iters, unsigned long long* clk) {
    clock_mark(clk, 0);
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
    const float b = 0.9999f, c = 1e-4f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live
    clock_mark(clk, 1);
}

__global__ void fma64_kernel(double* out, int iters) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    const double b = 0.9999, c = 1e-4;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678) out[blockIdx.x] = s;
}

__global__ void ex2_kernel(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = -1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            a[k] = -r;  // x -> -2^x stays in [-1, 0)
        }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// n_bar grid barriers back to back across a cooperative launch
__global__ void barrier_kernel(unsigned* count, int* status, int n_bar, long long timeout_ns) {
    for (int k = 1; k <= n_bar; ++k)
        if (!grid_sync_count(count, status, (unsigned)k * gridDim.x, timeout_ns)) return;
}

template <class F>
cudaError_t timed_ms(F launch, cudaStream_t st, float* ms) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    e = launch();  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

}  // namespace
}  // namespace laps

using namespace laps;

extern "C" laps_status laps_measure_peaks(laps_peaks* out, void* stream) {
    if (!out) return fail(LAPS_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    laps_peaks p{};
    p.sm_count = nsm;
    float* fbuf = nullptr;
    double* dbuf = nullptr;
    unsigned long long* clk = nullptr;
    unsigned* count = nullptr;
    int* status = nullptr;
    const int blocks = 8 * nsm, threads = 256;
    e = cudaMalloc(&fbuf, blocks * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dbuf, blocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&clk, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&count, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    float ms = 0.0f;
    // FP32: blocks x threads x kChains x iters FMAs, 2 FLOP each
    const int it32 = 4096;
    if (e == cudaSuccess)
        e = timed_ms([&] {
                fma32_kernel<<<blocks, threads, 0, st>>>(fbuf, it32, clk);
                return cudaGetLastError();
            }, st, &ms);
    if (e == cudaSuccess) {
        p.fp32_tflops = 2.0 * blocks * threads * kChains * (double)it32 / (ms * 1e-3) / 1e12;
        unsigned long long h[4];
        e = cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && h[3] > h[1]) p.sm_mhz = (double)(h[2] - h[0]) / (double)(h[3] - h[1]) * 1e3;
    }
    const int it64 = 256;
    if (e == cudaSuccess)
        e = timed_ms([&] {
                fma64_kernel<<<blocks, threads, 0, st>>>(dbuf, it64);
                return cudaGetLastError();
            }, st, &ms);
    if (e == cudaSuccess) p.fp64_tflops = 2.0 * blocks * threads * kChains * (double)it64 / (ms * 1e-3) / 1e12;
    const int itx = 1024;
    if (e == cudaSuccess)
        e = timed_ms([&] {
                ex2_kernel<<<blocks, threads, 0, st>>>(fbuf, itx);
                return cudaGetLastError();
            }, st, &ms);
    if (e == cudaSuccess && p.sm_mhz > 0.0)
        p.ex2_per_clk_sm = (double)blocks * threads * kChains * itx / (ms * 1e-3) / (p.sm_mhz * 1e6) / nsm;
    // grid barrier: one block per SM, all co-resident (cooperative launch)
    const int n_bar = 2000;
    long long tmo = 2000000000LL;
    if (e == cudaSuccess)
        e = timed_ms([&] {
                cudaError_t r = cudaMemsetAsync(count, 0, sizeof(unsigned), st);
                if (r == cudaSuccess) r = cudaMemsetAsync(status, 0, sizeof(int), st);
                int nb = n_bar;
                void* args[] = {&count, &status, &nb, &tmo};
                if (r == cudaSuccess)
                    r = cudaLaunchCooperativeKernel((void*)barrier_kernel, dim3(nsm), dim3(threads), args, 0, st);
                return r;
            }, st, &ms);
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        p.grid_barrier_us = hs == ST_OK ? (double)ms * 1e3 / n_bar : -1.0;
        p.barrier_blocks = nsm;
    }
    cudaFree(fbuf);
    cudaFree(dbuf);
    cudaFree(clk);
    cudaFree(count);
    cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(e, "laps_measure_peaks");
    if (hs != ST_OK) return status_error(hs);
    *out = p;
    return LAPS_OK;
}
