// Test-only: Philox4x32-10 as cuRAND's device header computes it, so that the
// oracle's restatement of Salmon et al. (SC'11) can be checked against an
// implementation this repository did not write.  Built by the test that uses it.
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>
#include <stdint.h>

__global__ void curand_philox_kernel(const uint4* ctr, const uint2* key, uint4* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// ctr: device [n][4] counters, key: device [n][2] keys, out: device [n][4].
// Returns the cudaError_t of the launch (0 on success); stream-ordered.
extern "C" int curand_philox_ref(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                                 void* stream) {
    if (n <= 0) return 0;
    int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    curand_philox_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        (const uint4*)ctr, (const uint2*)key, (uint4*)out, n);
    return (int)cudaGetLastError();
}
