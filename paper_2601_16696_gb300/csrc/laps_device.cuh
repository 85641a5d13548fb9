// laps_device.cuh -- device building blocks of the LAPS kernels (sm_103a).
//
// Counter-based noise (Philox4x32-10, Salmon et al. SC'11) with Box-Muller
// normals; compensated float-float sums (TwoSum, Knuth) for the per-chain
// log-density and energy error; sub-warp reductions; and a grid barrier whose
// wait is bounded by %globaltimer so that no launch can hang the GPU.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace laps {

// ---------------------------------------------------------------- status codes
enum : int { ST_OK = 0, ST_BADPARAM = 1, ST_TIMEOUT = 4, ST_NONFINITE = 5 };

// ---------------------------------------------------------------- Philox4x32-10
// Ten rounds; each multiplies words 0 and 2 by the round multipliers, xors the
// high halves into the other words with the round key, bumps the key by the
// Weyl increments.  Counter = (coordinate block, chain, step, tag | pid << 8),
// key = (seed low, seed high).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per word: both halves from one multiply
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The ten round keys of key (k0, k1): round r xors with (k0 + r W0, k1 + r W1)
// (the Weyl increments above).  A kernel that takes them as a parameter finds
// them in the constant bank, so a round needs no key additions.
struct PhiloxKeys {
    uint32_t k[20];
};
__host__ __device__ inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys K;
    for (int r = 0; r < 10; ++r) {
        K.k[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        K.k[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ K.k[2 * r], lo1, hi0 ^ c.w ^ K.k[2 * r + 1], lo0);
    }
    return c;
}

// ((r >> 9) + 1/2) 2^-23 = (r >> 9) 2^-23 + 2^-24: a binary32 value in (0, 1), exact.
// The 23 bits become the fraction of 1 + (r >> 9) 2^-23 in [1, 2); subtracting
// 1 - 2^-24 (0x3F7FFFFF) is exact, since the result (2 (r >> 9) + 1) 2^-24 has a
// 24-bit significand.  No integer-to-float conversion.
__device__ __forceinline__ float u01(uint32_t r) {
    return __uint_as_float(0x3F800000u | (r >> 9)) - 0.99999994039535522f;
}

// sqrt(-2 ln u) for u in (0, 1): the argument is > 0, so x rsqrt(x) is finite;
// rsqrtf is within 2 ulp, the product within ~3 ulp (4e-7 relative).
__device__ __forceinline__ float bm_radius(float u) {
    const float x = -2.0f * logf(u);
    return x * rsqrtf(x);
}

// cos(2 pi u) and sin(2 pi u) for u in (0, 1) from the hardware sine / cosine
// on theta = pi (2u - 1) in (-pi, pi) (2u - 1 is exact here), where their
// absolute error is about 2^-21: cos(2 pi u) = -cos(theta), sin = -sin(theta).
__device__ __forceinline__ void cos_sin_2pi(float u, float& c, float& s) {
    float st, ct;
    __sincosf(3.14159265358979323846f * fmaf(2.0f, u, -1.0f), &st, &ct);
    c = -ct;
    s = -st;
}

// Four standard normals for coordinates 4j..4j+3 (Box-Muller on (r0,r1), (r2,r3)).
__device__ __forceinline__ void box_muller4(const uint4 r, float z[4]) {
    float s, c;
    float rad = bm_radius(u01(r.x));
    cos_sin_2pi(u01(r.y), c, s);
    z[0] = rad * c;
    z[1] = rad * s;
    rad = bm_radius(u01(r.z));
    cos_sin_2pi(u01(r.w), c, s);
    z[2] = rad * c;
    z[3] = rad * s;
}
__device__ __forceinline__ void normals4(uint32_t j, uint32_t m, uint32_t t, uint32_t tagpid,
                                         const PhiloxKeys& K, float z[4]) {
    box_muller4(philox4x32_10(make_uint4(j, m, t, tagpid), K), z);
}
__device__ __forceinline__ void normals4(uint32_t j, uint32_t m, uint32_t t, uint32_t tagpid,
                                         uint32_t k0, uint32_t k1, float z[4]) {
    const uint4 r = philox4x32_10(make_uint4(j, m, t, tagpid), k0, k1);
    float s, c;
    float rad = bm_radius(u01(r.x));
    cos_sin_2pi(u01(r.y), c, s);
    z[0] = rad * c;
    z[1] = rad * s;
    rad = bm_radius(u01(r.z));
    cos_sin_2pi(u01(r.w), c, s);
    z[2] = rad * c;
    z[3] = rad * s;
}

// Rademacher entry z_k,i (full-rank bias proxy) of step t: bit (i mod 32) of word
// (i / 32 mod 4) of Philox(counter (i / 128, k, t, 5 | pid << 8)); set means +1.
__device__ __forceinline__ float rademacher(uint32_t i, uint32_t k, uint32_t t, uint32_t pid,
                                            uint32_t k0, uint32_t k1) {
    const uint4 r = philox4x32_10(make_uint4(i >> 7, k, t, 5u | (pid << 8)), k0, k1);
    const uint32_t sel = (i >> 5) & 3u;
    const uint32_t w = sel == 0 ? r.x : sel == 1 ? r.y : sel == 2 ? r.z : r.w;
    return ((w >> (i & 31u)) & 1u) ? 1.0f : -1.0f;
}

// ---------------------------------------------------------------- float-float
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }
// exact sum of two floats as hi + lo (TwoSum); symmetric in its arguments
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    const float hi = s + e;
    return ff{hi, e - (hi - s)};
}
__device__ __forceinline__ ff ff_add(ff a, float b) { return ff_add(a, ff{b, 0.0f}); }
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------- reductions
// Sum over the LPC lanes of a chain's group (xor butterfly: every lane of the
// group ends with the same bits, since each level adds a commutative pair).
template <int LPC>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int LPC>
__device__ __forceinline__ ff group_sum_ff(ff v) {
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}
// Sum over the groups of a warp of the values held by lanes with equal
// in-group index (same coordinates of different chains).
template <int LPC>
__device__ __forceinline__ float across_groups(float v) {
#pragma unroll
    for (int o = LPC; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// ---------------------------------------------------------------- timers, barrier
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident) on a
// monotone arrival counter (reset to 0 before the launch): barrier number k
// (k = 1, 2, ...) waits until the counter reaches k * expected.  One release
// reduction per block and acquire polling; no reset between barriers.  The
// block's writes reach other blocks through the release: __syncthreads orders
// them before thread 0's release reduction, which is cumulative; on the way out
// thread 0's acquire load (it reads the count the last arrival's reduction
// left, so it synchronises with every block's release), then __syncthreads,
// orders the block's later reads after the other blocks' releases.  So no
// separate fences (measured over 128 blocks: 1.42 us per barrier with fences,
// 1.19 without; whole banana run 32.2 -> 31.1 ms).  The wait is bounded: after timeout_ns
// the block records ST_TIMEOUT in *status and returns false, as does every
// block that sees a recorded error, so the kernel always terminates.
// The barrier comes in two halves, for a block that has work touching no other
// block's data to do while the others arrive: grid_arrive (all threads), that
// work, then grid_wait (all threads); grid_sync_count is the two back to back.
__device__ __forceinline__ void grid_arrive(unsigned* count) {
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
}
__device__ __forceinline__ bool grid_wait(const unsigned* count, int* status, unsigned target,
                                          long long timeout_ns) {
    __shared__ int s_ok2;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_u32(count) < target) {
            const uint64_t t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(count) < target) {
                if ((++spins & 31u) == 0u) {
                    if (ld_volatile_i32(status) != ST_OK) { ok = 0; break; }
                    if ((long long)(global_ns() - t0) > timeout_ns) {
                        atomicCAS(status, ST_OK, ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (ok && ld_volatile_i32(status) != ST_OK) ok = 0;
        s_ok2 = ok;
    }
    __syncthreads();
    return s_ok2 != 0;
}
__device__ __forceinline__ bool grid_sync_count(unsigned* count, int* status, unsigned target,
                                                long long timeout_ns) {
    grid_arrive(count);
    return grid_wait(count, status, target, timeout_ns);
}

}  // namespace laps
