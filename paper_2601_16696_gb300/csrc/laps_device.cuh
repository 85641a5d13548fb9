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
enum : int { ST_OK = 0, ST_BADPARAM = 1, ST_TIMEOUT = 4, ST_NONFINITE = 5, ST_OVERFLOW = 6 };

// ---------------------------------------------------------------- Philox4x32-10
// Ten rounds; each multiplies words 0 and 2 by the round multipliers, xors the
// high halves into the other words with the round key, bumps the key by the
// Weyl increments.  Counter = (coordinate block, chain, step, tag | pid << 8),
// key = (seed low, seed high).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// (r >> 9) + 1/2 scaled by 2^-23: a binary32 value in (0, 1), exact.
__device__ __forceinline__ float u01(uint32_t r) {
    return (static_cast<float>(r >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// Four standard normals for coordinates 4j..4j+3 (Box-Muller on (r0,r1), (r2,r3)).
__device__ __forceinline__ void normals4(uint32_t j, uint32_t m, uint32_t t, uint32_t tagpid,
                                         uint32_t k0, uint32_t k1, float z[4]) {
    const uint4 r = philox4x32_10(make_uint4(j, m, t, tagpid), k0, k1);
    float s, c;
    float rad = sqrtf(-2.0f * logf(u01(r.x)));
    sincospif(2.0f * u01(r.y), &s, &c);
    z[0] = rad * c;
    z[1] = rad * s;
    rad = sqrtf(-2.0f * logf(u01(r.z)));
    sincospif(2.0f * u01(r.w), &s, &c);
    z[2] = rad * c;
    z[3] = rad * s;
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
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v || w != w) ? w : v;  // NaN propagates
    }
    return v;
}

// ---------------------------------------------------------------- fixed point
// Exact, order-independent accumulation across blocks: a value is converted to
// a 128-bit two's-complement integer with FX_FRAC = 48 fractional bits
// (resolution 2^-48 ~ 3.6e-15, range |v| < 2^77 ~ 1.5e23), split into four
// 32-bit limbs, and each limb is added with a 64-bit integer atomic into its
// own accumulator.  Integer addition commutes, so the totals, and everything
// computed from them, are bit-identical from run to run whatever order the
// blocks arrive in.  A value outside the range (or not finite) raises `bad`.
constexpr int FX_FRAC = 48;
struct i128 {
    unsigned long long lo;
    long long hi;
};
__device__ __forceinline__ i128 f32_to_fx(float f, int& bad) {
    i128 r{0ull, 0ll};
    const unsigned b = __float_as_uint(f);
    const int e = (b >> 23) & 0xff;
    if (e == 0) return r;  // zero or subnormal: below the resolution
    if (e == 0xff) { bad = 1; return r; }
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;  // |f| = m 2^(e-150)
    const int sh = e - 150 + FX_FRAC;  // bit position of m's lsb in |f| 2^FX_FRAC
    if (sh < 0) {
        if (sh > -24) r.lo = m >> (-sh);
    } else if (sh < 64) {
        r.lo = m << sh;
        r.hi = (sh > 40) ? (long long)(m >> (64 - sh)) : 0ll;
    } else if (sh < 64 + 38) {
        r.hi = (long long)(m << (sh - 64));
    } else {
        bad = 1;
        return r;
    }
    if (b >> 31) {  // two's-complement negation
        r.lo = ~r.lo + 1ull;
        r.hi = ~r.hi + (r.lo == 0ull ? 1ll : 0ll);
    }
    return r;
}
__device__ __forceinline__ i128 fx_add(i128 a, i128 b) {
    i128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ll : 0ll);
    return r;
}
// Each limb accumulator sits alone in a 128-byte line (FX_STRIDE u64 apart):
// integer atomics to one L2 line serialise, so limbs sharing lines would make
// every block's additions queue behind each other.
constexpr int FX_STRIDE = 16;
// acc: the four limb accumulators of one quantity, FX_STRIDE apart
__device__ __forceinline__ void fx_atomic_add(unsigned long long* acc, ff v, int& bad) {
    const i128 x = fx_add(f32_to_fx(v.hi, bad), f32_to_fx(v.lo, bad));
    atomicAdd(acc + 0 * FX_STRIDE, x.lo & 0xffffffffull);
    atomicAdd(acc + 1 * FX_STRIDE, x.lo >> 32);
    atomicAdd(acc + 2 * FX_STRIDE, (unsigned long long)x.hi & 0xffffffffull);
    atomicAdd(acc + 3 * FX_STRIDE, (unsigned long long)(x.hi >> 32));  // signed limb
}
// total of the four limb sums: exact 128-bit integer, then to FP64 (53 bits)
// and split into a float-float
__device__ __forceinline__ ff fx_read(const unsigned long long* acc) {
    const unsigned long long a0 = __ldcg(acc + 0 * FX_STRIDE), a1 = __ldcg(acc + 1 * FX_STRIDE);
    const unsigned long long a2 = __ldcg(acc + 2 * FX_STRIDE);
    const long long a3 = (long long)__ldcg(acc + 3 * FX_STRIDE);
    const unsigned long long t0 = a0;
    const unsigned long long t1 = a1 + (t0 >> 32);
    const unsigned long long t2 = a2 + (t1 >> 32);
    const long long t3 = a3 + (long long)(t2 >> 32);
    const unsigned long long lo = (t0 & 0xffffffffull) | (t1 << 32);
    const long long hi = (long long)((t2 & 0xffffffffull) | ((unsigned long long)t3 << 32));
    // value = (hi 2^64 + lo) 2^-48 = hi 2^16 + lo 2^-48
    const double v = fma((double)hi, 65536.0, (double)lo * 3.552713678800501e-15);
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
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
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// Grid-wide barrier on a monotone arrival counter (reset to 0 before the
// launch): barrier number k (k = 1, 2, ...) waits until the counter reaches
// k * expected.  One atomic per block and a polling read; no reset between
// barriers.  Bounded exactly like grid_barrier below.
__device__ __forceinline__ bool grid_sync_count(unsigned* count, int* status, unsigned target,
                                                long long timeout_ns) {
    __shared__ int s_ok2;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
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
        __threadfence();
        if (ok && ld_volatile_i32(status) != ST_OK) ok = 0;
        s_ok2 = ok;
    }
    __syncthreads();
    return s_ok2 != 0;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: after timeout_ns the block records ST_TIMEOUT in *status
// and returns false, as does every block that sees a recorded error, so the
// kernel always terminates.  Returns true when all blocks arrived.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, int* status,
                                             unsigned nblocks, long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g0 = ld_acquire_u32(gen);
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == nblocks - 1) {
            *count = 0u;
            __threadfence();
            st_release_u32(gen, g0 + 1u);
        } else {
            const uint64_t t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(gen) == g0) {
                if ((++spins & 63u) == 0u) {
                    if (ld_volatile_i32(status) != ST_OK) { ok = 0; break; }
                    if ((long long)(global_ns() - t0) > timeout_ns) {
                        atomicCAS(status, ST_OK, ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        if (ok && ld_volatile_i32(status) != ST_OK) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace laps
