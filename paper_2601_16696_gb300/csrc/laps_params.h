// laps_params.h -- parameter and state blocks shared by the host API and the
// kernels (plain structs, no CUDA types beyond the vector types).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/laps.h"

#ifndef LAPS_PHASE_BLOCK
#define LAPS_PHASE_BLOCK 0  // diagnostic builds: the block whose phases are timed
#endif

namespace laps {

// Hyperparameters and phase machine of Alg. 1 (identical in every block).
struct Hyper {
    float eps, L, lo, hi, a_target, eps_used;
    float eevpd, eevpd_wanted, dtilde, max_delta, acc, b2_max, b2_avg, sum_var;
    double b2_first_ns;
    long long grads, b2_first_grads;
    unsigned long long t0_ns;
    int phase, t, t_switch, integ, adapting, p, done, iters, win_n, nonfinite_total;
    int nonfinite_last, b2_first_t;
};

enum : int { TGT_GAUSS = 0, TGT_BANANA = 1, TGT_FUNNEL = 2, TGT_LOGREG = 3, TGT_GAUSS_DENSE = 4, TGT_USER = 5 };
enum : int { INTEG_LF = 0, INTEG_MN2 = 1, INTEG_MN4 = 2 };
enum : int { TAG_X0 = 0, TAG_O1 = 1, TAG_O2 = 2, TAG_REFRESH = 3, TAG_MH = 4, TAG_Z = 5 };

// per-coordinate sums (y, y^2, g, y g) and per-chain sums kept per iteration
enum : int { NQ = 4 };
enum : int { CS_DSUM = 0, CS_DSQ, CS_NFIN, CS_NBAD, CS_ASUM, NCS };
enum : int { NCSF = 6 };  // floats per chain slot in shared memory (Delta as hi, lo)
// per-coordinate results of the slice owners: Var y, Var x, (1 - V)^2, delta, b^2
// (slot 5: the full-rank proxy's sum over k; 6, 7: ensemble means of y and g, kept
// for the next iteration's full-rank block products)
enum : int { CO_VARY = 0, CO_VARX, CO_DV, CO_DEL, CO_B2, NCO = 8 };
enum : int { SL_VAR = 0, SL_DV, SL_MAXDEL, SL_B2SUM, SL_B2MAX, NSL };

struct KParams {
    // problem
    int M, d, d_pad, nblk;
    int kind;
    float inv_s2;       // banana: 1 / sb^2
    float inv_sv2;      // funnel: 1 / sv^2
    const float* prec;  // gauss: [d_pad], zero padded
    // ensemble state, sampler coordinates, [M][d_pad]
    float *y, *u, *g;
    float2* logp_ff;    // [M] log p as float-float
    float* sigma;       // [d_pad] preconditioner (1 before the switch)
    const float* x0;    // init: [M][d] caller layout, or nullptr for Philox
    float x0_scale;
    // reduction and window state (global)
    float2* part;             // [NQ * d_pad + NCS][G] per-block float-float sums (+ full-rank records)
    float* cstat;             // [d_pad][NCO] per-coordinate results of the slice owners
    float2* ctot;             // [NCS] chain totals (written by the last block)
    float2* ring;             // [T + 1][d_pad] window values E[x_i^2] (float-float)
    float4* win_sums;         // [d_pad] running window sums (s1, s2 as float-float)
    const float2* Ex2;        // [d_pad] truth E_p[x_i^2] (float-float) or nullptr
    const float* inv_varx2;   // [d_pad] 1 / Var_p[x_i^2]
    Hyper* hyper;
    laps_trace_row* trace;
    int trace_cap;
    unsigned* bar_count;
    int* status;
    // configuration
    float C, alpha, switch_tol, acc_tol, adj_L_factor, eps0, a_target_mn2, a_target_mn4;
    float stop_b2, fixed_eps;
    int stop_b2_max;
    int T, n_total, N, mn4_min_dim, eevpd_centered, adjusted, force_switch_at;
    long long timeout_ns;
    uint32_t seed_lo, seed_hi, pid;
    int mode;       // 0: initialise, 1: iterate
    int n_iters;    // iterations of this launch
    int G;          // blocks in the grid
    int qpp;        // per-coordinate quantities reduced per shared-memory pass
    int smax;       // largest coordinate slice of a block
    int bar_extra;  // extra arrivals every barrier waits for (test hook; 0 normally)
    unsigned long long* phase_ns;  // diagnostic build only: [5] time per phase
    // streamed path: the state lives in global memory and the gradient comes
    // from a separate kernel (y, u, g, logp_ff above are the accepted state)
    float *yw, *uw;           // [M][d_pad] working position / velocity of the iteration
    float2* dlw;              // [M] energy error of the iteration so far (float-float)
    float2* lpw;              // [M] log p at yw (float-float)
    float* W;                 // [M][d_pad] x = sigma o yw, the gradient kernel's input
    const float* gpart;       // [S][M][d_pad] x-space gradient partials of the gradient kernel
    const float2* lpart;      // [S][M] log p partials
    int nsplit;               // S
    int* go;                  // [2]: the iteration is live; it switched to the adjusted phase
    void* Wb;                 // mixed precision: [M_pad][2 d_pad] BF16 (hi | lo) copy of W
    int gauss_derived;        // batched diagonal Gaussians: only y, y^2 are summed per coordinate
    int dfull_K;              // > 0: full-rank D~ over this many Rademacher vectors (else diagonal)
    // chain-sharded ensemble (streamed path): this context holds chains m0 .. m0 + M - 1 of an
    // ensemble of Mn chains; the Philox counters carry the global index, the finalise divides
    // by Mn.  m0 = 0, Mn = 0 (meaning M): the whole ensemble.
    int m0, Mn;
};
// chains of the whole ensemble (the finalise's normalisation)
__host__ __device__ inline int ens_chains(const KParams& P) { return P.Mn > 0 ? P.Mn : P.M; }

// per-coordinate result slot of the full-rank bias proxy: sum_k (z_ki + c_ik)^2,
// and the ensemble means E[y_i], E[g_i] it centres the next iteration on
enum : int { CO_DFULL = 5, CO_MY = 6, CO_MG = 7 };
// rows of the per-block columns: NQ d_pad coordinate rows, NCS chain rows
__host__ __device__ inline size_t rows_fb(int d_pad) { return (size_t)NQ * d_pad + NCS; }

// The full-rank proxy's per-block records (K vectors) follow the rows, 16-byte
// aligned: one record of fr_stride() floats per block b.  With the common shifts
// ybar', gbar' (the previous iteration's ensemble means, the same in every block),
// y' = y - ybar' and s'_k = (g - gbar') . z_k:
//   [d_pad][K4]  Q_ik = sum_{m in b} y'_mi s'_mk
//   [K4]         sum_{m in b} s'_mk
__host__ __device__ inline int fr_k4(int K) { return (K + 3) & ~3; }
__host__ __device__ inline size_t fr_stride(int d_pad, int K) {
    const size_t K4 = (size_t)fr_k4(K);
    return (size_t)d_pad * K4 + K4;
}
__host__ __device__ inline size_t fr_offset(int d_pad, int G) {  // bytes from the start of part
    return ((rows_fb(d_pad) * (size_t)G * 8 + 15) / 16) * 16;
}
__host__ __device__ inline size_t part_bytes(int d_pad, int G, int K) {
    return K > 0 ? fr_offset(d_pad, G) + (size_t)G * fr_stride(d_pad, K) * 4 : rows_fb(d_pad) * (size_t)G * 8;
}
// the block product s = G Z is split over this many ranges of coordinates when its
// 4 x 4 output tiles alone would leave threads idle
__host__ __device__ inline int fr_jsplit(int d_pad, int slots, int K, int threads) {
    const int tiles = ((slots + 3) / 4) * (fr_k4(K) / 4);
    int js = threads / (tiles > 0 ? tiles : 1);
    js = js < 8 ? js : 8;
    js = js < d_pad / 4 ? js : d_pad / 4;
    return js > 1 ? js : 1;
}
// shared memory of the dense-precision Gaussian on the resident kernel (bytes,
// after the reduction's slice rows): 16 bytes of alignment, P [d_pad][d_pad] and
// one [d_pad] row of x per chain slot
__host__ __device__ inline size_t dense_smem(int d_pad, int slots) {
    return 16 + 4 * ((size_t)d_pad * d_pad + (size_t)slots * d_pad);
}
// the largest padded dimension the resident kernel serves it for (P in shared memory)
constexpr int kDenseResidentMax = 128;

// shared memory of the full-rank proxy (bytes, after the reduction's slice rows):
// [smax K + 3 threads] float-float for the slice owners, 16 bytes of alignment,
// y and g [slots][d_pad], s [slots][K4], the shifts ybar' and gbar' [d_pad] each,
// Rademacher words [4 ceil(d_pad/128)][K4], partial products of s [jsplit - 1][slots][K4]
__host__ __device__ inline size_t fullrank_smem(int d_pad, int slots, int smax, int K, int threads) {
    if (K <= 0) return 0;
    const size_t K4 = (size_t)fr_k4(K), nzw = (size_t)((d_pad + 127) / 128) * 4;
    const size_t js = (size_t)fr_jsplit(d_pad, slots, K, threads);
    return ((size_t)smax * K + 3 * (size_t)threads) * 8 + 16 +
           4 * (2 * (size_t)slots * d_pad + js * (size_t)slots * K4 + 2 * (size_t)d_pad + nzw * K4);
}

// one launch of the streamed path's chain-update kernel: the maps it applies,
// in this order, to every chain (App. E "discrete update", App. F)
struct SegOp {
    int phase;       // phase of the iteration this launch belongs to
    int first;       // 1: first launch of the iteration (sets the guard, reads the accepted state)
    int init;        // 1: draw / copy x0;  2: finish the initialisation from the gradient;
                     // 3: gradient input from the accepted state;  4: accepted g, log p from
                     //    the gradient kernel (re-evaluation after a change of arithmetic)
    int refresh;     // 1: full refresh u = Z / |Z| (App. F step 2, tag 3)
    int after_grad;  // 1: take g and log p of the working point from the gradient kernel
    float bA;        // B_{bA eps} first (0: none)
    int o2_step;     // >= 0: O_{eps/2} of step t0 + o2_step (tag 2)
    int o1_step;     // >= 0: O_{eps/2} of step t0 + o1_step (tag 1)
    float bB;        // then B_{bB eps} (0: none)
    float a;         // then A_{a eps} and write the gradient input (0: none)
    int close;       // 1: last launch: non-finite check, MH test, keep / revert, block columns
};

}  // namespace laps
