// laps_logreg.cuh -- the Bayesian logistic-regression target (the paper's
// German Credit model, Sec. 6, on synthetic data):
//   log p(w) = sum_n [y_n z_n - softplus(z_n)] - |w|^2 / (2 v),   z = X w,
//   grad     = X^T (y - sigmoid(z)) - w / v.
// Over an ensemble W [M][kp] of points this is two chains-by-data
// contractions, Z = W X^T and G = R X with R = Y - sigmoid(Z); the kernels
// fuse them per tile of chains so that Z never reaches memory.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace laps {

// device copies a LOGREG target keeps (owned by laps_target)
struct LogregData {
    int n;            // data rows N
    int d;            // features (intercept included)
    int kp;           // padded feature count, a multiple of 64, >= d
    float* X;         // [n][kp] FP32, zero padded
    float* y;         // [n] labels
    float inv_v;      // 1 / prior variance
    // tensor-core form (kp <= 128): BF16 copies and their TMA descriptors
    int n_pad;        // n rounded up to the 64-row chunk
    void* Xb;         // [n_pad][kp] BF16
    void* Xtb;        // [kp][n_pad] BF16 (X transposed)
    alignas(64) unsigned char tmX[128];   // CUtensorMap of Xb
    alignas(64) unsigned char tmXt[128];  // CUtensorMap of Xtb
    // FP32-accurate tensor-core form: the three BF16 terms of X, [3][n_pad][kp]
    void* X3b;
    alignas(64) unsigned char tmX3[128];  // CUtensorMap of X3b
};

// Largest padded dimension the gradient kernels take.
constexpr int kLogregMaxKp = 256;

// ---- tensor-core (tcgen05, BF16) gradient: laps_logreg_mma.cu
bool logreg_mma_supported(int kp);
// BF16 copies of X and their tensor maps (allocates Xb, Xtb; synchronises)
cudaError_t logreg_mma_prepare(LogregData& D);
// tensor map of the [M_pad][2 kp] BF16 (hi | lo) copy of the points
cudaError_t logreg_mma_wmap(void* tmW, const void* Wb, int64_t M_pad, int kp);
// data splits of the launch (every split non-empty) and rows per split
int logreg_mma_splits(const LogregData& D, int64_t M, int nsm, int* rps);
// points [M][d] -> FP32 [M][kp] and BF16 hi | lo [M_pad][2 kp] (rows past M untouched)
cudaError_t logreg_pack_points(const float* x, int64_t M, int d, int kp, float* W32, void* Wb,
                               cudaStream_t st);
// gradient partials like logreg_grad_f32; W32 is the FP32 [M][kp] copy of the
// points (prior terms); a bounded wait that expires sets *status
cudaError_t logreg_grad_mma(const LogregData& D, const void* tmW, const float* W32, int64_t M, int S,
                            int rps, float* gpart, float2* lpart, int* status, long long timeout_ns,
                            cudaStream_t st, const int* guard = nullptr);

// ---- tensor-core gradient at FP32 accuracy (three-term BF16 split): laps_logreg_x3.cu
bool logreg_x3_supported(int kp);
// the split copy of X and its tensor map (allocates X3b; synchronises)
cudaError_t logreg_x3_prepare(LogregData& D);
size_t logreg_x3_smem(int kp);
// data splits of the launch (every split non-empty) and rows per split
int logreg_x3_splits(const LogregData& D, int64_t M, int nsm, int* rps);
// gradient partials like logreg_grad_f32 from the FP32 points W32 [M][kp], the
// data split by logreg_x3_splits; a bounded wait that expires sets *status
cudaError_t logreg_grad_x3(const LogregData& D, const float* W32, int64_t M, int S, int rps, float* gpart,
                           float2* lpart, int* status, long long timeout_ns, cudaStream_t st,
                           const int* guard = nullptr);

// log p and gradient at the M points W [M][kp] (x-space, padding columns 0),
// with the data split into S row ranges: gpart [S][M][kp] and lpart [S][M]
// (float-float) receive the per-range sums; range 0 also carries the prior.
// The consumer adds the S partials in order.  Every gradient entry point takes
// an optional guard: a device word that a launch earlier on the stream set to 0
// when this evaluation belongs to an iteration that no longer runs (past a stop
// or a switch); the kernel then returns at once.
cudaError_t logreg_grad_f32(const LogregData& D, const float* W, int64_t M, int S, float* gpart,
                            float2* lpart, cudaStream_t st, const int* guard = nullptr);
// The data split S of logreg_grad_f32 for M points on nsm SMs: the number of row
// ranges (1 .. 16) that minimises waves of blocks x rows per block, so that the
// last wave of chain tiles x ranges fills the GPU (M = 8192 on 152 SMs: 7).
int logreg_f32_splits(const LogregData& D, int64_t M, int nsm);

}  // namespace laps
