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
};

// Largest padded dimension the gradient kernels take.
constexpr int kLogregMaxKp = 256;

// log p and gradient at the M points W [M][kp] (x-space, padding columns 0),
// with the data split into S row ranges: gpart [S][M][kp] and lpart [S][M]
// (float-float) receive the per-range sums; range 0 also carries the prior.
// The consumer adds the S partials in order.
cudaError_t logreg_grad_f32(const LogregData& D, const float* W, int64_t M, int S, float* gpart,
                            float2* lpart, cudaStream_t st);

}  // namespace laps
