// Launchers of the cost model's MLP kernels (mlp.cu).
#pragma once
#include <cuda_runtime.h>

#include "tuning.h"

namespace gb {

constexpr int kMlpHidden = kHidden;

int mlp_param_count();
// y = MLP(X) for n samples of kFeatures features; Z1, Z2 ([n][64]) receive
// the pre-activations when non-null.
cudaError_t mlp_forward_launch(const float* X, int n, const float* theta, float* y, float* Z1,
                               float* Z2, cudaStream_t s);
// Per-sample part of the backward pass of the MSE loss (see mlp.cu).
cudaError_t mlp_backward_sample_launch(const float* t, int n, const float* theta, const float* y,
                                       const float* Z1, const float* Z2, float* dZ1T, float* dZ2T,
                                       float* H1, float* H2, float* dy, cudaStream_t s);
cudaError_t mse_launch(const float* y, const float* t, int n, float* out, cudaStream_t s);
cudaError_t adam_launch(float* theta, const float* g, float* m, float* v, int P, int step, float lr,
                        float b1, float b2, float eps, cudaStream_t s);
cudaError_t fill_value_launch(float* x, int n, float v, cudaStream_t s);
// out[r][c] = sum_{i<n} A[r lda + i] B[i ldb + c] for r < R, c < C (both
// <= 64); part holds batch_outer_parts(n) * R * C floats of scratch.
int batch_outer_parts(int n);
cudaError_t batch_outer_launch(const float* A, int lda, const float* B, int ldb, int R, int C, int n,
                               float* part, float* out, cudaStream_t s);

}  // namespace gb
