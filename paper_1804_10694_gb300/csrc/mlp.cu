// Kernels of the tile-choice cost model: an MLP F -> 64 -> ReLU -> 64 -> ReLU
// -> 1 predicting log execution time (the paper autotunes tile sizes by
// search, Section VI-A; the learned model predicts the search's winner).
//
// Flat parameter layout: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
//
//   forward : one thread per sample, parameters staged in shared memory;
//             stores the pre-activations z1, z2 for the backward pass.
//   backward: one thread per sample computes dy = 2 (y - t) / n and the
//             pre-activation gradients dz2 = dy w3 [z2 > 0],
//             dz1 = W2^T dz2 [z1 > 0], written transposed ([H][n]) next to the
//             activations h1, h2 ([n][H]); the weight gradients are then
//             products over the batch, dW = dZ^T H (batch_outer_launch:
//             per-chunk partials summed in a fixed order).
//   mse     : one CTA, fixed summation order (deterministic).
//   adam    : elementwise Adam update (Kingma & Ba, Algorithm 1).
#include <cuda_runtime.h>

#include "mlp.h"

namespace gb {
namespace {

constexpr int H = kMlpHidden;

__host__ __device__ constexpr int param_count(int F) { return H * F + H + H * H + H + H + 1; }

template <int F>
__global__ void mlp_forward_kernel(const float* __restrict__ X, int n, const float* __restrict__ theta,
                                   float* __restrict__ y, float* __restrict__ Z1,
                                   float* __restrict__ Z2) {
  extern __shared__ float sp[];
  constexpr int P = param_count(F);
  for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = theta[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float* W1 = sp;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float b3 = w3[H];
  float x[F];
#pragma unroll
  for (int f = 0; f < F; ++f) x[f] = X[static_cast<int64_t>(s) * F + f];
  float h1[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float z = b1[j];
#pragma unroll
    for (int f = 0; f < F; ++f) z = fmaf(W1[j * F + f], x[f], z);
    if (Z1) Z1[static_cast<int64_t>(s) * H + j] = z;
    h1[j] = z > 0.0f ? z : 0.0f;
  }
  float out = b3;
  for (int j = 0; j < H; ++j) {
    float z = b2[j];
#pragma unroll
    for (int i = 0; i < H; ++i) z = fmaf(W2[j * H + i], h1[i], z);
    if (Z2) Z2[static_cast<int64_t>(s) * H + j] = z;
    out = fmaf(w3[j], z > 0.0f ? z : 0.0f, out);
  }
  y[s] = out;
}

template <int F>
__global__ void mlp_backward_sample_kernel(const float* __restrict__ t, int n,
                                           const float* __restrict__ theta, const float* __restrict__ y,
                                           const float* __restrict__ Z1, const float* __restrict__ Z2,
                                           float* __restrict__ dZ1T, float* __restrict__ dZ2T,
                                           float* __restrict__ H1, float* __restrict__ H2,
                                           float* __restrict__ dy) {
  extern __shared__ float sp[];
  constexpr int P = param_count(F);
  for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = theta[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float* W2 = sp + H * F + H;
  const float* w3 = W2 + H * H + H;
  const float d = 2.0f * (y[s] - t[s]) / static_cast<float>(n);
  dy[s] = d;
  float dz2[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const float z = Z2[static_cast<int64_t>(s) * H + j];
    dz2[j] = z > 0.0f ? d * w3[j] : 0.0f;
    dZ2T[static_cast<int64_t>(j) * n + s] = dz2[j];
    H2[static_cast<int64_t>(s) * H + j] = z > 0.0f ? z : 0.0f;
  }
  for (int i = 0; i < H; ++i) {
    float g = 0.0f;
#pragma unroll
    for (int j = 0; j < H; ++j) g = fmaf(W2[j * H + i], dz2[j], g);
    const float z = Z1[static_cast<int64_t>(s) * H + i];
    dZ1T[static_cast<int64_t>(i) * n + s] = z > 0.0f ? g : 0.0f;
    H1[static_cast<int64_t>(s) * H + i] = z > 0.0f ? z : 0.0f;
  }
}

__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int n,
                           float* __restrict__ out) {
  __shared__ float part[1024];
  float acc = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = y[i] - t[i];
    acc = fmaf(d, d, acc);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0] / static_cast<float>(n);
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int P, float lr, float b1,
                            float b2, float eps, float corr1, float corr2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / corr1) / (sqrtf(vi / corr2) + eps);
  }
}

// Products over the batch, out[r][c] = sum_i A[r lda + i] B[i ldb + c]
// (r < R <= 64, c < C <= 64): CTA p sums samples [p kOuterChunk, ...) into
// partial p, staging 32 samples of both operands in shared memory per step;
// a second kernel adds the partials in increasing p (a fixed order, so the
// gradient does not depend on timing).
constexpr int kOuterChunk = 512;

__global__ void __launch_bounds__(256) outer_partial_kernel(const float* __restrict__ A, int lda,
                                                            const float* __restrict__ B, int ldb,
                                                            int R, int C, int n,
                                                            float* __restrict__ part) {
  __shared__ float sA[64][33];
  __shared__ float sB[32][65];
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * kOuterChunk;
  const int i1 = min(n, i0 + kOuterChunk);
  const int m = R * C;
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
  for (int s0 = i0; s0 < i1; s0 += 32) {
    for (int idx = t; idx < R * 32; idx += 256) {
      const int r = idx >> 5, j = idx & 31;
      sA[r][j] = s0 + j < i1 ? A[static_cast<int64_t>(r) * lda + s0 + j] : 0.0f;
    }
    for (int idx = t; idx < 32 * C; idx += 256) {
      const int j = idx / C, c = idx - j * C;
      sB[j][c] = s0 + j < i1 ? B[static_cast<int64_t>(s0 + j) * ldb + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int o = t + 256 * k;
      if (o < m) {
        const int r = o / C, c = o - r * C;
        float a = acc[k];
#pragma unroll 8
        for (int j = 0; j < 32; ++j) a = fmaf(sA[r][j], sB[j][c], a);
        acc[k] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int o = t + 256 * k;
    if (o < m) part[static_cast<int64_t>(blockIdx.x) * m + o] = acc[k];
  }
}

__global__ void sum_partials_kernel(const float* __restrict__ part, int nparts, int m,
                                    float* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= m) return;
  float s = 0.0f;
  for (int p = 0; p < nparts; ++p) s += part[static_cast<int64_t>(p) * m + o];
  out[o] = s;
}

__global__ void fill_value_kernel(float* x, int n, float v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

}  // namespace

int mlp_param_count() { return param_count(kFeatures); }

cudaError_t mlp_forward_launch(const float* X, int n, const float* theta, float* y, float* Z1,
                               float* Z2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int smem = param_count(kFeatures) * sizeof(float);
  mlp_forward_kernel<kFeatures><<<(n + 127) / 128, 128, smem, s>>>(X, n, theta, y, Z1, Z2);
  return cudaGetLastError();
}

cudaError_t mlp_backward_sample_launch(const float* t, int n, const float* theta, const float* y,
                                       const float* Z1, const float* Z2, float* dZ1T, float* dZ2T,
                                       float* H1, float* H2, float* dy, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int smem = param_count(kFeatures) * sizeof(float);
  mlp_backward_sample_kernel<kFeatures><<<(n + 127) / 128, 128, smem, s>>>(t, n, theta, y, Z1, Z2, dZ1T,
                                                                          dZ2T, H1, H2, dy);
  return cudaGetLastError();
}

cudaError_t mse_launch(const float* y, const float* t, int n, float* out, cudaStream_t s) {
  mse_kernel<<<1, 1024, 0, s>>>(y, t, n, out);
  return cudaGetLastError();
}

cudaError_t adam_launch(float* theta, const float* g, float* m, float* v, int P, int step, float lr,
                        float b1, float b2, float eps, cudaStream_t s) {
  // bias corrections 1 - beta^step, computed once on the host in double
  double c1 = 1.0, c2 = 1.0, p1 = 1.0, p2 = 1.0;
  for (int i = 0; i < step; ++i) p1 *= b1, p2 *= b2;
  c1 -= p1;
  c2 -= p2;
  adam_kernel<<<(P + 255) / 256, 256, 0, s>>>(theta, g, m, v, P, lr, b1, b2, eps, (float)c1, (float)c2);
  return cudaGetLastError();
}

int batch_outer_parts(int n) { return (n + kOuterChunk - 1) / kOuterChunk; }

cudaError_t batch_outer_launch(const float* A, int lda, const float* B, int ldb, int R, int C, int n,
                               float* part, float* out, cudaStream_t s) {
  if (R < 1 || R > 64 || C < 1 || C > 64 || n < 1) return cudaErrorInvalidValue;
  const int parts = batch_outer_parts(n);
  outer_partial_kernel<<<parts, 256, 0, s>>>(A, lda, B, ldb, R, C, n, part);
  sum_partials_kernel<<<(R * C + 255) / 256, 256, 0, s>>>(part, parts, R * C, out);
  return cudaGetLastError();
}

cudaError_t fill_value_launch(float* x, int n, float v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fill_value_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(x, n, v);
  return cudaGetLastError();
}

}  // namespace gb
