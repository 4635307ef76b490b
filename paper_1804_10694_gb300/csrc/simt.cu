// Plain FP32 CUDA-core gemm, the reference form of C = alpha * A * B + beta * C
// (the kind of kernel the paper generates for its GPU target, Section V-B).
//
// Two-level tiling: 128 x 128 output tiles per CTA, a 16-deep k-slice staged
// in shared memory (double buffered, next slice prefetched into registers
// while the current one is consumed), and register blocking of 8 x 8 outputs
// per thread.  Full tiles (all 128 rows and columns in range, k-slice
// complete) take unpredicated, vectorised loads when the leading dimensions
// allow it; partial tiles predicate every access.  The full/partial choice is
// uniform per CTA, so it introduces no divergence.  TA / TB: A stored K x M
// (lda >= M), B stored N x K (ldb >= K); the slices are loaded along the
// stored rows and land in the same shared-memory layout, so the arithmetic
// (and its order) is that of the untransposed kernel.
#include <cuda_runtime.h>

#include "internal.h"

namespace gb {

namespace {

// (a 16-deep slice reads 64 contiguous bytes of each row of A: 8192^3 ran at
// 55.3 TFLOP/s, against 52.8 with an 8-deep slice; two CTAs a SM)
constexpr int BM = 128, BN = 128, BKs = 16, THREADS = 256;

struct Frag {
  float a[8];
  float b[8];
};

// Four consecutive floats of a stored row (row r, columns c..c+3), in range
// when r < rows and c + i < cols.
template <bool FULL, bool VEC>
__device__ __forceinline__ void load4(float* v, const float* __restrict__ X, int64_t ld,
                                      int64_t r, int64_t c, int64_t rows, int64_t cols) {
  if (FULL && VEC) {
    const float4 q = *reinterpret_cast<const float4*>(X + r * ld + c);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else if (FULL) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = X[r * ld + c + i];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (r < rows && c + i < cols) ? X[r * ld + c + i] : 0.0f;
  }
}

// Load the A slice (128 rows x 16 k) and B slice (16 k x 128 cols) of one
// k-step into registers, along the stored rows.  A row-major: thread t loads
// row t/2, k (t%2)*8..+7; A stored K x M: k-rows t/32 and t/32 + 8, m
// (t%32)*4..+3.  B row-major: k-rows t/32 and t/32 + 8, columns
// (t%32)*4..+3; B stored N x K: column t/2, k (t%2)*8..+7.
template <bool FULL, bool VEC, bool TA, bool TB>
__device__ __forceinline__ void load_slice(Frag& f, const float* __restrict__ A, int64_t lda,
                                           const float* __restrict__ B, int64_t ldb, int64_t M,
                                           int64_t N, int64_t K, int64_t m0, int64_t n0,
                                           int64_t k0, int tid) {
  const int hi2 = tid >> 1, lo2 = (tid & 1) * 8;
  const int hi32 = tid >> 5, lo32 = (tid & 31) * 4;
  if (TA) {
    load4<FULL, VEC>(f.a, A, lda, k0 + hi32, m0 + lo32, K, M);
    load4<FULL, VEC>(f.a + 4, A, lda, k0 + hi32 + 8, m0 + lo32, K, M);
  } else {
    load4<FULL, VEC>(f.a, A, lda, m0 + hi2, k0 + lo2, M, K);
    load4<FULL, VEC>(f.a + 4, A, lda, m0 + hi2, k0 + lo2 + 4, M, K);
  }
  if (TB) {
    load4<FULL, VEC>(f.b, B, ldb, n0 + hi2, k0 + lo2, N, K);
    load4<FULL, VEC>(f.b + 4, B, ldb, n0 + hi2, k0 + lo2 + 4, N, K);
  } else {
    load4<FULL, VEC>(f.b, B, ldb, k0 + hi32, n0 + lo32, K, N);
    load4<FULL, VEC>(f.b + 4, B, ldb, k0 + hi32 + 8, n0 + lo32, K, N);
  }
}

// Into shared memory, As[k][m] and Bs[k][n] whatever the stored layout.
template <bool TA, bool TB>
__device__ __forceinline__ void store_slice(const Frag& f, float (*As)[BM], float (*Bs)[BN],
                                            int tid) {
  const int hi2 = tid >> 1, lo2 = (tid & 1) * 8;
  const int hi32 = tid >> 5, lo32 = (tid & 31) * 4;
  if (TA) {
    *reinterpret_cast<float4*>(&As[hi32][lo32]) = make_float4(f.a[0], f.a[1], f.a[2], f.a[3]);
    *reinterpret_cast<float4*>(&As[hi32 + 8][lo32]) = make_float4(f.a[4], f.a[5], f.a[6], f.a[7]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) As[lo2 + i][hi2] = f.a[i];
  }
  if (TB) {
#pragma unroll
    for (int i = 0; i < 8; ++i) Bs[lo2 + i][hi2] = f.b[i];
  } else {
    *reinterpret_cast<float4*>(&Bs[hi32][lo32]) = make_float4(f.b[0], f.b[1], f.b[2], f.b[3]);
    *reinterpret_cast<float4*>(&Bs[hi32 + 8][lo32]) = make_float4(f.b[4], f.b[5], f.b[6], f.b[7]);
  }
}

// As, Bs: the kernel's double-buffered shared slices ([2][BKs][BM] and
// [2][BKs][BN]), declared once for both tile paths.
template <bool FULL, bool VEC, bool TA, bool TB>
__device__ __forceinline__ void gemm_tile(int64_t M, int64_t N, int64_t K, float alpha,
                                          const float* __restrict__ A, int64_t lda,
                                          const float* __restrict__ B, int64_t ldb, float beta,
                                          float* __restrict__ C, int64_t ldc, int64_t m0,
                                          int64_t n0, bool cvec, float (*As)[BKs][BM],
                                          float (*Bs)[BKs][BN]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  const int64_t kfull = K / BKs;          // complete k-slices
  const int64_t ksteps = (K + BKs - 1) / BKs;
  Frag f;
  if (kfull > 0)
    load_slice<FULL, VEC, TA, TB>(f, A, lda, B, ldb, M, N, K, m0, n0, 0, tid);
  else
    load_slice<false, false, TA, TB>(f, A, lda, B, ldb, M, N, K, m0, n0, 0, tid);
  store_slice<TA, TB>(f, As[0], Bs[0], tid);
  __syncthreads();

  for (int64_t ks = 0; ks < ksteps; ++ks) {
    const int cur = ks & 1;
    const bool has_next = ks + 1 < ksteps;
    if (has_next) {
      if (ks + 1 < kfull)
        load_slice<FULL, VEC, TA, TB>(f, A, lda, B, ldb, M, N, K, m0, n0, (ks + 1) * BKs, tid);
      else
        load_slice<false, false, TA, TB>(f, A, lda, B, ldb, M, N, K, m0, n0, (ks + 1) * BKs, tid);
    }
#pragma unroll
    for (int k = 0; k < BKs; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (has_next) {
      store_slice<TA, TB>(f, As[cur ^ 1], Bs[cur ^ 1], tid);
      __syncthreads();
    }
  }

  // epilogue: rows ty*4+i (+64), columns tx*4+j (+64)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (!FULL && row >= M) continue;
    float* crow = C + row * ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t col = n0 + h * 64 + tx * 4;
      const float* a4 = &acc[i][h * 4];
      if (FULL && cvec) {
        float4* cp = reinterpret_cast<float4*>(crow + col);
        float4 o;
        if (beta != 0.0f) {
          const float4 old = *cp;
          o = make_float4(fmaf(alpha, a4[0], beta * old.x), fmaf(alpha, a4[1], beta * old.y),
                          fmaf(alpha, a4[2], beta * old.z), fmaf(alpha, a4[3], beta * old.w));
        } else {
          o = make_float4(alpha * a4[0], alpha * a4[1], alpha * a4[2], alpha * a4[3]);
        }
        *cp = o;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (FULL || col + j < N) {
            float* cp = crow + col + j;
            *cp = beta != 0.0f ? fmaf(alpha, a4[j], beta * *cp) : alpha * a4[j];
          }
        }
      }
    }
  }
}

template <bool VEC, bool TA, bool TB>
__global__ void __launch_bounds__(THREADS, 2) simt_gemm_kernel(int64_t M, int64_t N, int64_t K,
                                                            float alpha, const float* A,
                                                            int64_t lda, const float* B,
                                                            int64_t ldb, float beta, float* C,
                                                            int64_t ldc, bool cvec) {
  __shared__ __align__(16) float As[2][BKs][BM];
  __shared__ __align__(16) float Bs[2][BKs][BN];
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * BM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;
  if (m0 + BM <= M && n0 + BN <= N)
    gemm_tile<true, VEC, TA, TB>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, m0, n0, cvec, As, Bs);
  else
    gemm_tile<false, VEC, TA, TB>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, m0, n0, cvec, As, Bs);
}

template <bool TA, bool TB>
cudaError_t simt_launch(dim3 grid, bool vec, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                        int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                        bool cvec, cudaStream_t s) {
  if (vec)
    simt_gemm_kernel<true, TA, TB><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec);
  else
    simt_gemm_kernel<false, TA, TB><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec);
  return cudaGetLastError();
}

__global__ void scale_c_kernel(int64_t M, int64_t N, float beta, float* C, int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float* cp = C + (idx / N) * ldc + idx % N;
    *cp = beta != 0.0f ? beta * *cp : 0.0f;
  }
}

}  // namespace

cudaError_t simt_gemm_launch(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                             int64_t ldc, cudaStream_t s, bool transA, bool transB) {
  const dim3 grid(static_cast<unsigned>((N + BN - 1) / BN), static_cast<unsigned>((M + BM - 1) / BM));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) &&
                   (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(B) % 16 == 0);
  const bool cvec = (ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
  if (transA && transB) return simt_launch<true, true>(grid, vec, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec, s);
  if (transA) return simt_launch<true, false>(grid, vec, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec, s);
  if (transB) return simt_launch<false, true>(grid, vec, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec, s);
  return simt_launch<false, false>(grid, vec, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec, s);
}

cudaError_t scale_c_launch(int64_t M, int64_t N, float beta, float* C, int64_t ldc, cudaStream_t s) {
  const int64_t total = M * N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  scale_c_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(M, N, beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace gb
