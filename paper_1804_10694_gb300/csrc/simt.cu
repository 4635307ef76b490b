// Plain FP32 CUDA-core gemm, the reference form of C = alpha * A * B + beta * C
// (the kind of kernel the paper generates for its GPU target, Section V-B).
//
// Two-level tiling: 128 x 128 output tiles per CTA, an 8-deep k-slice staged
// in shared memory (double buffered, next slice prefetched into registers
// while the current one is consumed), and register blocking of 8 x 8 outputs
// per thread.  Full tiles (all 128 rows and columns in range, k-slice
// complete) take unpredicated, vectorised loads when the leading dimensions
// allow it; partial tiles predicate every access.  The full/partial choice is
// uniform per CTA, so it introduces no divergence.
#include <cuda_runtime.h>

#include "internal.h"

namespace gb {

namespace {

constexpr int BM = 128, BN = 128, BKs = 8, THREADS = 256;

struct Frag {
  float a[4];
  float b[4];
};

// Load the A slice (128 rows x 8 k) and B slice (8 k x 128 cols) of one k-step
// into registers.  Thread t loads A row t/2, k (t%2)*4..+3 and B k-row t/32,
// columns (t%32)*4..+3.
template <bool FULL, bool VEC>
__device__ __forceinline__ void load_slice(Frag& f, const float* __restrict__ A, int64_t lda,
                                           const float* __restrict__ B, int64_t ldb, int64_t M,
                                           int64_t N, int64_t K, int64_t m0, int64_t n0,
                                           int64_t k0, int tid) {
  const int ar = tid >> 1, ak = (tid & 1) * 4;
  const int bk = tid >> 5, bn = (tid & 31) * 4;
  const int64_t grow = m0 + ar, gka = k0 + ak;
  const int64_t gkb = k0 + bk, gcol = n0 + bn;
  if (FULL && VEC) {
    const float4 va = *reinterpret_cast<const float4*>(A + grow * lda + gka);
    f.a[0] = va.x, f.a[1] = va.y, f.a[2] = va.z, f.a[3] = va.w;
    const float4 vb = *reinterpret_cast<const float4*>(B + gkb * ldb + gcol);
    f.b[0] = vb.x, f.b[1] = vb.y, f.b[2] = vb.z, f.b[3] = vb.w;
  } else if (FULL) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f.a[i] = A[grow * lda + gka + i];
      f.b[i] = B[gkb * ldb + gcol + i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f.a[i] = (grow < M && gka + i < K) ? A[grow * lda + gka + i] : 0.0f;
      f.b[i] = (gkb < K && gcol + i < N) ? B[gkb * ldb + gcol + i] : 0.0f;
    }
  }
}

__device__ __forceinline__ void store_slice(const Frag& f, float (*As)[BM], float (*Bs)[BN],
                                            int tid) {
  const int ar = tid >> 1, ak = (tid & 1) * 4;
  const int bk = tid >> 5, bn = (tid & 31) * 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) As[ak + i][ar] = f.a[i];
  *reinterpret_cast<float4*>(&Bs[bk][bn]) = make_float4(f.b[0], f.b[1], f.b[2], f.b[3]);
}

template <bool FULL, bool VEC>
__device__ __forceinline__ void gemm_tile(int64_t M, int64_t N, int64_t K, float alpha,
                                          const float* __restrict__ A, int64_t lda,
                                          const float* __restrict__ B, int64_t ldb, float beta,
                                          float* __restrict__ C, int64_t ldc, int64_t m0,
                                          int64_t n0, bool cvec) {
  __shared__ __align__(16) float As[2][BKs][BM];
  __shared__ __align__(16) float Bs[2][BKs][BN];
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
    load_slice<FULL, VEC>(f, A, lda, B, ldb, M, N, K, m0, n0, 0, tid);
  else
    load_slice<false, false>(f, A, lda, B, ldb, M, N, K, m0, n0, 0, tid);
  store_slice(f, As[0], Bs[0], tid);
  __syncthreads();

  for (int64_t ks = 0; ks < ksteps; ++ks) {
    const int cur = ks & 1;
    const bool has_next = ks + 1 < ksteps;
    if (has_next) {
      if (ks + 1 < kfull)
        load_slice<FULL, VEC>(f, A, lda, B, ldb, M, N, K, m0, n0, (ks + 1) * BKs, tid);
      else
        load_slice<false, false>(f, A, lda, B, ldb, M, N, K, m0, n0, (ks + 1) * BKs, tid);
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
      store_slice(f, As[cur ^ 1], Bs[cur ^ 1], tid);
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

template <bool VEC>
__global__ void __launch_bounds__(THREADS) simt_gemm_kernel(int64_t M, int64_t N, int64_t K,
                                                            float alpha, const float* A,
                                                            int64_t lda, const float* B,
                                                            int64_t ldb, float beta, float* C,
                                                            int64_t ldc, bool cvec) {
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * BM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;
  if (m0 + BM <= M && n0 + BN <= N)
    gemm_tile<true, VEC>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, m0, n0, cvec);
  else
    gemm_tile<false, VEC>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, m0, n0, cvec);
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
                             int64_t ldc, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>((N + BN - 1) / BN), static_cast<unsigned>((M + BM - 1) / BM));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) &&
                   (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(B) % 16 == 0);
  const bool cvec = (ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
  if (vec)
    simt_gemm_kernel<true><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec);
  else
    simt_gemm_kernel<false><<<grid, THREADS, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cvec);
  return cudaGetLastError();
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
