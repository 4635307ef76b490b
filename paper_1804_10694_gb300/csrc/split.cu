// Operand packing for the split-precision gemm ("array packing" in the
// paper's gemm recipe, Section I and Section VI-A).  Each FP32 operand is
// rewritten once, before the main loop, as two planes of lower precision:
//     x' = x * 2^-e            (e = block exponent, exponent-field arithmetic)
//     hi = RN(x'),  lo = RN(x' - hi)
// with RN round-to-nearest-even to bf16 (hardware conversion) or to tf32
// (bit arithmetic below; the planes keep tf32 values in 32-bit containers).
// A is kept row-major (K contiguous); B is transposed so that both operands
// are K-major for the tensor-core kernel.  Rows of the planes are padded to
// a 16-byte pitch with zeros.
//
// Blocks: A uses one exponent per 128 rows (all of K), B one per 128 columns
// (all of K), from a first pass that takes max |x| per block.
//
// Every kernel is a thin wrapper around a per-tile device function; the
// single-problem kernels map blockIdx to a tile, the grouped kernels map a
// flattened item index to (problem, tile) through prefix sums, so one launch
// packs every problem of a grouped gemm.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "scale.cuh"

namespace gb {

namespace {

// ------------------------------------------------------------------ max |x|
// One CTA (256 threads) reduces a 32-row x 128-column tile, which lies inside
// one block of either kind, and folds it into the block's slot with an
// unsigned atomicMax on the bit pattern of |x| (non-negative floats order like
// their bits; NaN patterns sort above Inf, so a NaN marks the block as
// non-finite).
__device__ __forceinline__ void absmax_tile(const float* __restrict__ X, int64_t rows, int64_t cols,
                                            int64_t ld, int64_t r0, int64_t c0, bool vec,
                                            bool blocks_along_rows, unsigned* __restrict__ amax) {
  __shared__ unsigned wm[8];
  const int t = threadIdx.x;
  const int cq = (t & 31) * 4;
  unsigned m = 0;
  for (int rr = t >> 5; rr < 32; rr += 8) {
    const int64_t r = r0 + rr;
    if (r >= rows) break;
    const float* p = X + r * ld + c0 + cq;
    if (vec && c0 + cq + 3 < cols) {
      const float4 v = *reinterpret_cast<const float4*>(p);
      m = max(m, __float_as_uint(v.x) & 0x7FFFFFFFu);
      m = max(m, __float_as_uint(v.y) & 0x7FFFFFFFu);
      m = max(m, __float_as_uint(v.z) & 0x7FFFFFFFu);
      m = max(m, __float_as_uint(v.w) & 0x7FFFFFFFu);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (c0 + cq + i < cols) m = max(m, __float_as_uint(p[i]) & 0x7FFFFFFFu);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((t & 31) == 0) wm[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    unsigned b = wm[0];
    for (int i = 1; i < 8; ++i) b = max(b, wm[i]);
    const int64_t slot = blocks_along_rows ? r0 / kScaleBlock : c0 / kScaleBlock;
    atomicMax(amax + slot, b);
  }
  __syncthreads();   // wm is reused by the next tile of a grouped launch
}

// ---------------------------------------------------------------- rounding
__device__ __forceinline__ float round_tf32_rne(float x) {
  const unsigned u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;   // Inf / NaN unchanged
  const unsigned r = (u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
  return __uint_as_float(r);
}

struct HiLoBf16 {
  __nv_bfloat16 hi, lo;
};

__device__ __forceinline__ HiLoBf16 split_bf16(float xs) {
  HiLoBf16 o;
  o.hi = __float2bfloat16_rn(xs);
  o.lo = isfinite(xs) ? __float2bfloat16_rn(xs - __bfloat162float(o.hi)) : __float2bfloat16_rn(0.0f);
  return o;
}

__device__ __forceinline__ void split_tf32(float xs, float& hi, float& lo) {
  hi = round_tf32_rne(xs);
  lo = isfinite(xs) ? round_tf32_rne(xs - hi) : 0.0f;
}

// --------------------------------------------------------- A: row-major split
// One CTA writes a 32-row x 128-column tile of the planes (columns of the
// padded pitch); each thread handles 4 quads of 4 consecutive k.  Padding
// k in [K, pitch) gets 0.
template <bool TF32>
__device__ __forceinline__ void split_rows_tile(const float* __restrict__ X, int64_t rows,
                                                int64_t cols, int64_t ld, bool vec,
                                                const unsigned* __restrict__ amax,
                                                void* __restrict__ planes, int64_t pitch,
                                                int64_t r0, int64_t k0) {
  const int64_t plane = rows * pitch;
  const int t = threadIdx.x;
  const int kq = (t & 31) * 4;
  for (int rr = t >> 5; rr < 32; rr += 8) {
    const int64_t r = r0 + rr;
    const int64_t k = k0 + kq;
    if (r >= rows || k >= pitch) continue;
    const float sc = pow2f(-block_exponent(amax[r / kScaleBlock]));
    float v[4];
    const float* p = X + r * ld + k;
    if (vec && k + 3 < cols) {
      const float4 q = *reinterpret_cast<const float4*>(p);
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = (k + i < cols) ? p[i] : 0.0f;
    }
    const int64_t o = r * pitch + k;
    if (TF32) {
      float* P = static_cast<float*>(planes);
      float4 h, l;
      split_tf32(v[0] * sc, h.x, l.x);
      split_tf32(v[1] * sc, h.y, l.y);
      split_tf32(v[2] * sc, h.z, l.z);
      split_tf32(v[3] * sc, h.w, l.w);
      *reinterpret_cast<float4*>(P + o) = h;
      *reinterpret_cast<float4*>(P + plane + o) = l;
    } else {
      __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
      __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const HiLoBf16 s = split_bf16(v[i] * sc);
        h[i] = s.hi;
        l[i] = s.lo;
      }
      *reinterpret_cast<uint2*>(P + o) = *reinterpret_cast<const uint2*>(h);
      *reinterpret_cast<uint2*>(P + plane + o) = *reinterpret_cast<const uint2*>(l);
    }
  }
}

// ---------------------------------------------------- B: transposing split
// One CTA handles a 64 (k) x 64 (n) tile: coalesced loads along n into shared
// memory, then each thread writes 16 consecutive k of one output row n.
template <bool TF32>
__device__ __forceinline__ void split_cols_tile(const float* __restrict__ X, int64_t K, int64_t N,
                                                int64_t ld, bool vec,
                                                const unsigned* __restrict__ amax,
                                                void* __restrict__ planes, int64_t pitch,
                                                int64_t n0, int64_t k0) {
  __shared__ float tile[64][65];
  const int t = threadIdx.x;
  {
    const int cn = (t & 15) * 4;
    for (int kr = t >> 4; kr < 64; kr += 16) {
      const int64_t k = k0 + kr;
      float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (k < K) {
        const float* p = X + k * ld + n0 + cn;
        if (vec && n0 + cn + 3 < N) {
          const float4 q = *reinterpret_cast<const float4*>(p);
          v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (n0 + cn + i < N) v[i] = p[i];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) tile[kr][cn + i] = v[i];
    }
  }
  __syncthreads();
  const int nl = t >> 2;              // 0..63
  const int kl = (t & 3) * 16;        // 0, 16, 32, 48
  const int64_t n = n0 + nl;
  if (n < N && k0 + kl < pitch) {
    const float sc = pow2f(-block_exponent(amax[n / kScaleBlock]));
    const int64_t plane = N * pitch;
    const int64_t obase = n * pitch + k0 + kl;
    const bool whole = k0 + kl + 16 <= pitch;
    if (TF32) {
      float* P = static_cast<float*>(planes);
      float h[16], l[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) split_tf32(tile[kl + i][nl] * sc, h[i], l[i]);
      if (whole) {
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
          *reinterpret_cast<float4*>(P + obase + i) = make_float4(h[i], h[i + 1], h[i + 2], h[i + 3]);
          *reinterpret_cast<float4*>(P + plane + obase + i) =
              make_float4(l[i], l[i + 1], l[i + 2], l[i + 3]);
        }
      } else {
        for (int i = 0; i < 16 && k0 + kl + i < pitch; ++i) {
          P[obase + i] = h[i];
          P[plane + obase + i] = l[i];
        }
      }
    } else {
      __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
      __align__(16) __nv_bfloat16 h[16], l[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const HiLoBf16 s = split_bf16(tile[kl + i][nl] * sc);
        h[i] = s.hi;
        l[i] = s.lo;
      }
      if (whole) {
        *reinterpret_cast<uint4*>(P + obase) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(P + obase + 8) = *reinterpret_cast<const uint4*>(h + 8);
        *reinterpret_cast<uint4*>(P + plane + obase) = *reinterpret_cast<const uint4*>(l);
        *reinterpret_cast<uint4*>(P + plane + obase + 8) = *reinterpret_cast<const uint4*>(l + 8);
      } else {
        // pitch is a multiple of 8 elements: write whole 8-element groups
        for (int i = 0; i < 16 && k0 + kl + i < pitch; i += 8) {
          *reinterpret_cast<uint4*>(P + obase + i) = *reinterpret_cast<const uint4*>(h + i);
          *reinterpret_cast<uint4*>(P + plane + obase + i) = *reinterpret_cast<const uint4*>(l + i);
        }
      }
    }
  }
  __syncthreads();   // the tile is reused by the next item of a grouped launch
}

// ------------------------------------------------ single-problem kernels
__global__ void absmax_kernel(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                              bool vec, bool blocks_along_rows, unsigned* __restrict__ amax) {
  absmax_tile(X, rows, cols, ld, static_cast<int64_t>(blockIdx.y) * 32,
              static_cast<int64_t>(blockIdx.x) * 128, vec, blocks_along_rows, amax);
}

template <bool TF32>
__global__ void split_rows_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                  int64_t ld, bool vec, const unsigned* __restrict__ amax,
                                  void* __restrict__ planes, int64_t pitch) {
  split_rows_tile<TF32>(X, rows, cols, ld, vec, amax, planes, pitch,
                        static_cast<int64_t>(blockIdx.y) * 32, static_cast<int64_t>(blockIdx.x) * 128);
}

template <bool TF32>
__global__ void split_cols_kernel(const float* __restrict__ X, int64_t K, int64_t N, int64_t ld,
                                  bool vec, const unsigned* __restrict__ amax,
                                  void* __restrict__ planes, int64_t pitch) {
  split_cols_tile<TF32>(X, K, N, ld, vec, amax, planes, pitch, static_cast<int64_t>(blockIdx.x) * 64,
                        static_cast<int64_t>(blockIdx.y) * 64);
}

// ------------------------------------------------------ grouped kernels
// Item i of a grouped pack launch: problem g with prefix[g] <= i < prefix[g+1];
// the problem's first items belong to A, the rest to B.
__device__ __forceinline__ int find_problem(const int* __restrict__ prefix, int G, int i) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool aligned16(const void* p, int64_t ld) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && (ld % 4 == 0);
}

// The problem prefix sums are staged in shared memory when they fit (the
// launch passes their size as dynamic shared memory, 0 otherwise).
__device__ __forceinline__ const int* stage_prefix(const int* __restrict__ prefix, int G) {
  extern __shared__ int s_prefix[];
  unsigned dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  if (dyn < (G + 1) * sizeof(int)) return prefix;
  for (int i = threadIdx.x; i <= G; i += blockDim.x) s_prefix[i] = prefix[i];
  __syncthreads();
  return s_prefix;
}

__global__ void grouped_absmax_kernel(const GroupedProblem* __restrict__ probs,
                                      const GroupedPtrs* __restrict__ ptrs,
                                      const int* __restrict__ prefix_g, int G) {
  const int* prefix = stage_prefix(prefix_g, G);
  const int total = prefix[G];
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const int g = find_problem(prefix, G, i);
    const GroupedProblem& p = probs[g];
    const GroupedPtrs& q = ptrs[g];
    if (q.alpha == 0.0f) continue;   // A and B are not read when alpha == 0
    const int local = i - prefix[g];
    const int a_cols = (p.K + 127) / 128;
    const int a_items = ((p.M + 31) / 32) * a_cols;
    if (local < a_items) {
      absmax_tile(q.A, p.M, p.K, p.lda, static_cast<int64_t>(local / a_cols) * 32,
                  static_cast<int64_t>(local % a_cols) * 128, aligned16(q.A, p.lda), true, p.amaxA);
    } else {
      const int l = local - a_items;
      const int b_cols = (p.N + 127) / 128;
      absmax_tile(q.B, p.K, p.N, p.ldb, static_cast<int64_t>(l / b_cols) * 32,
                  static_cast<int64_t>(l % b_cols) * 128, aligned16(q.B, p.ldb), false, p.amaxB);
    }
  }
}

template <bool TF32>
__global__ void grouped_split_kernel(const GroupedProblem* __restrict__ probs,
                                     const GroupedPtrs* __restrict__ ptrs,
                                     const int* __restrict__ prefix_g, int G) {
  const int* prefix = stage_prefix(prefix_g, G);
  const int total = prefix[G];
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const int g = find_problem(prefix, G, i);
    const GroupedProblem& p = probs[g];
    const GroupedPtrs& q = ptrs[g];
    if (q.alpha == 0.0f) continue;   // A and B are not read when alpha == 0
    const int local = i - prefix[g];
    const int a_cols = static_cast<int>((p.pitch + 127) / 128);
    const int a_items = ((p.M + 31) / 32) * a_cols;
    if (local < a_items) {
      split_rows_tile<TF32>(q.A, p.M, p.K, p.lda, aligned16(q.A, p.lda), p.amaxA, p.planesA, p.pitch,
                            static_cast<int64_t>(local / a_cols) * 32,
                            static_cast<int64_t>(local % a_cols) * 128);
    } else {
      const int l = local - a_items;
      const int b_ncols = (p.N + 63) / 64;
      split_cols_tile<TF32>(q.B, p.K, p.N, p.ldb, aligned16(q.B, p.ldb), p.amaxB, p.planesB, p.pitch,
                            static_cast<int64_t>(l % b_ncols) * 64,
                            static_cast<int64_t>(l / b_ncols) * 64);
    }
  }
}

bool vec_ok(const float* X, int64_t ld) {
  return ld % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
}

}  // namespace

// Items per problem of the grouped pack launches (host side, same tiling as
// the kernels above).
int grouped_absmax_items(int64_t M, int64_t N, int64_t K) {
  return static_cast<int>(((M + 31) / 32) * ((K + 127) / 128) + ((K + 31) / 32) * ((N + 127) / 128));
}
int grouped_split_items(int64_t M, int64_t N, int64_t pitch) {
  return static_cast<int>(((M + 31) / 32) * ((pitch + 127) / 128) + ((N + 63) / 64) * ((pitch + 63) / 64));
}

cudaError_t absmax_launch(const float* X, int64_t rows, int64_t cols, int64_t ld,
                          bool blocks_along_rows, unsigned* amax, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>((cols + 127) / 128), static_cast<unsigned>((rows + 31) / 32));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  absmax_kernel<<<grid, 256, 0, s>>>(X, rows, cols, ld, vec_ok(X, ld), blocks_along_rows, amax);
  return cudaGetLastError();
}

cudaError_t split_rows_launch(Prec p, const float* X, int64_t rows, int64_t cols, int64_t ld,
                              const unsigned* amax, void* planes, int64_t pitch, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>((pitch + 127) / 128), static_cast<unsigned>((rows + 31) / 32));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  const bool vec = vec_ok(X, ld);
  if (p == Prec::TF32)
    split_rows_kernel<true><<<grid, 256, 0, s>>>(X, rows, cols, ld, vec, amax, planes, pitch);
  else
    split_rows_kernel<false><<<grid, 256, 0, s>>>(X, rows, cols, ld, vec, amax, planes, pitch);
  return cudaGetLastError();
}

cudaError_t split_cols_launch(Prec p, const float* X, int64_t K, int64_t N, int64_t ld,
                              const unsigned* amax, void* planes, int64_t pitch, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>((N + 63) / 64), static_cast<unsigned>((pitch + 63) / 64));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  const bool vec = vec_ok(X, ld);
  if (p == Prec::TF32)
    split_cols_kernel<true><<<grid, 256, 0, s>>>(X, K, N, ld, vec, amax, planes, pitch);
  else
    split_cols_kernel<false><<<grid, 256, 0, s>>>(X, K, N, ld, vec, amax, planes, pitch);
  return cudaGetLastError();
}

cudaError_t grouped_pack_launch(Prec p, const GroupedProblem* probs, const GroupedPtrs* ptrs,
                                const int* absmax_prefix, int absmax_total, const int* split_prefix,
                                int split_total, int G, int sms, cudaStream_t s) {
  const int ga = absmax_total < sms * 8 ? absmax_total : sms * 8;
  const int gs = split_total < sms * 8 ? split_total : sms * 8;
  const size_t dyn = (G + 1) <= 4096 ? (size_t)(G + 1) * sizeof(int) : 0;
  if (ga > 0) grouped_absmax_kernel<<<ga, 256, dyn, s>>>(probs, ptrs, absmax_prefix, G);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (gs > 0) {
    if (p == Prec::TF32)
      grouped_split_kernel<true><<<gs, 256, dyn, s>>>(probs, ptrs, split_prefix, G);
    else
      grouped_split_kernel<false><<<gs, 256, dyn, s>>>(probs, ptrs, split_prefix, G);
  }
  return cudaGetLastError();
}

}  // namespace gb
