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
// (all of K).  Most blocks need no scaling (e = 0, see scale.cuh), so packing
// takes ONE pass over the operands: it writes the unscaled split and folds
// max |x| of each block into the block's slot.  A second, cheap pass then
// re-splits, with their exponent, only the blocks whose max lies outside the
// safe range; every other CTA of that pass returns after one load.
//
// Every kernel is a thin wrapper around per-tile device functions; the
// single-problem kernels walk the tiles of A and then of B in one launch, the
// grouped kernels map a flattened item index to (problem, tile) through
// prefix sums, so one launch packs every problem of a grouped gemm.
#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_runtime.h>

#include "internal.h"
#include "scale.cuh"
#include "split_arith.cuh"

namespace gb {

namespace {

enum Pass { kFirst = 0, kRescale = 1 };

// CTA-wide max of m folded into *slot (every thread of the CTA calls this).
// When the block's running max leaves the safe range, *flag is raised so that
// the rescale pass knows it has work (flag may be null: always check).
__device__ __forceinline__ void fold_block_max(unsigned m, unsigned* slot, unsigned* flag) {
  __shared__ unsigned wm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned b = wm[0];
    for (int i = 1; i < static_cast<int>(blockDim.x >> 5); ++i) b = max(b, wm[i]);
    if (b) {
      const unsigned old = atomicMax(slot, b);
      if (flag && block_exponent(max(old, b)) != 0) *flag = 1u;
    }
  }
  __syncthreads();   // wm is reused by the next tile of a looping launch
}

// --------------------------------------------------------- A: row-major split
// One CTA (256 threads, 8 warps) writes a 32-row x 256-column tile of the
// planes (columns of the padded pitch; k in [K, pitch) gets 0).  Thread
// (warp w, lane l) covers rows w, w+8, w+16, w+24 and the quads at columns
// 4l and 4l + 128: its eight loads are issued before any use, so that enough
// bytes are in flight to cover memory latency.  The 32 rows lie in one
// 128-row block.
template <bool TF32, Pass PASS>
__device__ __forceinline__ void split_rows_tile(const float* __restrict__ X, int64_t rows,
                                                int64_t cols, int64_t ld, bool vec,
                                                unsigned* __restrict__ amax, unsigned* flag,
                                                void* __restrict__ planes, int64_t plane,
                                                int64_t pitch, int64_t r0, int64_t k0) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float sc = PASS == kFirst ? 1.0f : pow2f(-block_exponent(amax[r0 / kScaleBlock]));
  float v[4][2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t r = r0 + w + 8 * i;
      const int64_t k = k0 + 128 * c + 4 * lane;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[i][c][j] = 0.0f;
      if (r >= rows || k >= cols) continue;
      const float* p = X + r * ld + k;
      if (vec && k + 3 < cols) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[i][c][0] = q.x, v[i][c][1] = q.y, v[i][c][2] = q.z, v[i][c][3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (k + j < cols) v[i][c][j] = p[j];
      }
    }
  }
  unsigned m = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t r = r0 + w + 8 * i;
      const int64_t k = k0 + 128 * c + 4 * lane;
      if (r >= rows || k >= pitch) continue;
      const float* x = v[i][c];
      if (PASS == kFirst) {
#pragma unroll
        for (int j = 0; j < 4; ++j) m = max(m, abs_bits(x[j]));
      }
      const int64_t o = r * pitch + k;
      if (TF32) {
        float* P = static_cast<float*>(planes);
        float4 h, l;
        split_tf32(x[0] * sc, h.x, l.x);
        split_tf32(x[1] * sc, h.y, l.y);
        split_tf32(x[2] * sc, h.z, l.z);
        split_tf32(x[3] * sc, h.w, l.w);
        *reinterpret_cast<float4*>(P + o) = h;
        *reinterpret_cast<float4*>(P + plane + o) = l;
      } else {
        __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
        __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const HiLoBf16 s = split_bf16(x[j] * sc);
          h[j] = s.hi;
          l[j] = s.lo;
        }
        *reinterpret_cast<uint2*>(P + o) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(P + plane + o) = *reinterpret_cast<const uint2*>(l);
      }
    }
  }
  if (PASS == kFirst) fold_block_max(m, amax + r0 / kScaleBlock, flag);
}

// ---------------------------------------------------- B: transposing split
// One CTA handles a 64 (k) x 128 (n) tile.  Load phase: warp w reads k-rows
// w + 8i (i < 8), each lane a float4 of n (512 contiguous bytes per warp and
// row); all eight loads are issued first, then stored to a shared tile whose
// 132-float pitch keeps both phases free of bank conflicts.  Write phase:
// thread t writes 32 consecutive k of output row n = t % 128 (k half t / 128).
// The 128 columns are one 128-column block.
constexpr int kColTilePitch = 132;

template <bool TF32, Pass PASS>
__device__ __forceinline__ void split_cols_tile(const float* __restrict__ X, int64_t K, int64_t N,
                                                int64_t ld, bool vec, unsigned* __restrict__ amax,
                                                unsigned* flag, void* __restrict__ planes,
                                                int64_t plane, int64_t pitch, int64_t n0, int64_t k0) {
  __shared__ __align__(16) float tile[64 * kColTilePitch];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned m = 0;
  {
    const int64_t n = n0 + 4 * lane;
    float4 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t k = k0 + w + 8 * i;
      v[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (k >= K || n >= N) continue;
      const float* p = X + k * ld + n;
      if (vec && n + 3 < N) {
        v[i] = *reinterpret_cast<const float4*>(p);
      } else {
        v[i].x = p[0];
        if (n + 1 < N) v[i].y = p[1];
        if (n + 2 < N) v[i].z = p[2];
        if (n + 3 < N) v[i].w = p[3];
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      *reinterpret_cast<float4*>(&tile[(w + 8 * i) * kColTilePitch + 4 * lane]) = v[i];
      if (PASS == kFirst) {
        m = max(m, abs_bits(v[i].x));
        m = max(m, abs_bits(v[i].y));
        m = max(m, abs_bits(v[i].z));
        m = max(m, abs_bits(v[i].w));
      }
    }
  }
  __syncthreads();
  const int nl = threadIdx.x & 127;
  const int kl = (threadIdx.x >> 7) * 32;
  const int64_t n = n0 + nl;
  if (n < N && k0 + kl < pitch) {
    const float sc = PASS == kFirst ? 1.0f : pow2f(-block_exponent(amax[n / kScaleBlock]));
    const int64_t obase = n * pitch + k0 + kl;
    const int64_t avail = pitch - (k0 + kl);   // multiple of 8 (bf16) or 4 (tf32)
    if (TF32) {
      float* P = static_cast<float*>(planes);
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        if (4 * g >= avail) break;
        float4 h, l;
        split_tf32(tile[(kl + 4 * g + 0) * kColTilePitch + nl] * sc, h.x, l.x);
        split_tf32(tile[(kl + 4 * g + 1) * kColTilePitch + nl] * sc, h.y, l.y);
        split_tf32(tile[(kl + 4 * g + 2) * kColTilePitch + nl] * sc, h.z, l.z);
        split_tf32(tile[(kl + 4 * g + 3) * kColTilePitch + nl] * sc, h.w, l.w);
        *reinterpret_cast<float4*>(P + obase + 4 * g) = h;
        *reinterpret_cast<float4*>(P + plane + obase + 4 * g) = l;
      }
    } else {
      __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        if (8 * g >= avail) break;
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const HiLoBf16 s = split_bf16(tile[(kl + 8 * g + i) * kColTilePitch + nl] * sc);
          h[i] = s.hi;
          l[i] = s.lo;
        }
        *reinterpret_cast<uint4*>(P + obase + 8 * g) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(P + plane + obase + 8 * g) = *reinterpret_cast<const uint4*>(l);
      }
    }
  }
  if (PASS == kFirst)
    fold_block_max(m, amax + n0 / kScaleBlock, flag);   // its barriers also guard `tile`
  else
    __syncthreads();   // the tile is reused by the next item of a looping launch
}

// ------------------------------------------------ A: block maxima only
// For the fused-split gemm, which splits A itself: one item is a 128-row
// block over a span of 64 loads per row (256 floats with float4 loads);
// thread (x, y) of the 64 x 4 CTA reads load x of rows y, y + 4, ... with
// eight loads in flight, and the CTA folds one max per item.
constexpr int kAmaxLoads = 64;

// Rows stored back to back (lda == K, 16-byte aligned): a block is one
// contiguous run of rows * K floats, streamed as float4 in `parts` pieces.
__global__ void __launch_bounds__(256) amax_flat_kernel(const float* __restrict__ A, int64_t M,
                                                        int64_t K, int parts,
                                                        unsigned* __restrict__ amax, unsigned* flag) {
  const int64_t nblk = (M + 127) / 128;
  for (int64_t item = blockIdx.x; item < nblk * parts; item += gridDim.x) {
    const int64_t b = item / parts;
    const int part = static_cast<int>(item - b * parts);
    const int64_t n4 = min(static_cast<int64_t>(128), M - b * 128) * K / 4;   // K % 4 == 0
    const int64_t per = (n4 + parts - 1) / parts;
    const int64_t lo = part * per, hi = min(n4, lo + per);
    const float4* p = reinterpret_cast<const float4*>(A + b * 128 * K);
    unsigned m = 0;
    for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += 8 * 256) {
      float4 v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int64_t idx = i0 + 256 * i;
        v[i] = idx < hi ? __ldg(p + idx) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
        m = max(m, max(max(abs_bits(v[i].x), abs_bits(v[i].y)), max(abs_bits(v[i].z), abs_bits(v[i].w))));
    }
    fold_block_max(m, amax + b, flag);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256) amax_rows_kernel(const float* __restrict__ A, int64_t M,
                                                        int64_t K, int64_t lda,
                                                        unsigned* __restrict__ amax, unsigned* flag) {
  constexpr int U = VEC ? 4 : 1;   // floats per load
  constexpr int64_t span = kAmaxLoads * U;
  const int64_t nblk = (M + 127) / 128, nspan = (K + span - 1) / span;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  for (int64_t item = blockIdx.x; item < nblk * nspan; item += gridDim.x) {
    const int64_t b = item / nspan;
    const int64_t k = (item - b * nspan) * span + static_cast<int64_t>(tx) * U;
    const int rows = static_cast<int>(min(static_cast<int64_t>(128), M - b * 128));
    const float* base = A + (b * 128) * lda + k;
    unsigned m = 0;
    if (k < K) {
      for (int r0 = ty; r0 < rows; r0 += 32) {
        float v[8][U];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = r0 + 4 * i;
#pragma unroll
          for (int e = 0; e < U; ++e) v[i][e] = 0.0f;
          if (r >= rows) continue;
          const float* p = base + r * lda;
          if (VEC && k + 4 <= K) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p));
            const float t[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < U; ++e) v[i][e] = t[e];
          } else {
#pragma unroll
            for (int e = 0; e < U; ++e)
              if (k + e < K) v[i][e] = __ldg(p + e);
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int e = 0; e < U; ++e) m = max(m, abs_bits(v[i][e]));
      }
    }
    fold_block_max(m, amax + b, flag);
  }
}

// --------------------------------------------------- tile decomposition
// First pass: A in 32-row x 256-column tiles, B in 64-k x 128-column tiles.
// Rescale pass: one item per scale block (128 rows of A or 128 columns of B,
// all of K); a block that needs no scaling costs one load, one that does is
// re-split tile by tile.
struct PackShape {
  const float* A;
  const float* B;
  int64_t M, N, K, lda, ldb, pitch;
  int64_t planeA, planeB;   // elements from the hi plane to the lo plane
  unsigned* flag;           // raised when some block needs a rescale (null: always check)
  bool vecA, vecB;
  unsigned* amaxA;
  unsigned* amaxB;
  void* planesA;
  void* planesB;

  __device__ int first_items_a() const { return (int)(((M + 31) / 32) * ((pitch + 255) / 256)); }
  __device__ int first_items_b() const { return (int)(((N + 127) / 128) * ((pitch + 63) / 64)); }
  __device__ int rescale_items_a() const { return (int)((M + 127) / 128); }
  __device__ int rescale_items_b() const { return (int)((N + 127) / 128); }
};

template <bool TF32>
__device__ __forceinline__ void first_item(const PackShape& p, int i) {
  const int na = p.first_items_a();
  if (i < na) {
    const int cols = (int)((p.pitch + 255) / 256);
    split_rows_tile<TF32, kFirst>(p.A, p.M, p.K, p.lda, p.vecA, p.amaxA, p.flag, p.planesA, p.planeA,
                                  p.pitch, (int64_t)(i / cols) * 32, (int64_t)(i % cols) * 256);
  } else {
    const int l = i - na;
    const int ncols = (int)((p.N + 127) / 128);
    split_cols_tile<TF32, kFirst>(p.B, p.K, p.N, p.ldb, p.vecB, p.amaxB, p.flag, p.planesB, p.planeB, p.pitch,
                                  (int64_t)(l % ncols) * 128, (int64_t)(l / ncols) * 64);
  }
}

template <bool TF32>
__device__ __forceinline__ void rescale_item(const PackShape& p, int i) {
  const int na = p.rescale_items_a();
  if (i < na) {
    const int64_t r0 = (int64_t)i * 128;
    if (block_exponent(p.amaxA[i]) == 0) return;   // uniform per CTA
    for (int64_t k0 = 0; k0 < p.pitch; k0 += 256)
      for (int q = 0; q < 4 && r0 + 32 * q < p.M; ++q)
        split_rows_tile<TF32, kRescale>(p.A, p.M, p.K, p.lda, p.vecA, p.amaxA, p.flag, p.planesA, p.planeA, p.pitch,
                                        r0 + 32 * q, k0);
  } else {
    const int l = i - na;
    const int64_t n0 = (int64_t)l * 128;
    if (block_exponent(p.amaxB[l]) == 0) return;
    for (int64_t k0 = 0; k0 < p.pitch; k0 += 64)
      split_cols_tile<TF32, kRescale>(p.B, p.K, p.N, p.ldb, p.vecB, p.amaxB, p.flag, p.planesB, p.planeB, p.pitch,
                                      n0, k0);
  }
}

// ------------------------------------------------ single-problem kernels
template <bool TF32>
__global__ void pack_first_kernel(const PackShape p) {
  const int total = p.first_items_a() + p.first_items_b();
  for (int i = blockIdx.x; i < total; i += gridDim.x) first_item<TF32>(p, i);
}

template <bool TF32>
__global__ void pack_rescale_kernel(const PackShape p) {
  if (p.flag && *p.flag == 0u) return;   // no block out of range
  const int total = p.rescale_items_a() + p.rescale_items_b();
  for (int i = blockIdx.x; i < total; i += gridDim.x) rescale_item<TF32>(p, i);
}

// ------------------------------------------------------ grouped kernels
// Item i of a grouped pack launch: problem g with prefix[g] <= i < prefix[g+1].
__device__ __forceinline__ int find_problem(const int* __restrict__ prefix, int G, int i) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
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

__device__ __forceinline__ PackShape problem_shape(const GroupedProblem& g, const GroupedPtrs& q) {
  PackShape p;
  p.A = q.A, p.B = q.B;
  p.M = g.M, p.N = g.N, p.K = g.K, p.lda = g.lda, p.ldb = g.ldb, p.pitch = g.pitch;
  p.planeA = static_cast<int64_t>(g.M) * g.pitch;
  p.planeB = static_cast<int64_t>(g.N) * g.pitch;
  p.vecA = (reinterpret_cast<uintptr_t>(q.A) % 16 == 0) && (g.lda % 4 == 0);
  p.vecB = (reinterpret_cast<uintptr_t>(q.B) % 16 == 0) && (g.ldb % 4 == 0);
  p.amaxA = g.amaxA, p.amaxB = g.amaxB;
  p.planesA = g.planesA, p.planesB = g.planesB;
  return p;
}

template <bool TF32, Pass PASS>
__global__ void grouped_pack_kernel(const GroupedProblem* __restrict__ probs,
                                    const GroupedPtrs* __restrict__ ptrs,
                                    const int* __restrict__ prefix_g, int G, unsigned* flag) {
  if (PASS == kRescale && *flag == 0u) return;   // no block of any problem out of range
  const int* prefix = stage_prefix(prefix_g, G);
  const int total = prefix[G];
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const int g = find_problem(prefix, G, i);
    const GroupedPtrs& q = ptrs[g];
    if (q.alpha == 0.0f) continue;   // A and B are not read when alpha == 0
    PackShape p = problem_shape(probs[g], q);
    p.flag = flag;
    if (PASS == kFirst)
      first_item<TF32>(p, i - prefix[g]);
    else
      rescale_item<TF32>(p, i - prefix[g]);
  }
}

int grid_for(int64_t items, int sms) {
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  return static_cast<int>(items < cap ? (items > 0 ? items : 1) : cap);
}

}  // namespace

// Items per problem of the two pack passes (host side, same tiling as above).
int pack_first_items(int64_t M, int64_t N, int64_t pitch) {
  return static_cast<int>(((M + 31) / 32) * ((pitch + 255) / 256) + ((N + 127) / 128) * ((pitch + 63) / 64));
}
int pack_rescale_items(int64_t M, int64_t N, int64_t pitch) {
  (void)pitch;
  return static_cast<int>((M + 127) / 128 + (N + 127) / 128);
}

cudaError_t pack_launch(Prec prec, const float* A, int64_t M, int64_t K, int64_t lda, const float* B,
                        int64_t N, int64_t ldb, unsigned* amaxA, unsigned* amaxB, unsigned* flag,
                        void* planesA, void* planesB, int64_t pitch, int sms, cudaStream_t s) {
  PackShape p;
  p.flag = flag;
  p.A = A, p.B = B, p.M = A ? M : 0, p.N = B ? N : 0, p.K = K, p.lda = lda, p.ldb = ldb;
  p.pitch = pitch;
  p.planeA = p.M * pitch;
  p.planeB = p.N * pitch;
  p.vecA = A && lda % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
  p.vecB = B && ldb % 4 == 0 && reinterpret_cast<uintptr_t>(B) % 16 == 0;
  p.amaxA = amaxA, p.amaxB = amaxB, p.planesA = planesA, p.planesB = planesB;
  const int64_t first = pack_first_items(p.M, p.N, pitch);
  const int64_t rescale = pack_rescale_items(p.M, p.N, pitch);
  if (first == 0) return cudaSuccess;
  if (prec == Prec::TF32) {
    pack_first_kernel<true><<<grid_for(first, sms), 256, 0, s>>>(p);
    pack_rescale_kernel<true><<<grid_for(rescale, sms), 256, 0, s>>>(p);
  } else {
    pack_first_kernel<false><<<grid_for(first, sms), 256, 0, s>>>(p);
    pack_rescale_kernel<false><<<grid_for(rescale, sms), 256, 0, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t pack_fused_launch(Prec prec, const float* A, int64_t M, int64_t K, int64_t lda,
                              const float* B, int64_t N, int64_t ldb, unsigned* amaxA,
                              unsigned* amaxB, unsigned* flag, void* planesB, int64_t pitch, int sms,
                              cudaStream_t s) {
  if (M > 0 && K > 0) {
    const bool vec = lda % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
    if (vec && lda == K) {
      const int64_t nblk = (M + 127) / 128;
      const int parts = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(
          (4 * static_cast<int64_t>(sms) + nblk - 1) / nblk, (128 * K / 4 + 2047) / 2048)));
      const int grid = static_cast<int>(std::min<int64_t>(nblk * parts, 8 * static_cast<int64_t>(sms)));
      amax_flat_kernel<<<grid, 256, 0, s>>>(A, M, K, parts, amaxA, flag);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      return pack_launch(prec, nullptr, 0, K, 1, B, N, ldb, nullptr, amaxB, flag, nullptr, planesB,
                         pitch, sms, s);
    }
    const int64_t span = kAmaxLoads * (vec ? 4 : 1);
    const int64_t items = ((M + 127) / 128) * ((K + span - 1) / span);
    const int grid = static_cast<int>(std::min<int64_t>(items, 8 * static_cast<int64_t>(sms)));
    if (vec)
      amax_rows_kernel<true><<<grid, 256, 0, s>>>(A, M, K, lda, amaxA, flag);
    else
      amax_rows_kernel<false><<<grid, 256, 0, s>>>(A, M, K, lda, amaxA, flag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // B as in the packed variant
  return pack_launch(prec, nullptr, 0, K, 1, B, N, ldb, nullptr, amaxB, flag, nullptr, planesB, pitch,
                     sms, s);
}

cudaError_t pack_rows_panel_launch(Prec prec, const float* A, int64_t rows, int64_t K, int64_t lda,
                                   unsigned* amaxA, unsigned* flag, void* planesA,
                                   int64_t plane_stride, int64_t pitch, int sms, cudaStream_t s) {
  PackShape p;
  p.flag = flag;
  p.A = A, p.B = nullptr, p.M = rows, p.N = 0, p.K = K, p.lda = lda, p.ldb = 1;
  p.pitch = pitch;
  p.planeA = plane_stride;
  p.planeB = 0;
  p.vecA = lda % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
  p.vecB = false;
  p.amaxA = amaxA, p.amaxB = nullptr, p.planesA = planesA, p.planesB = nullptr;
  const int64_t first = pack_first_items(rows, 0, pitch);
  const int64_t rescale = pack_rescale_items(rows, 0, pitch);
  if (first == 0) return cudaSuccess;
  if (prec == Prec::TF32) {
    pack_first_kernel<true><<<grid_for(first, sms), 256, 0, s>>>(p);
    pack_rescale_kernel<true><<<grid_for(rescale, sms), 256, 0, s>>>(p);
  } else {
    pack_first_kernel<false><<<grid_for(first, sms), 256, 0, s>>>(p);
    pack_rescale_kernel<false><<<grid_for(rescale, sms), 256, 0, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t grouped_pack_launch(Prec prec, const GroupedProblem* probs, const GroupedPtrs* ptrs,
                                const int* first_prefix, int first_total, const int* rescale_prefix,
                                int rescale_total, int G, unsigned* flag, int sms, cudaStream_t s) {
  const size_t dyn = (G + 1) <= 4096 ? static_cast<size_t>(G + 1) * sizeof(int) : 0;
  if (first_total == 0) return cudaSuccess;
  const int gf = grid_for(first_total, sms), gr = grid_for(rescale_total, sms);
  if (prec == Prec::TF32) {
    grouped_pack_kernel<true, kFirst><<<gf, 256, dyn, s>>>(probs, ptrs, first_prefix, G, flag);
    grouped_pack_kernel<true, kRescale><<<gr, 256, dyn, s>>>(probs, ptrs, rescale_prefix, G, flag);
  } else {
    grouped_pack_kernel<false, kFirst><<<gf, 256, dyn, s>>>(probs, ptrs, first_prefix, G, flag);
    grouped_pack_kernel<false, kRescale><<<gr, 256, dyn, s>>>(probs, ptrs, rescale_prefix, G, flag);
  }
  return cudaGetLastError();
}

}  // namespace gb
