// Operand packing for the split-precision gemm ("array packing" in the
// paper's gemm recipe, Section I and Section VI-A).  Each FP32 operand is
// rewritten once, before the main loop, as two planes of lower precision:
//     x' = x * 2^-e            (e = block exponent, exponent-field arithmetic)
//     hi = RN(x'),  lo = RN(x' - hi)
// with RN round-to-nearest-even to bf16 (hardware conversion) or to tf32
// (bit arithmetic; the planes keep tf32 values in 32-bit containers); the
// six-product bf16 mode writes three planes, hi, mid and lo.
// A is kept row-major (K contiguous); B is transposed so that both operands
// are K-major for the tensor-core kernel.  Rows of the planes are padded to
// a 16-byte pitch with zeros.
//
// Blocks: A uses one exponent per 128 rows (all of K), B one per 128 columns
// (all of K).  Most blocks need no scaling (e = 0, see scale.cuh), so packing
// is ONE launch: each item (tile) writes the unscaled split, folds max |x|
// into its block's slot and counts itself done on the block's counter; the
// CTA that completes a block thus sees the block's final max and, only if
// the block lies outside the safe range, re-splits it with its exponent.  No
// CTA ever waits for another.
//
// Every kernel is a thin wrapper around per-tile device functions; the
// single-problem kernel walks the tiles of A and then of B, the grouped
// kernel maps a flattened item index to (problem, tile) through prefix
// sums, so one launch packs every problem of a grouped gemm.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "internal.h"
#include "ptx.cuh"
#include "scale.cuh"
#include "split_arith.cuh"

namespace gb {

namespace {

enum Pass { kFirst = 0, kRescale = 1 };

// End of a run of items of one block processed by this CTA (every thread
// of the CTA calls this with its max |x| over the run): folds the CTA's max
// into the block's slot and counts the run's items on the block's counter.
// Returns, uniformly over the CTA, the block's final max bits when this run
// completed the block, else 0xFFFFFFFF.  The CTA barrier orders every
// thread's plane writes before thread 0's count, an acquire-release atomic
// at GPU scope, whose release is cumulative: they and the atomicMax are
// visible before the completing CTA, whose acquire observes the count, reads
// the max or re-splits the block (the pattern of a split-K semaphore).  No
// CTA waits for another.
__device__ __forceinline__ unsigned finish_run(unsigned m, unsigned* slot, unsigned* cnt,
                                               unsigned run, unsigned items) {
  __shared__ unsigned wm[32];
  __shared__ unsigned s_done;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned b = wm[0];
    for (int i = 1; i < static_cast<int>(blockDim.x >> 5); ++i) b = max(b, wm[i]);
    if (b) atomicMax(slot, b);
    const unsigned done = atom_add_acq_rel_gpu(cnt, run) + run;
    unsigned v = 0xFFFFFFFFu;
    if (done == items) v = *reinterpret_cast<const volatile unsigned*>(slot);
    s_done = v;
  }
  __syncthreads();
  const unsigned v = s_done;
  __syncthreads();   // wm and s_done are reused by the next run
  return v;
}

// CTA-wide max of m folded into *slot (the max-only pass; no counting).
__device__ __forceinline__ void fold_block_max(unsigned m, unsigned* slot) {
  __shared__ unsigned wm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned b = wm[0];
    for (int i = 1; i < static_cast<int>(blockDim.x >> 5); ++i) b = max(b, wm[i]);
    if (b) atomicMax(slot, b);
  }
  __syncthreads();   // wm is reused by the next item
}

// --------------------------------------------------------- A: row-major split
// One CTA (256 threads, 8 warps) writes a 32-row x 256-column tile of the
// planes (columns of the padded pitch; k in [K, pitch) gets 0).  Thread
// (warp w, lane l) covers rows w, w+8, w+16, w+24 and the quads at columns
// 4l and 4l + 128: its eight loads are issued before any use, so that enough
// bytes are in flight to cover memory latency.  The 32 rows lie in one
// 128-row block.
template <Prec PR, Pass PASS>
__device__ __forceinline__ unsigned split_rows_tile(const float* __restrict__ X, int64_t rows,
                                                int64_t cols, int64_t ld, bool vec,
                                                unsigned* __restrict__ amax,
                                                void* __restrict__ planes, int64_t plane,
                                                int64_t pitch, int64_t r0, int64_t k0) {
  constexpr bool TF32 = PR == Prec::TF32;
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
      } else if (PR == Prec::BF16X6) {
        __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
        __align__(8) __nv_bfloat16 h[4], mi[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const Split3Bf16 s = split3_bf16(x[j] * sc);
          h[j] = s.hi;
          mi[j] = s.mid;
          l[j] = s.lo;
        }
        *reinterpret_cast<uint2*>(P + o) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(P + plane + o) = *reinterpret_cast<const uint2*>(mi);
        *reinterpret_cast<uint2*>(P + 2 * plane + o) = *reinterpret_cast<const uint2*>(l);
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
  return m;   // this thread's max |x| (kFirst; 0 for kRescale)
}

// ---------------------------------------------------- B: transposing split
// One CTA handles a 64 (k) x 128 (n) tile through the shared `tile`
// (64 x 128 floats, declared once by the kernel).  Element (k, n) sits at
// tile[k * 128 + (n ^ col_swizzle(k))]: the XOR moves whole 4-float groups,
// so that both phases are free of bank conflicts (bf16; 2-way for tf32).
// Load phase: warp w reads k-rows w + 8i (i < 8), each lane a float4 of n
// (512 contiguous bytes per warp and row); all eight loads are issued first,
// then stored to the tile as float4.  Write phase: output row n's 64-k
// segment of a plane is 128 bytes (bf16) or 256 (tf32); UPR = 8 or 16
// threads write it as whole 16-byte units, so that a warp stores complete
// rows (4 or 2 per instruction) instead of one 16-byte piece of 32 rows.
// The 128 columns are one 128-column block.
constexpr int kColTileFloats = 64 * 128;

__device__ __forceinline__ int col_swizzle(int k) { return ((k >> 3) & 7) << 2; }

template <Prec PR, Pass PASS>
__device__ __forceinline__ unsigned split_cols_tile(const float* __restrict__ X, int64_t K, int64_t N,
                                                int64_t ld, bool vec, unsigned* __restrict__ amax,
                                                void* __restrict__ planes, int64_t plane,
                                                int64_t pitch, int64_t n0, int64_t k0,
                                                float* __restrict__ tile) {
  constexpr bool TF32 = PR == Prec::TF32;
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
      const int kr = w + 8 * i;
      *reinterpret_cast<float4*>(&tile[kr * 128 + ((4 * lane) ^ col_swizzle(kr))]) = v[i];
      if (PASS == kFirst) {
        m = max(m, abs_bits(v[i].x));
        m = max(m, abs_bits(v[i].y));
        m = max(m, abs_bits(v[i].z));
        m = max(m, abs_bits(v[i].w));
      }
    }
  }
  __syncthreads();
  constexpr int VPU = TF32 ? 4 : 8;          // values per 16-byte output unit
  constexpr int UPR = 64 / VPU;              // threads per output row segment
  constexpr int RPP = 256 / UPR;             // output rows per pass
  const int kl = (threadIdx.x % UPR) * VPU;  // first k of this thread's unit (tile row)
  const int rloc = threadIdx.x / UPR;
  const bool kin = k0 + kl < pitch;          // pitch is a multiple of VPU: units are whole
#pragma unroll 1
  for (int nl = rloc; nl < 128; nl += RPP) {
    const int64_t n = n0 + nl;
    if (n >= N || !kin) continue;
    const float sc = PASS == kFirst ? 1.0f : pow2f(-block_exponent(amax[n / kScaleBlock]));
    float x[VPU];
#pragma unroll
    for (int i = 0; i < VPU; ++i) x[i] = tile[(kl + i) * 128 + (nl ^ col_swizzle(kl + i))] * sc;
    const int64_t o = n * pitch + k0 + kl;
    if (TF32) {
      float* P = static_cast<float*>(planes);
      float4 h, l;
      split_tf32(x[0], h.x, l.x);
      split_tf32(x[1], h.y, l.y);
      split_tf32(x[2], h.z, l.z);
      split_tf32(x[3], h.w, l.w);
      *reinterpret_cast<float4*>(P + o) = h;
      *reinterpret_cast<float4*>(P + plane + o) = l;
    } else if (PR == Prec::BF16X6) {
      __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
      __align__(16) __nv_bfloat16 h[8], mi[8], l[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const Split3Bf16 t = split3_bf16(x[i]);
        h[i] = t.hi;
        mi[i] = t.mid;
        l[i] = t.lo;
      }
      *reinterpret_cast<uint4*>(P + o) = *reinterpret_cast<const uint4*>(h);
      *reinterpret_cast<uint4*>(P + plane + o) = *reinterpret_cast<const uint4*>(mi);
      *reinterpret_cast<uint4*>(P + 2 * plane + o) = *reinterpret_cast<const uint4*>(l);
    } else {
      __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
      __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const HiLoBf16 t = split_bf16(x[i]);
        h[i] = t.hi;
        l[i] = t.lo;
      }
      *reinterpret_cast<uint4*>(P + o) = *reinterpret_cast<const uint4*>(h);
      *reinterpret_cast<uint4*>(P + plane + o) = *reinterpret_cast<const uint4*>(l);
    }
  }
  __syncthreads();   // the tile is reused by the next item of a looping launch
  return m;          // this thread's max |x| (kFirst; 0 for kRescale)
}

// ------------------------------------------------ A: block maxima only
// For the fused-split gemm, which splits A itself.  An item is a piece of a
// 128-row block: a contiguous run of float4 when the rows are stored back to
// back (lda == K, 16-byte aligned), else a span of 64 loads of every row of
// the block (thread (x, y) of the 64 x 4 CTA reads load x of rows y, y + 4,
// ...); eight independent loads a thread are in flight, and the CTA folds
// one max per item.
constexpr int kAmaxLoads = 64;

enum AmaxMode { kAmaxFlat = 0, kAmaxRowsVec = 1, kAmaxRowsScalar = 2 };

struct AmaxShape {
  const float* A;
  int64_t M, K, lda;
  int parts;          // flat mode: pieces a block is cut into
  unsigned* amax;
};

template <int MODE>
__device__ __forceinline__ int64_t amax_items(const AmaxShape& a) {
  const int64_t nblk = (a.M + 127) / 128;
  if (MODE == kAmaxFlat) return nblk * a.parts;
  const int64_t span = kAmaxLoads * (MODE == kAmaxRowsVec ? 4 : 1);
  return nblk * ((a.K + span - 1) / span);
}

template <int MODE>
__device__ __forceinline__ void amax_item(const AmaxShape& a, int64_t item) {
  unsigned m = 0;
  int64_t b;
  if (MODE == kAmaxFlat) {
    b = item / a.parts;
    const int part = static_cast<int>(item - b * a.parts);
    const int64_t n4 = min(static_cast<int64_t>(128), a.M - b * 128) * a.K / 4;   // K % 4 == 0
    const int64_t per = (n4 + a.parts - 1) / a.parts;
    const int64_t lo = part * per, hi = min(n4, lo + per);
    const float4* p = reinterpret_cast<const float4*>(a.A + b * 128 * a.K);
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
  } else {
    constexpr int U = MODE == kAmaxRowsVec ? 4 : 1;   // floats per load
    constexpr int64_t span = kAmaxLoads * U;
    const int64_t nspan = (a.K + span - 1) / span;
    b = item / nspan;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int64_t k = (item - b * nspan) * span + static_cast<int64_t>(tx) * U;
    const int rows = static_cast<int>(min(static_cast<int64_t>(128), a.M - b * 128));
    const float* base = a.A + (b * 128) * a.lda + k;
    if (k < a.K) {
      for (int r0 = ty; r0 < rows; r0 += 32) {
        float v[8][U];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = r0 + 4 * i;
#pragma unroll
          for (int e = 0; e < U; ++e) v[i][e] = 0.0f;
          if (r >= rows) continue;
          const float* p = base + r * a.lda;
          if (U == 4 && k + 4 <= a.K) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p));
            const float t[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < U; ++e) v[i][e] = t[e];
          } else {
#pragma unroll
            for (int e = 0; e < U; ++e)
              if (k + e < a.K) v[i][e] = __ldg(p + e);
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int e = 0; e < U; ++e) m = max(m, abs_bits(v[i][e]));
      }
    }
  }
  fold_block_max(m, a.amax + b);
}

// --------------------------------------------------- tile decomposition
// One operand of the pack: its planes hold `rows` rows (M for A, N for B) of
// K values.  Stored with K contiguous (rows x K, ld >= K: A, or B given
// transposed) it is split in 32-row x 256-column tiles (rows_b/32 x
// ceil(pitch/256) a block of 128 rows); stored K x rows (ld >= rows: B, or A
// given transposed) in 64-k x 128-column tiles that transpose through shared
// memory (ceil(pitch/64) a block).  Items are numbered so that the items of
// one block are consecutive.  A CTA processes a contiguous range of items, so
// it meets a block boundary only every few dozen items and folds maxima and
// counts once per run of one block.
struct OpShape {
  const float* X;
  int64_t rows, ld;
  int64_t plane;            // elements from one plane to the next
  bool vec;                 // 16-byte aligned along the contiguous dimension
  bool kcontig;             // K contiguous in X (row tiles), else column tiles
  unsigned* amax;           // per block of 128 rows of the planes
  unsigned* cnt;            // per block: items done (zero on entry)
  void* planes;
};

struct PackShape {
  OpShape op[2];            // A, B
  int64_t K, pitch;

  __device__ int ktiles(const OpShape& o) const {
    return o.kcontig ? (int)((pitch + 255) / 256) : (int)((pitch + 63) / 64);
  }
  __device__ int items_of(const OpShape& o) const {
    if (!o.X || o.rows <= 0) return 0;
    return (int)((o.kcontig ? (o.rows + 31) / 32 : (o.rows + 127) / 128) * ktiles(o));
  }
  __device__ int items() const { return items_of(op[0]) + items_of(op[1]); }
  __device__ int64_t block_in(const OpShape& o, int l) const {
    return o.kcontig ? (int64_t)(l / ktiles(o)) / 4 : (int64_t)(l / ktiles(o));
  }
  // block of item i: A's blocks 0.., then B's blocks as -1 - b (operands are
  // selected by branches, never by a runtime index into op[])
  __device__ int64_t block_of(int i) const {
    const int na = items_of(op[0]);
    return i < na ? block_in(op[0], i) : -1 - block_in(op[1], i - na);
  }
};

// Split item l of operand o (unscaled); returns this thread's max |x|.
template <Prec PR>
__device__ __forceinline__ unsigned op_item(const PackShape& p, const OpShape& o, int l, float* tile) {
  const int kt = p.ktiles(o);
  if (o.kcontig)
    return split_rows_tile<PR, kFirst>(o.X, o.rows, p.K, o.ld, o.vec, o.amax, o.planes, o.plane, p.pitch,
                                         (int64_t)(l / kt) * 32, (int64_t)(l % kt) * 256);
  return split_cols_tile<PR, kFirst>(o.X, p.K, o.rows, o.ld, o.vec, o.amax, o.planes, o.plane, p.pitch,
                                       (int64_t)(l / kt) * 128, (int64_t)(l % kt) * 64, tile);
}

template <Prec PR>
__device__ __forceinline__ unsigned first_item(const PackShape& p, int i, float* tile) {
  const int na = p.items_of(p.op[0]);
  return i < na ? op_item<PR>(p, p.op[0], i, tile) : op_item<PR>(p, p.op[1], i - na, tile);
}

// The CTA that completed block b (fin: its final max bits) marks it ready
// (kBlockReady in its counter) once its planes are final: after the CTA's
// re-split, when there was one (the barrier orders every thread's stores
// before thread 0's release, which is cumulative over the counts it
// acquired as well).  A gemm launched while this kernel runs may load the
// block's planes as soon as it sees the bit.
__device__ __forceinline__ void mark_block_ready(unsigned* cnt, bool resplit) {
  if (resplit) __syncthreads();
  if (threadIdx.x == 0) red_or_release_gpu(cnt, kBlockReady);
}

// Close a run of `run` items of block `blk` (encoded as in block_of); the
// CTA that completes an out-of-range block re-splits it with its exponent.
template <Prec PR>
__device__ __forceinline__ void finish_op_block(const PackShape& p, const OpShape& o, int64_t b, unsigned m,
                                                unsigned run, float* tile) {
  const int kt = p.ktiles(o);
  if (o.kcontig) {
    const int64_t rows_b = min(static_cast<int64_t>(kScaleBlock), o.rows - b * kScaleBlock);
    const unsigned items = (unsigned)(((rows_b + 31) / 32) * kt);
    const unsigned fin = finish_run(m, o.amax + b, o.cnt + b, run, items);
    if (fin == 0xFFFFFFFFu) return;
    const bool resplit = block_exponent(fin) != 0;
    if (resplit) {
      for (int64_t k0 = 0; k0 < p.pitch; k0 += 256)
        for (int64_t q = b * kScaleBlock; q < b * kScaleBlock + rows_b; q += 32)
          split_rows_tile<PR, kRescale>(o.X, o.rows, p.K, o.ld, o.vec, o.amax, o.planes, o.plane,
                                          p.pitch, q, k0);
    }
    mark_block_ready(o.cnt + b, resplit);
  } else {
    const unsigned fin = finish_run(m, o.amax + b, o.cnt + b, run, (unsigned)kt);
    if (fin == 0xFFFFFFFFu) return;
    const bool resplit = block_exponent(fin) != 0;
    if (resplit) {
      for (int64_t k0 = 0; k0 < p.pitch; k0 += 64)
        split_cols_tile<PR, kRescale>(o.X, p.K, o.rows, o.ld, o.vec, o.amax, o.planes, o.plane, p.pitch,
                                        b * 128, k0, tile);
    }
    mark_block_ready(o.cnt + b, resplit);
  }
}

template <Prec PR>
__device__ __forceinline__ void finish_block(const PackShape& p, int64_t blk, unsigned m, unsigned run,
                                             float* tile) {
  if (blk >= 0)
    finish_op_block<PR>(p, p.op[0], blk, m, run, tile);
  else
    finish_op_block<PR>(p, p.op[1], -1 - blk, m, run, tile);
}

// Items [i0, i1) of one problem, in runs of one block each.
template <Prec PR>
__device__ __forceinline__ void pack_range(const PackShape& p, int i0, int i1, float* tile) {
  int i = i0;
  while (i < i1) {
    const int64_t blk = p.block_of(i);
    unsigned m = 0, run = 0;
    do {
      m = max(m, first_item<PR>(p, i, tile));
      ++run;
      ++i;
    } while (i < i1 && p.block_of(i) == blk);
    finish_block<PR>(p, blk, m, run, tile);
  }
}

// ------------------------------------------------ single-problem kernels
// CTA c takes the c-th contiguous share of the items.  Four CTAs a SM (at
// most 64 registers a thread).
template <Prec PR>
__global__ void __launch_bounds__(256, 4) pack_first_kernel(const PackShape p) {
  __shared__ __align__(16) float tile[kColTileFloats];
  // launched as a programmatic dependent of the stream's previous kernel
  // (often the previous execution's gemm, which reads these planes and
  // clears the block maxima and counters at its end)
  griddep_wait();
  // the gemm may be scheduled as soon as every CTA of this launch has
  // started (and so passed the wait above): its CTAs take the SMs this
  // launch leaves, run their prologue, and load each block of the planes
  // once the block is marked ready (or wait for this whole launch)
  griddep_launch_dependents();
  const int total = p.items();
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per;
  pack_range<PR>(p, i0, min(total, i0 + per), tile);
}

// Fused-split preparation in one launch: A's block maxima (grid-stride),
// then B packed as in pack_first_kernel (p holds B only; a contiguous
// share of its items per CTA).
template <Prec PR, int MODE>
__global__ void __launch_bounds__(256, 4) fused_prep_kernel(const AmaxShape a, const PackShape p) {
  __shared__ __align__(16) float tile[kColTileFloats];
  griddep_wait();   // as pack_first_kernel
  const int64_t na = amax_items<MODE>(a);
  for (int64_t i = blockIdx.x; i < na; i += gridDim.x) amax_item<MODE>(a, i);
  const int total = p.items();
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per;
  pack_range<PR>(p, i0, min(total, i0 + per), tile);
  griddep_launch_dependents();
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
  p.K = g.K, p.pitch = g.pitch;
  OpShape& a = p.op[0];
  a.X = q.A, a.rows = g.M, a.ld = g.lda, a.plane = static_cast<int64_t>(g.M) * g.pitch;
  a.vec = (reinterpret_cast<uintptr_t>(q.A) % 16 == 0) && (g.lda % 4 == 0);
  a.kcontig = true, a.amax = g.amaxA, a.cnt = g.cntA, a.planes = g.planesA;
  OpShape& b = p.op[1];
  b.X = q.B, b.rows = g.N, b.ld = g.ldb, b.plane = static_cast<int64_t>(g.N) * g.pitch;
  b.vec = (reinterpret_cast<uintptr_t>(q.B) % 16 == 0) && (g.ldb % 4 == 0);
  b.kcontig = false, b.amax = g.amaxB, b.cnt = g.cntB, b.planes = g.planesB;
  return p;
}

// Four CTAs a SM (64 registers a thread, a few dozen bytes of spills): the
// pack is bound by the bytes its CTAs hold in flight, and with three CTAs a SM
// (80 registers, no spills) the 512-problem group took 3% longer.
template <Prec PR>
__global__ void __launch_bounds__(256, 4) grouped_pack_kernel(const GroupedProblem* __restrict__ probs,
                                                           const GroupedPtrs* __restrict__ ptrs,
                                                           const int* __restrict__ prefix_g, int G) {
  __shared__ __align__(16) float tile[kColTileFloats];
  // the current problem's shape lives in shared memory: built in registers,
  // it held 128 registers a thread (two CTAs a SM)
  __shared__ PackShape shape;
  griddep_wait();   // launched as a programmatic dependent (as pack_first_kernel)
  const int* prefix = stage_prefix(prefix_g, G);
  const int total = prefix[G];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  int i = blockIdx.x * per;
  const int iend = min(total, i + per);
  while (i < iend) {
    // the part of this CTA's share that lies in problem g
    const int g = find_problem(prefix, G, i);
    const int e = min(iend, prefix[g + 1]);
    const GroupedPtrs& q = ptrs[g];
    if (q.alpha != 0.0f) {   // A and B are not read when alpha == 0 (uniform per CTA)
      __syncthreads();       // the previous problem's shape is no longer read
      if (threadIdx.x == 0) shape = problem_shape(probs[g], q);
      __syncthreads();
      pack_range<PR>(shape, i - prefix[g], e - prefix[g], tile);
    }
    i = e;
  }
  griddep_launch_dependents();
}

// ------------------------------------------- convolution image, split once
// The packed convolution splits its NHWC image once, element by element,
// into bf16 planes [plane][elems] (plane z = hi, mid, lo), or (ILV, two
// planes: bf16, or tf32 values in 32-bit words) into one image of twice the
// channels whose 16-channel groups hold hi then lo: element e = 16 g + j of
// a pixel's channels goes to 32 g + j (hi) and 32 g + 16 + j (lo), i.e.
// index 2e - (e mod 16) and 16 more.  One exponent for the whole image.  kFirst splits unscaled and folds max |x|
// into amax[0]; kRescale, launched after it, reads the final max and returns
// at once when the exponent is 0 (the usual case), else re-splits every
// element with it.  Four float4 loads a thread are in flight per iteration.
template <Prec PR, Pass PASS, bool ILV>
__global__ void __launch_bounds__(256) image_split_kernel(const float4* __restrict__ X, int64_t n4,
                                                           unsigned* __restrict__ amax,
                                                           void* __restrict__ planes, int64_t plane) {
  static_assert(PR != Prec::F32 && (ILV ? PR != Prec::BF16X6 : PR != Prec::TF32),
                "interleaved: two planes (bf16 or tf32); planar: bf16");
  __nv_bfloat16* P = static_cast<__nv_bfloat16*>(planes);
  float sc = 1.0f;
  if (PASS == kRescale) {
    const int e = block_exponent(*amax);
    if (e == 0) return;
    sc = pow2f(-e);
  }
  unsigned m = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i0 < n4; i0 += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + u * stride;
      v[u] = i < n4 ? X[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= n4) break;
      const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
      if (PASS == kFirst) {
#pragma unroll
        for (int j = 0; j < 4; ++j) m = max(m, abs_bits(x[j]));
      }
      if (PR == Prec::TF32) {
        float4 h, l;
        split_tf32(x[0] * sc, h.x, l.x);
        split_tf32(x[1] * sc, h.y, l.y);
        split_tf32(x[2] * sc, h.z, l.z);
        split_tf32(x[3] * sc, h.w, l.w);
        const int64_t e = 4 * i;
        float* Pf = static_cast<float*>(planes);
        *reinterpret_cast<float4*>(Pf + 2 * e - (e & 15)) = h;
        *reinterpret_cast<float4*>(Pf + 2 * e - (e & 15) + 16) = l;
      } else if (PR == Prec::BF16X6) {
        __align__(8) __nv_bfloat16 h[4], mi[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const Split3Bf16 t = split3_bf16(x[j] * sc);
          h[j] = t.hi;
          mi[j] = t.mid;
          l[j] = t.lo;
        }
        *reinterpret_cast<uint2*>(P + 4 * i) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(P + plane + 4 * i) = *reinterpret_cast<const uint2*>(mi);
        *reinterpret_cast<uint2*>(P + 2 * plane + 4 * i) = *reinterpret_cast<const uint2*>(l);
      } else {
        __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const HiLoBf16 t = split_bf16(x[j] * sc);
          h[j] = t.hi;
          l[j] = t.lo;
        }
        const int64_t e = 4 * i;
        const int64_t oh = ILV ? 2 * e - (e & 15) : e;
        const int64_t ol = ILV ? oh + 16 : plane + e;
        *reinterpret_cast<uint2*>(P + oh) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(P + ol) = *reinterpret_cast<const uint2*>(l);
      }
    }
  }
  if (PASS == kFirst) fold_block_max(m, amax);
}

// Launch with programmatic stream serialization: the kernel's CTAs may be
// scheduled while the stream's previous kernel finishes (its launch latency
// hidden); the kernel waits for that kernel (griddep_wait) before it reads
// or writes anything.
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), int grid, int threads, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

int grid_for(int64_t items, int sms) {
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  return static_cast<int>(items < cap ? (items > 0 ? items : 1) : cap);
}

OpShape make_op(const float* X, int64_t rows, int64_t ld, bool kcontig, unsigned* amax, unsigned* cnt,
                void* planes, int64_t plane) {
  OpShape o;
  o.X = X, o.rows = X ? rows : 0, o.ld = ld, o.plane = plane;
  o.vec = X && ld % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
  o.kcontig = kcontig, o.amax = amax, o.cnt = cnt, o.planes = planes;
  return o;
}

PackShape make_shape(const OpShape& a, const OpShape& b, int64_t K, int64_t pitch) {
  PackShape p;
  p.op[0] = a, p.op[1] = b, p.K = K, p.pitch = pitch;
  return p;
}

int64_t host_items(const OpShape& o, int64_t pitch) {
  if (!o.X || o.rows <= 0) return 0;
  return o.kcontig ? ((o.rows + 31) / 32) * ((pitch + 255) / 256) : ((o.rows + 127) / 128) * ((pitch + 63) / 64);
}

cudaError_t launch_first(Prec prec, const PackShape& p, int sms, cudaStream_t s) {
  const int64_t first = host_items(p.op[0], p.pitch) + host_items(p.op[1], p.pitch);
  if (first == 0) return cudaSuccess;
  const int grid = grid_for(first, sms);
  cudaError_t e;
  if (prec == Prec::TF32)
    e = launch_pdl(pack_first_kernel<Prec::TF32>, grid, 256, 0, s, p);
  else if (prec == Prec::BF16X6)
    e = launch_pdl(pack_first_kernel<Prec::BF16X6>, grid, 256, 0, s, p);
  else
    e = launch_pdl(pack_first_kernel<Prec::BF16>, grid, 256, 0, s, p);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

// Items per problem of the pack launch (host side, same tiling as above).
int pack_first_items(int64_t M, int64_t N, int64_t pitch) {
  return static_cast<int>(((M + 31) / 32) * ((pitch + 255) / 256) + ((N + 127) / 128) * ((pitch + 63) / 64));
}

cudaError_t pack_launch(Prec prec, const float* A, int64_t M, int64_t K, int64_t lda, const float* B,
                        int64_t N, int64_t ldb, unsigned* amaxA, unsigned* amaxB, unsigned* cntA,
                        unsigned* cntB, void* planesA, void* planesB, int64_t pitch, int sms,
                        cudaStream_t s, bool transA, bool transB) {
  const PackShape p = make_shape(make_op(A, M, lda, !transA, amaxA, cntA, planesA, M * pitch),
                                 make_op(B, N, ldb, transB, amaxB, cntB, planesB, N * pitch), K, pitch);
  return launch_first(prec, p, sms, s);
}

cudaError_t pack_fused_launch(Prec prec, const float* A, int64_t M, int64_t K, int64_t lda,
                              const float* B, int64_t N, int64_t ldb, unsigned* amaxA,
                              unsigned* amaxB, unsigned* cntB, void* planesB, int64_t pitch, int sms,
                              cudaStream_t s, int64_t K_b, bool transB) {
  // K_b: rows of B when they differ from A's row length (the convolution
  // scans its image as one M = 1 row of all its elements)
  const PackShape p = make_shape(make_op(nullptr, 0, 1, true, nullptr, nullptr, nullptr, 0),
                                 make_op(B, N, ldb, transB, amaxB, cntB, planesB, N * pitch),
                                 K_b >= 0 ? K_b : K, pitch);
  AmaxShape a;
  a.A = A, a.M = M, a.K = K, a.lda = lda, a.amax = amaxA, a.parts = 1;
  const int64_t nblk = (M + 127) / 128;
  const bool vec = lda % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
  int mode = vec ? kAmaxRowsVec : kAmaxRowsScalar;
  int64_t na;
  if (vec && lda == K) {
    mode = kAmaxFlat;
    a.parts = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(
        (4 * static_cast<int64_t>(sms) + nblk - 1) / nblk, (128 * K / 4 + 2047) / 2048)));
    na = nblk * a.parts;
  } else {
    const int64_t span = kAmaxLoads * (vec ? 4 : 1);
    na = nblk * ((K + span - 1) / span);
  }
  if (M == 0 || K == 0) na = 0, a.M = 0;
  const int64_t total = na + host_items(p.op[1], pitch);
  if (total == 0) return cudaSuccess;
  const int grid = grid_for(total, sms);
  cudaError_t e;
  if (prec == Prec::TF32) {
    if (mode == kAmaxFlat) e = launch_pdl(fused_prep_kernel<Prec::TF32, kAmaxFlat>, grid, 256, 0, s, a, p);
    else if (mode == kAmaxRowsVec) e = launch_pdl(fused_prep_kernel<Prec::TF32, kAmaxRowsVec>, grid, 256, 0, s, a, p);
    else e = launch_pdl(fused_prep_kernel<Prec::TF32, kAmaxRowsScalar>, grid, 256, 0, s, a, p);
  } else if (prec == Prec::BF16) {
    if (mode == kAmaxFlat) e = launch_pdl(fused_prep_kernel<Prec::BF16, kAmaxFlat>, grid, 256, 0, s, a, p);
    else if (mode == kAmaxRowsVec) e = launch_pdl(fused_prep_kernel<Prec::BF16, kAmaxRowsVec>, grid, 256, 0, s, a, p);
    else e = launch_pdl(fused_prep_kernel<Prec::BF16, kAmaxRowsScalar>, grid, 256, 0, s, a, p);
  } else {
    return cudaErrorInvalidValue;   // the fused kernel splits A in two (three-product modes only)
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t pack_rows_panel_launch(Prec prec, const float* A, int64_t rows, int64_t K, int64_t lda,
                                   unsigned* amaxA, unsigned* cntA, void* planesA,
                                   int64_t plane_stride, int64_t pitch, int sms, cudaStream_t s) {
  const PackShape p = make_shape(make_op(A, rows, lda, true, amaxA, cntA, planesA, plane_stride),
                                 make_op(nullptr, 0, 1, false, nullptr, nullptr, nullptr, 0), K, pitch);
  return launch_first(prec, p, sms, s);
}

cudaError_t image_split_launch(Prec prec, const float* X, int64_t elems, unsigned* amax, void* planes,
                               int sms, cudaStream_t s, bool interleave) {
  if (prec == Prec::F32) return cudaErrorInvalidValue;
  if (interleave ? (prec == Prec::BF16X6 || elems % 16 != 0) : prec == Prec::TF32) return cudaErrorInvalidValue;
  if (elems % 4 != 0 || reinterpret_cast<uintptr_t>(X) % 16 != 0) return cudaErrorInvalidValue;
  const int64_t n4 = elems / 4;
  if (n4 == 0) return cudaSuccess;
  const int grid = grid_for((n4 + 1023) / 1024, sms);
  const float4* X4 = reinterpret_cast<const float4*>(X);
  void* P = planes;
  if (prec == Prec::TF32) {
    image_split_kernel<Prec::TF32, kFirst, true><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
    image_split_kernel<Prec::TF32, kRescale, true><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
  } else if (prec == Prec::BF16X6) {
    image_split_kernel<Prec::BF16X6, kFirst, false><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
    image_split_kernel<Prec::BF16X6, kRescale, false><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
  } else if (interleave) {
    image_split_kernel<Prec::BF16, kFirst, true><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
    image_split_kernel<Prec::BF16, kRescale, true><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
  } else {
    image_split_kernel<Prec::BF16, kFirst, false><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
    image_split_kernel<Prec::BF16, kRescale, false><<<grid, 256, 0, s>>>(X4, n4, amax, P, elems);
  }
  return cudaGetLastError();
}

cudaError_t grouped_pack_launch(Prec prec, const GroupedProblem* probs, const GroupedPtrs* ptrs,
                                const int* first_prefix, int first_total, int G, int sms,
                                cudaStream_t s) {
  const size_t dyn = (G + 1) <= 4096 ? static_cast<size_t>(G + 1) * sizeof(int) : 0;
  if (first_total == 0) return cudaSuccess;
  // six waves of four CTAs a SM: the problems' items differ in size, and
  // with short shares the block scheduler evens out the SMs' work (512
  // problems: two waves 363 us, six 354 us; one wave of shares weighted by
  // their elements, without that rebalancing, 431 us)
  const int gf = static_cast<int>(std::min<int64_t>(first_total, static_cast<int64_t>(sms) * 24));
  cudaError_t e;
  if (prec == Prec::TF32)
    e = launch_pdl(grouped_pack_kernel<Prec::TF32>, gf, 256, dyn, s, probs, ptrs, first_prefix, G);
  else if (prec == Prec::BF16X6)
    e = launch_pdl(grouped_pack_kernel<Prec::BF16X6>, gf, 256, dyn, s, probs, ptrs, first_prefix, G);
  else
    e = launch_pdl(grouped_pack_kernel<Prec::BF16>, gf, 256, dyn, s, probs, ptrs, first_prefix, G);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace gb
