// Split-precision tensor-core gemm for sm_103a: C = alpha * A * B + beta * C
// with FP32 semantics, computed as three bf16 (or tf32) tensor-core products
// per k-step, hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory
// (or, with three bf16 planes hi/mid/lo, as the six products whose plane
// indices sum to at most two).
//
// The paper's gemm recipe (Section I; Section VI-A) is two-level tiling,
// array packing, register blocking and prefetching, with full tiles kept
// apart from partial ones, and on GPUs coalesced accesses plus explicit
// staging global -> shared -> registers with synchronization.  On sm_103a that
// becomes:
//   * packing: a separate pass writes each operand as hi/lo planes, K-major,
//     with per-block power-of-two scaling (split.cu);
//   * tiling: persistent CTAs walk 128 x BN output tiles (optionally split
//     along K); each tile's k-loop streams 128-byte k-chunks of the four
//     planes through a STAGES-deep shared-memory ring filled by TMA;
//   * register blocking -> tensor memory: one elected thread issues
//     tcgen05.mma into a TMEM accumulator (up to four buffers, so that the
//     epilogue of one accumulation block overlaps the MMAs of the next ones);
//   * full vs partial tiles: TMA zero-fills the out-of-range part of edge
//     tiles on load, so the main loop never branches; only the epilogue
//     masks rows/columns, and full tiles take a vectorised store path;
//   * accumulation blocks: every kb k-chunks the epilogue warps fold the TMEM
//     partial sum into FP32 registers with round-to-nearest adds, which bounds
//     how many products the tensor core's own accumulation chains together.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = MMA issuer and
// TMEM owner, warps 2..5 = epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
//
// Fused-split variant (the packing of A moved into the main loop): TMA
// brings only B's planes.  Copy warps stage 128 x 64 (bf16) or 128 x 32
// (tf32) FP32 blocks of A in shared memory with cp.async; split warps split
// them with the packing pass's arithmetic and the block exponent found by a
// max-only pass over A, and write hi/lo into the stage in the layout a
// 128-byte-swizzled TMA load would have produced, then arrive on the stage's
// full barrier (which completes on their arrivals plus B's bytes).  A never
// exists as planes in memory: its operand traffic is one FP32 read instead
// of a read, a write and a re-read.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "internal.h"
#include "ptx.cuh"
#include "scale.cuh"
#include "split_arith.cuh"
#include "epilogue.cuh"
#include "tile_order.cuh"

namespace gb {

// Tile and pipeline geometry of one kernel variant.  A k-chunk is one
// swizzle span of every row, 128 bytes.  Instantiated for tile widths 64 and
// 128.  A 256-wide tile (two epilogue warpgroups of 128 columns each, which
// this geometry supports) measured 1.1-1.2 PFLOP/s on GB300 against 1.6 for
// 128, with the 128-byte swizzle (2-deep ring) and with the 64-byte swizzle
// (4-deep ring) alike, so it is not offered.
//
// NP = 3: the six-product bf16 mode, three planes per operand (hi, mid, lo);
// a stage holds all six, so the ring is two stages deep.  Each accumulator
// buffer is two BN-column accumulators: hi*hi alone, and the five smaller
// products.  The tensor core's FP32 accumulation drops low bits of the
// running sum at every MMA; kept apart, the small products lose bits only
// relative to their own (2^-8 smaller) sum, and the hi*hi chain is one MMA
// per k-step instead of six.
template <int BN, bool TF32, bool FUSED = false, int NP = 2, int EPI = 0>
struct TcCfg {
  static_assert(NP == 2 || (NP == 3 && !TF32 && !FUSED), "three planes: packed bf16 only");
  static constexpr int BM = 128;
  static constexpr int SW = 128;                       // bytes of one row per k-chunk
  static constexpr int A_PLANE = BM * SW;
  static constexpr int B_PLANE = BN * SW;
  static constexpr int STAGE = NP * A_PLANE + NP * B_PLANE;
  // operand ring depth (the fused variant gives room to the staging of A)
  // (EPI = 2, the compensated epilogue: its second epilogue warpgroup's
  // staging buffers take the fourth stage's room at BN 64)
  static constexpr int STAGES = (FUSED || NP == 3) ? 2 : (BN == 64 ? (EPI == 2 ? 3 : 4) : BN == 128 ? 3 : 2);
  static constexpr int BK = SW / (TF32 ? 4 : 2);       // elements per k-chunk
  static constexpr int KSTEPS = SW / 32;               // MMAs (32-byte K slices) per chunk and product
  // epilogue warpgroups: two for the 128-wide tiles of the fused variant
  // (with its extra warps, one warpgroup holding 128 columns would run out of
  // registers) and of the grouped launch (EPI = 1: its tiles are short in K,
  // so the epilogue, at half the time per tile with each thread draining 64
  // columns, is what the MMAs wait for), and for every tile width of the
  // compensated epilogue (EPI = 2: it folds every k-chunk, six operations an
  // output per fold, so the fold is what the MMAs wait for); one elsewhere
  // (at long K the epilogue hides behind the MMAs, and the extra warps cost
  // about 2% there)
  static constexpr int EPI_WG = (BN == 256 || EPI == 2 || (BN == 128 && (FUSED || EPI == 1))) ? 2 : 1;
  static constexpr int EPI_COLS = BN / EPI_WG;         // columns per epilogue thread
  static constexpr int ACC_COLS = NP == 3 ? 2 * BN : BN;   // TMEM columns of one accumulator buffer
  // accumulator buffers: as many as TMEM holds, up to four, so that the MMA
  // thread runs ahead of the epilogue across short-K tiles
  static constexpr int NACC = 512 / ACC_COLS >= 4 ? 4 : 512 / ACC_COLS;
  static constexpr int TMEM_COLS = NACC * ACC_COLS;
  static constexpr int EPI_PITCH = 33;                 // floats per staged row (bank-conflict free)
  static constexpr int EPI_BYTES = 4 * EPI_WG * 32 * EPI_PITCH * 4;   // one 32x32 buffer per epilogue warp
  static constexpr int BAR_BYTES = 512;
  // fused variant: two staging buffers for one FP32 k-chunk of A each
  // (128 rows of BK floats, as 128-byte-wide boxes swizzled like a
  // SWIZZLE_128B TMA load), filled by TMA or cp.async
  static constexpr int STG_ROW = BK * 4;
  static constexpr int STG_BYTES = FUSED ? 128 * STG_ROW : 0;
  // (as deep as shared memory allows: the staging ring is what keeps enough
  // bytes of A in flight to cover memory latency)
  static constexpr int STG_STAGES = !FUSED ? 0 : BN == 64 ? (TF32 ? 6 : 3) : (TF32 ? 4 : 2);
  static constexpr int OFF_STG = STAGES * STAGE;
  static constexpr int OFF_EPI = OFF_STG + STG_STAGES * STG_BYTES;
  static constexpr int OFF_BAR = OFF_EPI + EPI_BYTES;
  static constexpr int SMEM = OFF_BAR + BAR_BYTES + 1024;
  // fused variant: SPLIT_THREADS threads stage A and split it into the
  // stage (at most 12 warps in all, which leaves 168 registers a thread)
  static constexpr int SPLIT0 = 64 + 128 * EPI_WG;
  static constexpr int SPLIT_THREADS = FUSED ? (BN == 128 ? 64 : 128) : 0;
  static constexpr int THREADS = SPLIT0 + SPLIT_THREADS;
  static_assert(SMEM <= 232448, "shared memory budget");
  static_assert(TMEM_COLS <= 512, "tensor memory budget");
};

// Source of A for the fused-split variant.
struct FusedA {
  const float* A;
  int64_t lda;
  int M, K;
  bool vec;                 // staged by TMA (rows 16-byte aligned; for a convolution,
                            // im2col boxes of whole taps), else by cp.async
  const unsigned* amaxA;    // block maxima from the max-only pass
  int amax_stride;          // 1, or 0 when one exponent covers all of A
  int conv, H, W, C;        // A = patch matrix of an NHWC image (R x S filter, odd
  int R, S;                 // sizes, zero padding (R-1)/2 and (S-1)/2)
  int box_c;                // channels per im2col box: 32 (128-byte rows) or 16 (64-byte rows)
  int N;                    // images (the packed variant's plane z starts at image z N)
};

// Scheduling policy of one gemm: units are (split, tile) pairs.
struct SingleSched {
  static constexpr int kEpi = 0;   // epilogue geometry (TcCfg's EPI)
  static constexpr bool kCompensated = false;
  static constexpr bool kDynamic = false;     // (the packed convolution takes units dynamically)
  const CUtensorMap* tmA;
  const CUtensorMap* tmB;
  const TcArgs* a;
  __device__ int units() const { return a->num_units; }
  __device__ int kb() const { return a->kb; }
  __device__ int* err() const { return a->err; }
  // L2 priority of A's loads: with tiles grouped along M, consecutive waves
  // of CTAs keep the same rows of A, so they are loaded evict-last (8192^3
  // under ncu: 1.98-2.05 ms with it, 2.02 ms without, within the spread
  // between boxes; marking B evict-first as well, as it is used within one
  // wave only, doubled the DRAM reads: its column blocks left L2 before the
  // wave's other CTAs had read them)
  __device__ int l2_hints() const { return a->group_m > 1 ? 1 : 0; }
  __device__ int* unit_ctr() const { return a->unit_ctr; }
  __device__ unsigned* state() const { return a->state; }
  __device__ int state_words() const { return a->state_words; }
  // pack counters of A's and B's blocks with their ready bit (null: wait
  // for the whole packing kernel)
  __device__ const unsigned* readyA() const { return a->readyA; }
  __device__ const unsigned* readyB() const { return a->readyB; }
  __device__ Work work(int u) const {
    Work w;
    const int t = u % a->num_tiles;
    w.prob = 0;
    w.ks = u / a->num_tiles;
    raster(t, a->tiles_m, a->tiles_n, a->group_m, w.tm, w.tn);
    w.tm += a->tm0;
    w.c0 = w.ks * a->chunks_per_split;
    w.c1 = min(w.c0 + a->chunks_per_split, a->chunks_total);
    return w;
  }
  __device__ const CUtensorMap* mapA(int) const { return tmA; }
  __device__ const CUtensorMap* mapB(int) const { return tmB; }
  __device__ EpiView epi(int) const {
    EpiView v;
    v.M = a->M, v.N = a->N, v.C = a->C, v.ldc = a->ldc, v.alpha = a->alpha, v.beta = a->beta;
    v.amaxA = a->amaxA, v.amaxB = a->amaxB, v.partial = a->partial, v.split_k = a->split_k;
    v.amaxA_stride = a->conv ? 0 : 1;
    return v;
  }
  __device__ FusedA srcA(int) const {
    return FusedA{a->A, a->lda, a->M, a->K, a->vecA != 0, a->amaxA, a->conv ? 0 : 1,
                  a->conv, a->conv_H, a->conv_W, a->conv_C, a->conv_R, a->conv_S, a->conv_box_c,
                  a->conv_N};
  }
};

// A single gemm with the compensated epilogue: the per-fold TMEM partial
// sums are added into the FP32 registers with an error-free transformation
// (TwoSum), the rounding error of every addition kept in a second register
// per output and added back once at the end, so that the register sum of
// the folds is as accurate as if it were computed in twice the precision.
// Each thread holds two values per column (32 columns a thread).
struct SingleSchedComp : SingleSched {
  static constexpr int kEpi = 2;
  static constexpr bool kCompensated = true;
};

// Scheduling policy of a grouped launch: units are the tiles of all problems,
// listed problem after problem (problems ordered longest-K first on the host,
// each problem's tiles in grouped raster order); the table gives a unit's
// problem, tile coordinates and k-chunk count in one 16-byte load.
struct GroupedSched {
  static constexpr int kEpi = 1;
  static constexpr bool kCompensated = false;
  static constexpr bool kDynamic = true;      // problems of every size: units taken dynamically
  const GroupedArgs* a;
  __device__ int l2_hints() const { return 0; }   // problems of every shape: no priority
  __device__ int* unit_ctr() const { return a->unit_ctr; }
  __device__ unsigned* state() const { return a->state; }
  __device__ int state_words() const { return a->state_words; }
  __device__ const unsigned* readyA() const { return nullptr; }
  __device__ const unsigned* readyB() const { return nullptr; }
  __device__ int units() const { return a->num_units; }
  __device__ int kb() const { return a->kb; }
  __device__ int* err() const { return a->err; }
  __device__ Work work(int u) const {
    const int4 e = __ldg(reinterpret_cast<const int4*>(a->units) + u);
    Work w;
    w.prob = e.x;
    w.tm = e.y;
    w.tn = e.z;
    w.ks = 0;
    w.c0 = 0;
    w.c1 = e.w;
    return w;
  }
  __device__ const CUtensorMap* mapA(int g) const { return &a->probs[g].tmA; }
  __device__ const CUtensorMap* mapB(int g) const { return &a->probs[g].tmB; }
  __device__ EpiView epi(int g) const {
    const GroupedProblem& p = a->probs[g];
    const GroupedPtrs& q = a->ptrs[g];
    EpiView v;
    v.M = p.M, v.N = p.N, v.C = q.C, v.ldc = p.ldc, v.alpha = q.alpha, v.beta = q.beta;
    v.amaxA = p.amaxA, v.amaxB = p.amaxB, v.partial = nullptr, v.split_k = 1;
    v.amaxA_stride = 1;
    return v;
  }
};

// Two floats rounded to bf16 (nearest even) in one instruction: a in the low
// half, b in the high half.
__device__ __forceinline__ unsigned cvt_bf16x2(float a, float b) {
  unsigned d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  return d;
}

// s + x with its rounding error kept: s becomes fl(s + x) and e gains the
// exact error (s + x) - fl(s + x) of that addition (Knuth's TwoSum, six
// round-to-nearest operations, no branch; exact unless an operation
// overflows).  Summing the errors in e and adding e to s once at the end is
// the compensated summation of the values x.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  const float t = __fadd_rn(s, x);
  const float xv = __fsub_rn(t, s);             // the part of x that went into t
  const float sv = __fsub_rn(t, xv);            // the part of s that went into t
  const float err = __fadd_rn(__fsub_rn(s, sv), __fsub_rn(x, xv));
  s = t;
  e = __fadd_rn(e, err);
}

// Fused variant: split one 16-byte output group (x scaled by sf) into the hi
// and lo planes of a stage.  Row r of a plane holds 128 bytes; its 16-byte
// group q sits at position q ^ (r % 8), the 128-byte swizzle.  FINITE: the
// block holds no Inf/NaN (its max is finite), so the non-finite cases of the
// split can be skipped and bf16 pairs converted in one instruction; for
// finite values the result is the same bits as split_bf16 / split_tf32.
template <bool TF32, int EPG, bool FINITE>
__device__ __forceinline__ void fused_store(uint8_t* hi_plane, uint8_t* lo_plane, int r, int q,
                                            const float (&x)[EPG], float sf) {
  const int off = r * 128 + ((q ^ (r & 7)) << 4);
  if (FINITE && TF32) {
    float hv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float xs = x[j] * sf;
      const unsigned u = __float_as_uint(xs);
      hv[j] = __uint_as_float((u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u);
      const unsigned d = __float_as_uint(__fsub_rn(xs, hv[j]));
      lv[j] = __uint_as_float((d + 0xFFFu + ((d >> 13) & 1u)) & 0xFFFFE000u);
    }
    *reinterpret_cast<float4*>(hi_plane + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4*>(lo_plane + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  } else if (FINITE) {
    unsigned hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float a = x[2 * j] * sf, b = x[2 * j + 1] * sf;
      const unsigned hp = cvt_bf16x2(a, b);
      const float ha = __uint_as_float(hp << 16), hb = __uint_as_float(hp & 0xFFFF0000u);
      hw[j] = hp;
      lw[j] = cvt_bf16x2(__fsub_rn(a, ha), __fsub_rn(b, hb));
    }
    *reinterpret_cast<uint4*>(hi_plane + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(lo_plane + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  } else if (TF32) {
    float4 h, l;
    split_tf32(x[0] * sf, h.x, l.x);
    split_tf32(x[1] * sf, h.y, l.y);
    split_tf32(x[2] * sf, h.z, l.z);
    split_tf32(x[3] * sf, h.w, l.w);
    *reinterpret_cast<float4*>(hi_plane + off) = h;
    *reinterpret_cast<float4*>(lo_plane + off) = l;
  } else {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const HiLoBf16 t = split_bf16(x[j] * sf);
      h[j] = t.hi;
      l[j] = t.lo;
    }
    *reinterpret_cast<uint4*>(hi_plane + off) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo_plane + off) = *reinterpret_cast<const uint4*>(l);
  }
}

// Fused variant: split rows t, t + NT, ... of a staged chunk into the hi/lo
// planes.  The chunk is a row of boxes of 128 rows each: BW = 128-byte box
// rows in the SWIZZLE_128B layout (16-byte unit u of row r at u ^ (r % 8)),
// or BW = 64-byte rows in the SWIZZLE_64B layout (u ^ ((r / 2) % 4)).
// PARTIAL: only the first `valid` 16-byte units of each row hold data (the
// last chunk of a convolution whose boxes past K were not loaded); the rest
// are split as zeros.
template <bool TF32, bool FINITE, int NT, int BW = 128, bool PARTIAL = false>
__device__ __forceinline__ void fused_split_rows(const uint8_t* sbuf, uint8_t* hi_plane,
                                                 uint8_t* lo_plane, int t, float sf, int valid = 0) {
  constexpr int EPG = TF32 ? 4 : 8;   // elements per 16-byte output group
  constexpr int UPB = BW / 16;        // 16-byte units per box row
  constexpr int BOXB = 128 * BW;      // bytes of one box
  static_assert(BW == 128 || BW == 64, "box width");
#pragma unroll 1
  for (int r = t; r < 128; r += NT) {
    const int sw = BW == 128 ? (r & 7) : ((r >> 1) & 3);
    float x[8][EPG];
#pragma unroll
    for (int g = 0; g < 8; ++g)
#pragma unroll
      for (int h = 0; h < EPG / 4; ++h) {
        const int j = g * (EPG / 4) + h;   // 16-byte unit of the row
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (!PARTIAL || j < valid)
          v = *reinterpret_cast<const float4*>(sbuf + (j / UPB) * BOXB + r * BW + (((j % UPB) ^ sw) << 4));
        x[g][4 * h] = v.x, x[g][4 * h + 1] = v.y, x[g][4 * h + 2] = v.z, x[g][4 * h + 3] = v.w;
      }
#pragma unroll
    for (int g = 0; g < 8; ++g) fused_store<TF32, EPG, FINITE>(hi_plane, lo_plane, r, g, x[g], sf);
  }
}

// FBW (fused variant): row bytes of the staged boxes of A, 128, or 64 for a
// convolution staged in 16-channel im2col boxes (its own instantiation, so
// that the 128-byte path keeps its registers).
// CONVA != 0: the packed convolution.  A is the patch matrix of the image's
// bf16 planes, loaded as im2col boxes of one tap; B's planes are packed as
// usual.  CONVA = 64 (C a multiple of 64): one box of 64 channels (128-byte
// rows) a plane and chunk, laid out as a packed A plane (128-byte swizzle).
// CONVA = 32 (two planes): the planes are interleaved by 16-channel groups
// (hi then lo of a group), and a box is one group: for bf16 64-byte rows in
// the 64-byte swizzle, four boxes a chunk, k-step kk reading box kk (hi at
// its rows' first 32 bytes, lo at their last); for tf32 128-byte rows in the
// 128-byte swizzle, two boxes a chunk, k-step kk reading box kk / 2 at
// 32 (kk mod 2) (hi) and 64 more (lo).  CONVA = 16 (any
// plane count): four boxes of 16 channels a plane, 32-byte rows in the
// 32-byte swizzle, k-step kk being the 4 KB sub-tile kk of each A plane.
// With 16-channel groups, boxes of a last, partial chunk past K are neither
// loaded nor multiplied.
template <int BN, bool TF32, class Sched, bool FUSED = false, int NP = 2, int FBW = 128,
          int CONVA = 0>
__device__ __forceinline__ void tc_gemm_body(const Sched& sc) {
  using Cfg = TcCfg<BN, TF32, FUSED, NP, Sched::kEpi>;
  static_assert(CONVA == 0 || (!FUSED && ((CONVA == 32 && NP == 2) || ((CONVA == 16 || CONVA == 64) && !TF32))),
                "packed convolution: 32 (interleaved planes), or bf16 16- or 64-channel boxes");
  constexpr bool CB16 = CONVA == 16;
  constexpr bool CB32 = CONVA == 32;
  constexpr bool CGRP = CB16 || CB32;   // k-steps lie in 16-channel groups of one tap
  constexpr int CBOX = 128 * 32;   // bytes of one 16-channel bf16 im2col box
  constexpr int IBOX = TF32 ? 128 * 128 : 128 * 64;   // bytes of one interleaved hi|lo box
  constexpr int GSTEPS = TF32 ? 2 : 1;                // k-steps per 16-channel group
  constexpr int KELEM = TF32 ? 8 : 16;                // elements per k-step
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (sbase - raw);
  int* const err = sc.err();
  const int nunits = sc.units();
  const int kb = sc.kb();

  // stage ring | A staging (fused) | epilogue buffers | barrier block
  float* epi_buf = reinterpret_cast<float*>(smem + Cfg::OFF_EPI);
  uint8_t* bar_area = smem + Cfg::OFF_BAR;
  const uint32_t bar0 = sbase + Cfg::OFF_BAR;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  constexpr int NACC = Cfg::NACC;
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + NACC + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 2 * NACC);
  // fused variant: staging buffer b holds a copied chunk / is free again
  constexpr int NSTG = Cfg::STG_STAGES;
  auto stg_full_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 * NACC + 1 + b); };
  auto stg_empty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 * NACC + 1 + NSTG + b); };
  constexpr int NBAR = 2 * STAGES + 2 * NACC + 1 + 2 * NSTG;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_area + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // DYN (the packed convolution, the grouped launch): units are taken from a
  // per-launch counter as a CTA becomes ready for one, instead of every
  // gridDim.x-th, so that SMs that run faster, or got shorter units, take
  // more (with a static order the SMs of the 16-channel convolution finished
  // up to a third apart).  The producer takes each unit (one unit ahead, so
  // that the atomic's latency overlaps a unit of loads), and publishes it
  // with its work entry in a shared-memory queue, which the MMA thread and
  // the epilogue warps read in the same order; -1 ends it.
  constexpr bool DYN = CONVA != 0 || Sched::kDynamic;
  constexpr int QD = 8;
  int* const q_unit = reinterpret_cast<int*>(bar_area + 8 * NBAR + 16);
  Work* const q_work = reinterpret_cast<Work*>(bar_area + 8 * NBAR + 16 + 4 * QD);
  const uint32_t qbar0 = bar0 + 8u * NBAR + 16u + 4u * QD + static_cast<uint32_t>(sizeof(Work)) * QD;
  auto qfull_bar = [&](int s) { return qbar0 + 8u * s; };
  auto qempty_bar = [&](int s) { return qbar0 + 8u * (QD + s); };
  static_assert((16 + 4 * QD + sizeof(Work) * QD) % 8 == 0, "queue barriers 8-byte aligned");
  static_assert(8 * NBAR + 16 + (DYN ? 4 * QD + static_cast<int>(sizeof(Work)) * QD + 16 * QD : 0) <=
                    Cfg::BAR_BYTES,
                "barrier block");

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1 + Cfg::SPLIT_THREADS / 32);   // producer + one per split warp
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 128 * Cfg::EPI_WG);
    }
    mbar_init(drain_bar, 1);
    if constexpr (DYN) {
      for (int s = 0; s < QD; ++s) {
        mbar_init(qfull_bar(s), 1);                         // the producer
        mbar_init(qempty_bar(s), 1 + 4 * Cfg::EPI_WG);      // the MMA thread, one per epilogue warp
      }
    }
    if constexpr (FUSED) {
      // a staging buffer fills on one TMA issuer's arrival (plus its bytes)
      // or on every split thread's cp.async arrival
      const uint32_t fill_count = sc.srcA(0).vec ? 1u : static_cast<uint32_t>(Cfg::SPLIT_THREADS);
      for (int b = 0; b < NSTG; ++b) {
        mbar_init(stg_full_bar(b), fill_count);
        mbar_init(stg_empty_bar(b), Cfg::SPLIT_THREADS / 32);
      }
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the first problem's tensor maps (kernel parameters or host-written
  // tables, not outputs of the previous kernel) are fetched meanwhile
  if (warp == 0 && lane == 0 && nunits > 0) {
    if (!FUSED && CONVA == 0) tma_prefetch_desc(sc.mapA(0));
    tma_prefetch_desc(sc.mapB(0));
  }
  // The prologue above overlaps the packing kernel.  Every role but the TMA
  // producer waits here until that kernel has completed and its writes are
  // visible.  The producer of a packed gemm whose operands that kernel packs
  // (readyA/readyB set; all of its CTAs have started when this launch
  // starts, so none waits for an SM this launch holds) instead waits for
  // each block of the planes it loads to be marked ready, so that its first
  // loads overlap the end of the packing; it reads nothing else that kernel
  // wrote.
  const unsigned* const readyA = (!FUSED && CONVA == 0 && !DYN) ? sc.readyA() : nullptr;
  const unsigned* const readyB = (!FUSED && CONVA == 0 && !DYN) ? sc.readyB() : nullptr;
  if (warp != 0 || readyA == nullptr) griddep_wait();
  // the stream's next kernel (the split-K fix-up, or the next execution's
  // packing) may be scheduled now: it waits for this launch to complete
  // before it touches anything, and only its launch latency overlaps
  griddep_launch_dependents();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    bool fused_tma = false;
    if constexpr (FUSED) fused_tma = sc.srcA(0).vec;
    if (lane == 0 && fused_tma) {
      if constexpr (FUSED) {
        // Fused variant with A staged by TMA: this thread feeds both rings,
        // A's staging buffers and B's stages, each as far ahead as its ring
        // allows, polling both without blocking.
        constexpr int NSTG_ = Cfg::STG_STAGES;
        constexpr int BOX = 128 * 128;
        const uint32_t stg0 = sbase + Cfg::OFF_STG;
        struct Cur {
          int u, c;
          Work w;
          bool have;
        };
        auto first_c = [&](Cur& q, int u0) {
          q.have = false;
          for (q.u = u0; q.u < nunits; q.u += gridDim.x) {
            q.w = sc.work(q.u);
            if (q.w.c0 < q.w.c1) {
              q.have = true;
              q.c = q.w.c0;
              break;
            }
          }
        };
        auto adv = [&](Cur& q) {
          if (++q.c >= q.w.c1) first_c(q, q.u + gridDim.x);
        };
        Cur aq{}, bq{};
        first_c(aq, blockIdx.x);
        bq = aq;
        const CUtensorMap* mA = sc.mapA(0);
        const CUtensorMap* mB = sc.mapB(0);
        const FusedA fa = sc.srcA(0);
        tma_prefetch_desc(mA);
        tma_prefetch_desc(mB);
        uint32_t aslot = 0, aph = 0, bstage = 0, bph = 0;
        uint32_t a_used = 0, a_par = 0, b_used = 0, b_par = 0;   // per buffer: filled once / last parity
        bool ok = true;
        uint32_t idle = 0;
        uint64_t t0 = 0;
        while (aq.have || bq.have) {
          bool prog = false;
          if (aq.have && mbar_test_wait(stg_empty_bar(aslot), aph ^ 1u)) {
            const uint32_t fb = stg_full_bar(aslot);
            if (fa.conv) {
              // patch-matrix boxes: 128 output pixels from the tile's first,
              // box_c channels of one tap (the host checked C % box_c == 0);
              // output (h, w) starts at input (h - (R-1)/2, w - (S-1)/2) and
              // tap (r, s) = (tap / S, tap % S) adds its offsets.  Boxes of
              // a last, partial chunk that lie past K are not loaded: the
              // split warps zero those units.
              const int hw = fa.H * fa.W;
              const int p0 = aq.w.tm * 128;
              const int n0 = p0 / hw, rem = p0 - n0 * hw;
              const int h0 = rem / fa.W, w0 = rem - h0 * fa.W;
              constexpr int BC = FBW / 4;                       // channels per box
              constexpr int BOXB = 128 * FBW;                   // bytes of one box
              constexpr int NBOX = Cfg::STG_ROW / FBW;
              const int kc0 = aq.c * Cfg::BK;
              // (32-channel boxes: the host chose them only when K has no partial chunk)
              const int nval = FBW == 128 ? NBOX : min(NBOX, (fa.K - kc0) / BC);
              mbar_arrive_expect_tx(fb, nval * BOXB);
#pragma unroll
              for (int h = 0; h < NBOX; ++h) {
                if (h >= nval) break;
                const int k0 = kc0 + BC * h;
                const int tap = k0 / fa.C, c0 = k0 - tap * fa.C;
                const int tr = tap / fa.S, ts = tap - tr * fa.S;
                tma_load_im2col_4d(stg0 + aslot * Cfg::STG_BYTES + h * BOXB, mA, fb, c0, w0 - fa.S / 2,
                                   h0 - fa.R / 2, n0, static_cast<uint16_t>(ts), static_cast<uint16_t>(tr));
              }
            } else {
              mbar_arrive_expect_tx(fb, Cfg::STG_BYTES);
#pragma unroll
              for (int h = 0; h < Cfg::STG_ROW / 128; ++h)
                tma_load_3d(stg0 + aslot * Cfg::STG_BYTES + h * BOX, mA, fb, aq.c * Cfg::BK + 32 * h,
                            aq.w.tm * 128, 0);
            }
            a_used |= 1u << aslot;
            a_par = (a_par & ~(1u << aslot)) | (aph << aslot);
            adv(aq);
            if (++aslot == NSTG_) {
              aslot = 0;
              aph ^= 1u;
            }
            prog = true;
          }
          if (bq.have && mbar_test_wait(empty_bar(bstage), bph ^ 1u)) {
            const uint32_t fb = full_bar(bstage);
            mbar_arrive_expect_tx(fb, NP * Cfg::B_PLANE);
            const uint32_t sB = sbase + bstage * Cfg::STAGE + NP * Cfg::A_PLANE;
            const int kx = bq.c * Cfg::BK;
            tma_load_3d(sB, mB, fb, kx, bq.w.tn * BN, 0);
            tma_load_3d(sB + Cfg::B_PLANE, mB, fb, kx, bq.w.tn * BN, 1);
            b_used |= 1u << bstage;
            b_par = (b_par & ~(1u << bstage)) | (bph << bstage);
            adv(bq);
            if (++bstage == STAGES) {
              bstage = 0;
              bph ^= 1u;
            }
            prog = true;
          }
          if (prog) {
            idle = 0;
            continue;
          }
          if (*abort_flag) {
            ok = false;
            break;
          }
          if (idle++ == 0) {
            t0 = global_timer_ns();
          } else if ((idle & 255u) == 0 && global_timer_ns() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            atomicOr(err, kErrTimeout);
            ok = false;
            break;
          }
          __nanosleep(32);
        }
        if (!ok) {
          // abort: let every copy this thread started land before shared memory is released
          for (int b = 0; b < NSTG_; ++b)
            if (a_used & (1u << b)) mbar_wait_drain(stg_full_bar(b), (a_par >> b) & 1u);
          for (int b = 0; b < STAGES; ++b)
            if (b_used & (1u << b)) mbar_wait_drain(full_bar(b), (b_par >> b) & 1u);
        }
      }
    } else if (lane == 0) {
      const int hints = sc.l2_hints();
      const uint64_t polA = l2_policy_evict_last();
      uint32_t stage = 0, phase = 0;
      uint32_t last_phase[STAGES];
      bool issued[STAGES];
      for (int s = 0; s < STAGES; ++s) issued[s] = false, last_phase[s] = 0;
      bool ok = true;
      int last_prob = -1;
      Work wn = nunits > 0 ? sc.work(min(static_cast<int>(blockIdx.x), nunits - 1)) : Work{};
      int qk = 0, u_pre = 0;   // DYN: units published; the next unit, taken one unit ahead
      Work wd{};               // DYN: the work entry of the unit to publish next
      auto publish = [&](int u) -> bool {   // DYN: unit u (or the end) into the queue
        if constexpr (DYN) {
          const int s = qk % QD;
          if (!mbar_wait(qempty_bar(s), ((qk / QD) & 1) ^ 1u, abort_flag, err)) return false;
          q_unit[s] = u < nunits ? u : -1;
          q_work[s] = wd;
          mbar_arrive(qfull_bar(s));
          ++qk;
        }
        return true;
      };
      int u0 = static_cast<int>(blockIdx.x);
      if constexpr (DYN) {
        u0 = atomicAdd(sc.unit_ctr(), 1);
        if (u0 < nunits) wd = sc.work(u0);
      }
      int ready_a = -1, ready_b = -1;   // the last blocks seen ready
      for (int u = u0; ok && (ok = publish(u)) && u < nunits; u = DYN ? u_pre : u + static_cast<int>(gridDim.x)) {
        if constexpr (DYN) u_pre = atomicAdd(sc.unit_ctr(), 1);
        const Work w = DYN ? wd : wn;              // next unit's entry loads early
        if (!DYN && u + static_cast<int>(gridDim.x) < nunits) wn = sc.work(u + gridDim.x);
        if (readyA != nullptr) {
          // this unit's row block of A and column block of B (tiles start
          // inside M and N, so both blocks exist)
          const int ba = w.tm, bb = (w.tn * BN) / kScaleBlock;
          if (ba != ready_a || bb != ready_b) {
            if (!wait_flag_bit(readyA + ba, kBlockReady, abort_flag, err) ||
                !wait_flag_bit(readyB + bb, kBlockReady, abort_flag, err)) {
              ok = false;
              break;
            }
            fence_proxy_async_global();
            ready_a = ba, ready_b = bb;
          }
        }
        const CUtensorMap* mA = sc.mapA(w.prob);
        const CUtensorMap* mB = sc.mapB(w.prob);
        if (w.prob != last_prob) {
          if (!FUSED) tma_prefetch_desc(mA);
          tma_prefetch_desc(mB);
          last_prob = w.prob;
        }
        // CONVA: image, row and column of the tile's first pixel; channel, tap
        // column and tap row of the next box, stepped box by box (no
        // divisions on the issuing thread's path: they were its bottleneck)
        int cn0 = 0, ch0 = 0, cw0 = 0, bc = 0, bs = 0, br = 0;
        if constexpr (CONVA != 0) {
          const FusedA fa = sc.srcA(0);
          const int hw = fa.H * fa.W;
          const int p0 = w.tm * 128;
          cn0 = p0 / hw;
          const int rem = p0 - cn0 * hw;
          ch0 = rem / fa.W;
          cw0 = rem - ch0 * fa.W;
          const int k0 = w.c0 * Cfg::BK;
          const int tap = k0 / fa.C;
          bc = k0 - tap * fa.C;
          br = tap / fa.S;
          bs = tap - br * fa.S;
        }
        for (int c = w.c0; c < w.c1; ++c) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t fb = full_bar(stage);
          const uint32_t sA = sbase + stage * Cfg::STAGE;
          const int kx = c * Cfg::BK;
          if constexpr (CONVA == 64) {
            // one box a plane: 128 output pixels from the tile's first
            // (output (h, w) starts at input (h - (R-1)/2, w - (S-1)/2); tap
            // (r, s) adds its offsets) times the chunk's 64 channels, all of
            // one tap (C % 64 == 0, so K has no partial chunk)
            const FusedA fa = sc.srcA(0);
            mbar_arrive_expect_tx(fb, Cfg::STAGE);
#pragma unroll
            for (int z = 0; z < NP; ++z)
              tma_load_im2col_4d(sA + z * Cfg::A_PLANE, mA, fb, bc, cw0 - fa.S / 2, ch0 - fa.R / 2,
                                 cn0 + z * fa.N, static_cast<uint16_t>(bs), static_cast<uint16_t>(br));
            if ((bc += 64) == fa.C) {
              bc = 0;
              if (++bs == fa.S) bs = 0, ++br;
            }
#pragma unroll
            for (int z = 0; z < NP; ++z)
              tma_load_3d(sA + NP * Cfg::A_PLANE + z * Cfg::B_PLANE, mB, fb, kx, w.tn * BN, z);
          } else if constexpr (CB32) {
            // boxes: the same pixels times one 16-channel group of one tap,
            // hi and lo interleaved (channel 2c of the interleaved image),
            // one per k-step
            const FusedA fa = sc.srcA(0);
            const int nval = min(Cfg::KSTEPS / GSTEPS, (fa.K - kx) / 16);
            mbar_arrive_expect_tx(fb, nval * IBOX + NP * Cfg::B_PLANE);
            for (int h = 0; h < Cfg::KSTEPS / GSTEPS; ++h) {
              if (h >= nval) break;
              tma_load_im2col_4d(sA + h * IBOX, mA, fb, 2 * bc, cw0 - fa.S / 2, ch0 - fa.R / 2, cn0,
                                 static_cast<uint16_t>(bs), static_cast<uint16_t>(br));
              if ((bc += 16) == fa.C) {
                bc = 0;
                if (++bs == fa.S) bs = 0, ++br;
              }
            }
#pragma unroll
            for (int z = 0; z < NP; ++z)
              tma_load_3d(sA + NP * Cfg::A_PLANE + z * Cfg::B_PLANE, mB, fb, kx, w.tn * BN, z);
          } else if constexpr (CB16) {
            // boxes: the same pixels times 16 channels of one tap, one per k-step
            const FusedA fa = sc.srcA(0);
            const int nval = min(Cfg::KSTEPS, (fa.K - kx) / 16);
            mbar_arrive_expect_tx(fb, NP * (nval * CBOX + Cfg::B_PLANE));
            for (int h = 0; h < Cfg::KSTEPS; ++h) {
              if (h >= nval) break;
#pragma unroll
              for (int z = 0; z < NP; ++z)
                tma_load_im2col_4d(sA + z * Cfg::A_PLANE + h * CBOX, mA, fb, bc, cw0 - fa.S / 2,
                                   ch0 - fa.R / 2, cn0 + z * fa.N, static_cast<uint16_t>(bs),
                                   static_cast<uint16_t>(br));
              if ((bc += 16) == fa.C) {
                bc = 0;
                if (++bs == fa.S) bs = 0, ++br;
              }
            }
#pragma unroll
            for (int z = 0; z < NP; ++z)
              tma_load_3d(sA + NP * Cfg::A_PLANE + z * Cfg::B_PLANE, mB, fb, kx, w.tn * BN, z);
          } else if (hints) {
            mbar_arrive_expect_tx(fb, FUSED ? NP * Cfg::B_PLANE : Cfg::STAGE);
            if (!FUSED) {
#pragma unroll
              for (int z = 0; z < NP; ++z)
                tma_load_3d_hint(sA + z * Cfg::A_PLANE, mA, fb, kx, w.tm * Cfg::BM, z, polA);
            }
#pragma unroll
            for (int z = 0; z < NP; ++z)
              tma_load_3d(sA + NP * Cfg::A_PLANE + z * Cfg::B_PLANE, mB, fb, kx, w.tn * BN, z);
          } else {
            mbar_arrive_expect_tx(fb, FUSED ? NP * Cfg::B_PLANE : Cfg::STAGE);
            if (!FUSED) {
#pragma unroll
              for (int z = 0; z < NP; ++z) tma_load_3d(sA + z * Cfg::A_PLANE, mA, fb, kx, w.tm * Cfg::BM, z);
            }
#pragma unroll
            for (int z = 0; z < NP; ++z)
              tma_load_3d(sA + NP * Cfg::A_PLANE + z * Cfg::B_PLANE, mB, fb, kx, w.tn * BN, z);
          }
          issued[stage] = true;
          last_phase[stage] = phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        // DYN: the next unit's entry, loaded while this unit's last stages fill
        if constexpr (DYN) {
          if (u_pre < nunits) wd = sc.work(u_pre);
        }
      }
      if (!ok) {
        // abort: let every copy this thread started land before shared memory is released
        for (int s = 0; s < STAGES; ++s)
          if (issued[s]) mbar_wait_drain(full_bar(s), last_phase[s]);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f32acc(TF32, 128, BN);
      int convK = 0;   // 16-channel boxes: K of the patch matrix
      if constexpr (CGRP) convK = sc.srcA(0).K;
      uint32_t stage = 0, phase = 0, ab = 0, aphase = 0;
      bool ok = true;
      bool any = false;
      Work wn = nunits > 0 ? sc.work(min(static_cast<int>(blockIdx.x), nunits - 1)) : Work{};
      int qk = 0;   // DYN: units read from the queue
      Work wq{};    // DYN: the work entry read with the unit
      auto take = [&]() -> int {   // DYN: the next unit from the queue (-1: the end, or an abort)
        int u = -1;
        if constexpr (DYN) {
          const int s = qk % QD;
          if (!mbar_wait(qfull_bar(s), (qk / QD) & 1, abort_flag, err)) {
            ok = false;
            return -1;
          }
          u = q_unit[s];
          wq = q_work[s];
          mbar_arrive(qempty_bar(s));
          ++qk;
        }
        return u;
      };
      for (int u = DYN ? take() : static_cast<int>(blockIdx.x); ok && u >= 0 && u < nunits;
           u = DYN ? take() : u + static_cast<int>(gridDim.x)) {
        const Work w = DYN ? wq : wn;
        if (!DYN && u + static_cast<int>(gridDim.x) < nunits) wn = sc.work(u + gridDim.x);
        for (int cb = w.c0; ok && cb < w.c1; cb += kb) {
          const int ce = min(cb + kb, w.c1);
          if (!mbar_wait(acce_bar(ab), aphase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + ab * Cfg::ACC_COLS;
          for (int c = cb; c < ce; ++c) {
            if (!mbar_wait(full_bar(stage), phase, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sAhi = sbase + stage * Cfg::STAGE;
            const uint32_t sAlo = sAhi + Cfg::A_PLANE;
            const uint32_t sBhi = sAhi + NP * Cfg::A_PLANE;
            const uint32_t sBlo = sBhi + Cfg::B_PLANE;
            // 16-channel groups: k-steps of this chunk inside K (its boxes that were loaded)
            const int kv = CGRP ? min(Cfg::KSTEPS, (convK - c * Cfg::BK) / KELEM) : Cfg::KSTEPS;
#pragma unroll
            for (int kk = 0; kk < Cfg::KSTEPS; ++kk) {
              if (CGRP && kk >= kv) break;
              const uint32_t off = kk * 32;   // 32 bytes = one MMA's K slice
              // interleaved box of this k-step and the hi part's offset in its rows
              const uint32_t ib = sAhi + (kk / GSTEPS) * IBOX + (kk % GSTEPS) * 32;
              const uint64_t dAhi = CB32   ? (TF32 ? sdesc_k_sw128(ib) : sdesc_k_sw64(ib))
                                    : CB16 ? sdesc_k_sw32(sAhi + kk * CBOX)
                                           : sdesc_k<Cfg::SW>(sAhi + off);
              const uint64_t dAlo = CB32   ? (TF32 ? sdesc_k_sw128(ib + 64) : sdesc_k_sw64(ib + 32))
                                    : CB16 ? sdesc_k_sw32(sAlo + kk * CBOX)
                                           : sdesc_k<Cfg::SW>(sAlo + off);
              const uint64_t dBhi = sdesc_k<Cfg::SW>(sBhi + off);
              const uint64_t dBlo = sdesc_k<Cfg::SW>(sBlo + off);
              const uint32_t acc = (c > cb || kk > 0) ? 1u : 0u;
              if constexpr (NP == 3) {
                // planes 0, 1, 2 = hi, mid, lo; the six products whose
                // plane indices sum to at most 2: the five smaller ones into
                // the second accumulator (smallest first), hi*hi into the first
                const uint32_t d2 = d + BN;
                const uint64_t dAl2 = CB16 ? sdesc_k_sw32(sAhi + 2 * Cfg::A_PLANE + kk * CBOX)
                                            : sdesc_k<Cfg::SW>(sAhi + 2 * Cfg::A_PLANE + off);
                const uint64_t dBl2 = sdesc_k<Cfg::SW>(sBhi + 2 * Cfg::B_PLANE + off);
                umma_bf16(d2, dAl2, dBhi, idesc, acc);
                umma_bf16(d2, dAlo, dBlo, idesc, 1u);
                umma_bf16(d2, dAhi, dBl2, idesc, 1u);
                umma_bf16(d2, dAlo, dBhi, idesc, 1u);
                umma_bf16(d2, dAhi, dBlo, idesc, 1u);
                umma_bf16(d, dAhi, dBhi, idesc, acc);
              } else if (TF32) {
                umma_tf32(d, dAlo, dBhi, idesc, acc);
                umma_tf32(d, dAhi, dBlo, idesc, 1u);
                umma_tf32(d, dAhi, dBhi, idesc, 1u);
              } else {
                umma_bf16(d, dAlo, dBhi, idesc, acc);
                umma_bf16(d, dAhi, dBlo, idesc, 1u);
                umma_bf16(d, dAhi, dBhi, idesc, 1u);
              }
            }
            any = true;
            umma_commit(empty_bar(stage));
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          umma_commit(accf_bar(ab));
          if (++ab == NACC) {
            ab = 0;
            aphase ^= 1u;
          }
        }
      }
      if (any) {
        // every MMA this thread issued has finished before TMEM is released
        umma_commit(drain_bar);
        mbar_wait_drain(drain_bar, 0);
      }
    }
    __syncwarp();
  } else if (warp < 2 + 4 * Cfg::EPI_WG) {
    // ------------------------------------------------------------ epilogue
    constexpr int EC = Cfg::EPI_COLS;
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int half = (warp - 2) >> 2;       // column group of this warpgroup
    uint32_t ab = 0, aphase = 0;
    bool ok = true;
    Work wn = nunits > 0 ? sc.work(min(static_cast<int>(blockIdx.x), nunits - 1)) : Work{};
    int qk = 0;   // DYN: units read from the queue
    Work wq{};    // DYN: the work entry read with the unit
    auto take = [&]() -> int {   // DYN, whole warp: the next unit from the queue (-1: end or abort)
      int u = -1;
      if constexpr (DYN) {
        const int s = qk % QD;
        const bool waited = mbar_wait(qfull_bar(s), (qk / QD) & 1, abort_flag, err);
        if (!__all_sync(0xffffffffu, waited)) {
          ok = false;
          return -1;
        }
        u = q_unit[s];
        wq = q_work[s];
        __syncwarp();
        if (lane == 0) mbar_arrive(qempty_bar(s));
        ++qk;
      }
      return u;
    };
    for (int u = DYN ? take() : static_cast<int>(blockIdx.x); ok && u >= 0 && u < nunits;
         u = DYN ? take() : u + static_cast<int>(gridDim.x)) {
      const Work w = DYN ? wq : wn;
      if (!DYN && u + static_cast<int>(gridDim.x) < nunits) wn = sc.work(u + gridDim.x);
      // The unit's epilogue values and block exponents are loaded before its
      // accumulator is waited for (the pack has completed: every role passed
      // griddep_wait), and L2 is warmed with the part of C this thread will
      // read (beta != 0): their latency overlaps the unit's main loop, which
      // short-K tiles (grouped problems) do not cover otherwise.
      const EpiView v = sc.epi(w.prob);
      const int col0 = w.tn * BN + half * EC;
      const int e = block_exponent(v.amaxA[w.tm * v.amaxA_stride]) +
                    block_exponent(v.amaxB[col0 / kScaleBlock]);
      {
        const int prow = w.tm * 128 + q * 32 + lane;
        if (v.beta != 0.0f && v.split_k == 1 && prow < v.M && col0 < v.N) {
          const float* rp = v.C + static_cast<int64_t>(prow) * v.ldc + col0;
          const int ncols = min(EC, v.N - col0);
#pragma unroll
          for (int j = 0; j < EC; j += 32)
            if (j < ncols) prefetch_l2(rp + j);
          prefetch_l2(rp + ncols - 1);
        }
      }
      float S[EC];
      // compensated epilogue: rounding errors of the fold additions
      constexpr bool COMP = Sched::kCompensated;
      float E[COMP ? EC : 1];
      int blk = 0;
      for (int cb = w.c0; cb < w.c1; cb += kb, ++blk) {
        // the whole warp must agree before the warp-collective TMEM loads
        const bool waited = mbar_wait(accf_bar(ab), aphase, abort_flag, err);
        if (!__all_sync(0xffffffffu, waited)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr =
            tmem_base + (static_cast<uint32_t>(q * 32) << 16) + ab * Cfg::ACC_COLS + half * EC;
        if constexpr (COMP) {
          // 32 columns a thread (two epilogue warpgroups)
          static_assert(EC == 32, "compensated epilogue: 32 columns a thread");
          uint32_t r[32];
          tmem_ld_32x32b_x32(taddr, r);
          tmem_wait_ld();
          if (blk == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) S[i] = __uint_as_float(r[i]), E[i] = 0.0f;
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) two_sum_acc(S[i], E[i], __uint_as_float(r[i]));
          }
          if constexpr (NP == 3) {
            tmem_ld_32x32b_x32(taddr + BN, r);   // the five smaller products
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) two_sum_acc(S[i], E[i], __uint_as_float(r[i]));
          }
        } else {
#pragma unroll
        for (int j = 0; j < EC / 32; ++j) {
          uint32_t r[32];
          tmem_ld_32x32b_x32(taddr + j * 32, r);
          tmem_wait_ld();
          if (blk == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) S[j * 32 + i] = __uint_as_float(r[i]);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) S[j * 32 + i] += __uint_as_float(r[i]);
          }
          if constexpr (NP == 3) {
            // the five smaller products' accumulator, BN columns further on
            tmem_ld_32x32b_x32(taddr + BN + j * 32, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) S[j * 32 + i] += __uint_as_float(r[i]);
          }
        }
        }
        tc_fence_before();
        mbar_arrive(acce_bar(ab));
        if (++ab == NACC) {
          ab = 0;
          aphase ^= 1u;
        }
      }
      if (!ok) break;
      if constexpr (COMP) {
        // the sum's rounding errors added back once
#pragma unroll
        for (int i = 0; i < EC; ++i) S[i] = __fadd_rn(S[i], E[i]);
      }
      if (blk == 0 || v.alpha == 0.0f) {
        // K == 0 or alpha == 0 (grouped problems only): C = beta * C; the
        // planes of such a problem are not packed, so their TMEM sum is unused
#pragma unroll
        for (int i = 0; i < EC; ++i) S[i] = 0.0f;
      }

      epilogue_store<EC, Cfg::EPI_PITCH>(S, v, e, w.ks, w.tm * 128 + q * 32, col0, lane,
                                         epi_buf + (warp - 2) * 32 * Cfg::EPI_PITCH);
    }
  } else if constexpr (FUSED) {
    // ------------------------------------------------------------ A (fused)
    // FP32 chunks of A (128 rows x BK) are staged in a ring of STG_STAGES
    // buffers, that many chunks ahead: by the producer thread with one TMA
    // load per 128-byte-wide box when A's rows are 16-byte aligned, else by
    // the split threads with 4-byte cp.async copies; both leave the
    // SWIZZLE_128B layout, row r's 16-byte unit u at u ^ (r % 8).  Split
    // thread t splits rows t, t + SPLIT_THREADS, ... of a staged chunk into
    // the stage's hi/lo planes (conflict-free shared accesses on both
    // sides) and fences its writes for the async proxy; then one lane a
    // warp arrives on the stage's full barrier and frees the staging
    // buffer.  The split warps never wait for one another.  Every wait is
    // bounded.
    constexpr int UPR = Cfg::STG_ROW / 16;            // 16-byte units per staged row
    constexpr int BOX = 128 * 128;                    // bytes of one 128-byte-wide staging box
    const int ct = threadIdx.x - Cfg::SPLIT0;
    const uint32_t stg0 = sbase + Cfg::OFF_STG;
    const uint8_t* stg_gen = smem + Cfg::OFF_STG;
    const bool tma = sc.srcA(0).vec;                  // uniform: the producer stages A by TMA

    // split cursor (sc_) and, when the split threads stage A themselves with
    // cp.async, fill cursor (fc) over this CTA's (unit, chunk)s
    struct Cursor {
      int u, c;
      Work w;
      bool have;
    };
    auto first = [&](Cursor& q, int u0) {
      q.have = false;
      for (q.u = u0; q.u < nunits; q.u += gridDim.x) {
        q.w = sc.work(q.u);
        if (q.w.c0 < q.w.c1) {
          q.have = true;
          q.c = q.w.c0;
          break;
        }
      }
    };
    auto advance = [&](Cursor& q) {
      if (++q.c >= q.w.c1) first(q, q.u + gridDim.x);
    };
    Cursor sc_{}, fc{};
    first(sc_, blockIdx.x);
    fc = sc_;
    // cp.async staging of the fill cursor's chunk into buffer b (4-byte
    // copies: A's rows are not 16-byte aligned), same layout as the TMA boxes
    auto fill = [&](int b) {
      const FusedA src = sc.srcA(fc.w.prob);
      const int64_t kbase = static_cast<int64_t>(fc.c) * Cfg::BK;
      if (src.conv) {
        // Patch-matrix gather of an R x S convolution: column k = (tap, c),
        // tap = S r + s; row = output pixel (n, h, w) reads the input pixel
        // (n, h + r - (R-1)/2, w + s - (S-1)/2), zero outside.  C % 4 == 0, so a 16-byte
        // unit is four channels of one tap.  With SPLIT_THREADS a multiple of
        // UPR, this thread's unit j is fixed and its rows step by RS pixels.
        static_assert(Cfg::SPLIT_THREADS % UPR == 0, "unit mapping");
        constexpr int RS = Cfg::SPLIT_THREADS / UPR;
        const int j = ct % UPR;
        const int64_t k = kbase + 4 * j;
        const bool kin = k < src.K;
        const int tap = kin ? static_cast<int>(k / src.C) : 0;
        const int c = static_cast<int>(k - static_cast<int64_t>(tap) * src.C);
        const int dr = tap / src.S - src.R / 2, ds = tap % src.S - src.S / 2;
        const int hw = src.H * src.W;
        int64_t pix = static_cast<int64_t>(fc.w.tm) * 128 + ct / UPR;
        int n = static_cast<int>(pix / hw);
        int rem = static_cast<int>(pix - static_cast<int64_t>(n) * hw);
        int h = rem / src.W, w = rem - h * src.W;
        for (int r = ct / UPR; r < 128; r += RS) {
          const uint32_t dst = stg0 + b * Cfg::STG_BYTES + (j >> 3) * BOX + r * 128 +
                               (((j & 7) ^ (r & 7)) << 4);
          const int hh = h + dr, ww = w + ds;
          const bool in = kin && pix < src.M && hh >= 0 && hh < src.H && ww >= 0 && ww < src.W;
          const float* p = in ? src.A + ((static_cast<int64_t>(n) * src.H + hh) * src.W + ww) * src.C + c
                              : src.A;
          cp_async_16(dst, p, in ? 16u : 0u);
          // next row: RS pixels further
          pix += RS;
          w += RS;
          while (w >= src.W) {
            w -= src.W;
            if (++h == src.H) h = 0, ++n;
          }
        }
        cp_async_mbar_arrive(stg_full_bar(b));
        advance(fc);
        return;
      }
      for (int i = ct; i < 128 * UPR; i += Cfg::SPLIT_THREADS) {
        const int r = i / UPR, j = i % UPR;
        const uint32_t dst = stg0 + b * Cfg::STG_BYTES + (j >> 3) * BOX + r * 128 +
                             (((j & 7) ^ (r & 7)) << 4);
        const int64_t row = static_cast<int64_t>(fc.w.tm) * 128 + r;
        const int64_t k = kbase + 4 * j;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool in = row < src.M && k + e < src.K;
          cp_async_4(dst + 4 * e, in ? src.A + row * src.lda + k + e : src.A, in ? 4u : 0u);
        }
      }
      cp_async_mbar_arrive(stg_full_bar(b));
      advance(fc);
    };

    if (!tma) {
#pragma unroll
      for (int b = 0; b < NSTG; ++b)
        if (fc.have) fill(b);
    }
    uint32_t stage = 0, phase = 0, slot = 0, sphase = 0;
    unsigned amax = 0;
    int last_prob = -1, last_tm = -1;
    int kdata = 0;                    // 16-channel boxes: K (boxes past it are not loaded)
    while (sc_.have) {
      if (sc_.w.prob != last_prob || sc_.w.tm != last_tm) {
        const FusedA sa = sc.srcA(sc_.w.prob);
        amax = sa.amaxA[sc_.w.tm * sa.amax_stride];
        last_prob = sc_.w.prob;
        last_tm = sc_.w.tm;
        kdata = sa.K;
      }
      // lane 0 waits for the warp; __syncwarp orders its acquire before the
      // other lanes' accesses
      int w_ok = 1;
      if (lane == 0)
        w_ok = mbar_wait(stg_full_bar(slot), sphase, abort_flag, err) &&
               mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, err);
      if (!__shfl_sync(0xffffffffu, w_ok, 0)) break;
      const float sf = pow2f(-block_exponent(amax));
      const bool finite = amax < 0x7F800000u;
      uint8_t* hi = smem + stage * Cfg::STAGE;
      const uint8_t* sbuf = stg_gen + slot * Cfg::STG_BYTES;
      // one branch for the whole chunk, so that the eight groups of a row
      // form one straight-line block the compiler can interleave
      constexpr int NT = Cfg::SPLIT_THREADS;
      uint8_t* lo = hi + Cfg::A_PLANE;
      if constexpr (FBW == 64) {
        const int rest = kdata - sc_.c * Cfg::BK;             // elements of the chunk that were loaded
        const int valid = rest >= Cfg::BK ? UPR : rest / 4;   // 16-byte units per row
        if (finite) fused_split_rows<TF32, true, NT, 64, true>(sbuf, hi, lo, ct, sf, valid);
        else fused_split_rows<TF32, false, NT, 64, true>(sbuf, hi, lo, ct, sf, valid);
      } else if (finite) {
        fused_split_rows<TF32, true, NT>(sbuf, hi, lo, ct, sf);
      } else {
        fused_split_rows<TF32, false, NT>(sbuf, hi, lo, ct, sf);
      }
      // every lane fences its writes for the async proxy; after __syncwarp
      // lane 0 arrives for the warp (one arrival per warp)
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(full_bar(stage));
        mbar_arrive(stg_empty_bar(slot));
      }
      // cp.async staging: refill this buffer with the chunk STG_STAGES ahead
      // once every split warp has read it
      if (!tma && fc.have) {
        int e_ok = 1;
        if (lane == 0) e_ok = mbar_wait(stg_empty_bar(slot), sphase, abort_flag, err);
        if (!__shfl_sync(0xffffffffu, e_ok, 0)) break;
        fill(slot);
      }
      advance(sc_);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
      if (++slot == NSTG) {
        slot = 0;
        sphase ^= 1u;
      }
    }
    if (!tma) cp_async_wait_all();   // no copy may land after the shared memory is released
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
  // every role of this CTA is past its last read of the block maxima and
  // the unit counter (the barrier above)
  clear_execution_state(sc.state(), sc.state_words());
}

template <int BN, bool TF32, int NP>
__global__ void __launch_bounds__(TcCfg<BN, TF32, false, NP>::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs a) {
  SingleSched sc{&tmA, &tmB, &a};
  tc_gemm_body<BN, TF32, SingleSched, false, NP>(sc);
}

// Compensated epilogue (SingleSchedComp): packed operands, every fold added
// with its rounding error kept; instantiated for 128 x 64 tiles drained by
// two epilogue warpgroups, 32 columns a thread (a 128-wide tile would need
// 64 sums and 64 errors a thread at the 168 registers a thread that 320
// threads leave, and spilled).
template <int BN, bool TF32, int NP>
__global__ void __launch_bounds__(TcCfg<BN, TF32, false, NP, 2>::THREADS, 1)
    tc_gemm_comp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const TcArgs a) {
  SingleSchedComp sc{{&tmA, &tmB, &a}};
  tc_gemm_body<BN, TF32, SingleSchedComp, false, NP>(sc);
}

// Packed convolution: A's planes loaded as im2col boxes (CB channels) of
// the split image.
template <int BN, bool TF32, int NP, int CB>
__global__ void __launch_bounds__(TcCfg<BN, TF32, false, NP>::THREADS, 1)
    tc_conv_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs a) {
  SingleSched sc{&tmA, &tmB, &a};
  tc_gemm_body<BN, TF32, SingleSched, false, NP, 128, CB>(sc);
}

// Packed convolution with few output features (at most 32): 128 x 32 tiles,
// two-deep ring, TWO CTAs a SM.  The 16-feature layer is latency-bound (a
// tile is a chain of dependent steps on a few threads, about one tile of
// loads in flight a CTA, 18 % tensor and 11 % DRAM activity with 64-wide
// tiles); a narrower tile needs 100 KB of shared memory and 128 TMEM
// columns, so that a SM holds two CTAs and twice the units in flight, and
// its MMAs and B loads carry no empty columns.
template <bool TF32, int NP, int CB>
__global__ void __launch_bounds__(TcCfg<32, TF32, false, NP>::THREADS, 2)
    tc_conv_narrow_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                          const TcArgs a) {
  SingleSched sc{&tmA, &tmB, &a};
  tc_gemm_body<32, TF32, SingleSched, false, NP, 128, CB>(sc);
}

template <int BN, bool TF32, int NP>
__global__ void __launch_bounds__(TcCfg<BN, TF32, false, NP, 1>::THREADS, 1)
    tc_grouped_kernel(const GroupedArgs a) {
  GroupedSched sc{&a};
  tc_gemm_body<BN, TF32, GroupedSched, false, NP>(sc);
}

// Fused variant: tmA maps A itself (FP32, 128-byte-wide boxes of 128 rows)
// when its rows are 16-byte aligned, or a convolution's image for im2col
// loads (FBW = 64: boxes of 16 channels); otherwise it is unused.
template <int BN, bool TF32, int FBW>
__global__ void __launch_bounds__(TcCfg<BN, TF32, true>::THREADS, 1)
    tc_gemm_fused_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const TcArgs a) {
  SingleSched sc{&tmA, &tmB, &a};
  tc_gemm_body<BN, TF32, SingleSched, true, 2, FBW>(sc);
}

// Split-K fix-up: C = sum_s partial[s] + beta * C, where each partial already
// holds alpha * (its share of A*B); partials are summed in increasing s (a
// fixed order, so results do not depend on timing).  A thread covers four
// consecutive columns of one row (rows by blockIdx.y, strided; columns by
// blockIdx.x), with float4 loads of the partials when N % 4 == 0 and float4
// accesses of C when its rows are 16-byte aligned as well: no index
// division, every warp access contiguous.
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ partial,
                                     float beta, float* __restrict__ C, int64_t ldc) {
  griddep_wait();   // launched as a dependent of the gemm kernel
  const int64_t plane = static_cast<int64_t>(M) * N;
  const bool vp = (N & 3) == 0;
  const bool vc = vp && (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
  const int c = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (c >= N) return;
  for (int r = blockIdx.y; r < M; r += gridDim.y) {
    const float* pp = partial + static_cast<int64_t>(r) * N + c;
    float* cp = C + static_cast<int64_t>(r) * ldc + c;
    if (vp) {
      float4 s = __ldg(reinterpret_cast<const float4*>(pp));
      for (int k = 1; k < splits; ++k) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(pp + k * plane));
        s.x += t.x, s.y += t.y, s.z += t.z, s.w += t.w;
      }
      if (vc) {
        float4* c4 = reinterpret_cast<float4*>(cp);
        if (beta != 0.0f) {
          const float4 o = *c4;
          s.x = s.x + beta * o.x, s.y = s.y + beta * o.y, s.z = s.z + beta * o.z, s.w = s.w + beta * o.w;
        }
        *c4 = s;
      } else {
        const float v[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) cp[j] = beta != 0.0f ? v[j] + beta * cp[j] : v[j];
      }
    } else {
      const int n = min(4, N - c);
      for (int j = 0; j < n; ++j) {
        float s = pp[j];
        for (int k = 1; k < splits; ++k) s += pp[k * plane + j];
        cp[j] = beta != 0.0f ? s + beta * cp[j] : s;
      }
    }
  }
}

// Launch with programmatic stream serialization: the kernel may begin (its
// prologue, up to griddep_wait) while the previous kernel of the stream
// finishes.
template <typename... Params, typename... Args>
static cudaError_t launch_dependent(void (*kernel)(Params...), int grid, int threads, int smem,
                                    cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

int tc_smem_bytes(int bn, Prec prec, bool fused) {
  if (fused) {
    if (prec == Prec::TF32) return bn == 64 ? TcCfg<64, true, true>::SMEM : TcCfg<128, true, true>::SMEM;
    return bn == 64 ? TcCfg<64, false, true>::SMEM : TcCfg<128, false, true>::SMEM;
  }
  if (prec == Prec::TF32) return bn == 64 ? TcCfg<64, true>::SMEM : TcCfg<128, true>::SMEM;
  if (prec == Prec::BF16X6)
    return bn == 64 ? TcCfg<64, false, false, 3>::SMEM : TcCfg<128, false, false, 3>::SMEM;
  return bn == 64 ? TcCfg<64, false>::SMEM : TcCfg<128, false>::SMEM;
}

int tc_chunk_bytes(int bn) {
  (void)bn;   // every variant steps in 128-byte chunks (see TcCfg)
  return 128;
}

// The dynamic shared memory limit of every kernel variant is raised once per
// device and thread, outside any stream capture: plans call tc_prepare when
// they are created, launches call it again (a no-op after the first time).
template <int BN, bool TF32, bool FUSED, int NP = 2>
static cudaError_t prepare_variant() {
  using Cfg = TcCfg<BN, TF32, FUSED, NP>;
  static thread_local int configured_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device != dev) {
    if constexpr (FUSED) {
      e = cudaFuncSetAttribute(tc_gemm_fused_kernel<BN, TF32, 128>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_gemm_fused_kernel<BN, TF32, 64>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    } else {
      e = cudaFuncSetAttribute(tc_gemm_kernel<BN, TF32, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               Cfg::SMEM);
      if constexpr (BN == 64) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(tc_gemm_comp_kernel<BN, TF32, NP>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   TcCfg<BN, TF32, false, NP, 2>::SMEM);
      }
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_grouped_kernel<BN, TF32, NP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcCfg<BN, TF32, false, NP, 1>::SMEM);
      if constexpr (!TF32) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(tc_conv_kernel<BN, false, NP, 16>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(tc_conv_kernel<BN, false, NP, 64>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
      }
      if constexpr (NP == 2) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(tc_conv_kernel<BN, TF32, NP, 32>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
      }
    }
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  return cudaSuccess;
}

template <bool FUSED>
static cudaError_t prepare_fused(int bn, Prec prec) {
  if (prec == Prec::TF32) {
    if (bn == 64) return prepare_variant<64, true, FUSED>();
    if (bn == 128) return prepare_variant<128, true, FUSED>();
  } else if (prec == Prec::BF16X6) {
    if (FUSED) return cudaErrorInvalidValue;   // the fused kernel splits A in two
    if (bn == 64) return prepare_variant<64, false, false, 3>();
    if (bn == 128) return prepare_variant<128, false, false, 3>();
  } else {
    if (bn == 64) return prepare_variant<64, false, FUSED>();
    if (bn == 128) return prepare_variant<128, false, FUSED>();
  }
  return cudaErrorInvalidValue;
}

// The narrow convolution kernels (tile width 32, two CTAs a SM).
template <bool TF32, int NP, int CB>
static cudaError_t prepare_narrow_one() {
  return cudaFuncSetAttribute(tc_conv_narrow_kernel<TF32, NP, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<32, TF32, false, NP>::SMEM);
}

// (every precision's variants at once: the per-thread flag covers them all)
static cudaError_t prepare_narrow(Prec) {
  static thread_local int configured_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device == dev) return cudaSuccess;
  e = prepare_narrow_one<true, 2, 32>();
  if (e == cudaSuccess) e = prepare_narrow_one<false, 3, 16>();
  if (e == cudaSuccess) e = prepare_narrow_one<false, 3, 64>();
  if (e == cudaSuccess) e = prepare_narrow_one<false, 2, 32>();
  if (e == cudaSuccess) e = prepare_narrow_one<false, 2, 64>();
  if (e == cudaSuccess) configured_device = dev;
  return e;
}

cudaError_t tc_prepare(int bn, Prec prec, bool fused) {
  if (bn == 32) return fused ? cudaErrorInvalidValue : prepare_narrow(prec);
  return fused ? prepare_fused<true>(bn, prec) : prepare_fused<false>(bn, prec);
}

int tc_narrow_ctas_per_sm(Prec prec) {
  // (the system reserves 1 KB of shared memory a CTA; 228 KB a SM)
  const int smem = prec == Prec::TF32 ? TcCfg<32, true, false, 2>::SMEM
                   : prec == Prec::BF16X6 ? TcCfg<32, false, false, 3>::SMEM
                                          : TcCfg<32, false, false, 2>::SMEM;
  return 2 * (smem + 1024) <= 233472 ? 2 : 1;
}

static cudaError_t launch_narrow(int grid, Prec prec, const CUtensorMap& tmA, const CUtensorMap& tmB,
                                 const TcArgs& a, cudaStream_t s) {
  if (!a.conv) return cudaErrorInvalidValue;   // a convolution tile only
  cudaError_t e = prepare_narrow(prec);
  if (e != cudaSuccess) return e;
  if (prec == Prec::TF32) {
    if (a.conv_box_c != 32) return cudaErrorInvalidValue;
    using Cfg = TcCfg<32, true, false, 2>;
    e = launch_dependent(tc_conv_narrow_kernel<true, 2, 32>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
  } else if (prec == Prec::BF16X6) {
    using Cfg = TcCfg<32, false, false, 3>;
    if (a.conv_box_c == 64)
      e = launch_dependent(tc_conv_narrow_kernel<false, 3, 64>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
    else if (a.conv_box_c == 16)
      e = launch_dependent(tc_conv_narrow_kernel<false, 3, 16>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
    else
      return cudaErrorInvalidValue;
  } else {
    using Cfg = TcCfg<32, false, false, 2>;
    if (a.conv_box_c == 64)
      e = launch_dependent(tc_conv_narrow_kernel<false, 2, 64>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
    else if (a.conv_box_c == 32)
      e = launch_dependent(tc_conv_narrow_kernel<false, 2, 32>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
    else
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int BN, bool TF32, int NP = 2>
static cudaError_t launch_variant(int grid, bool fused, bool comp, const CUtensorMap& tmA,
                                  const CUtensorMap& tmB, const TcArgs& a, cudaStream_t s) {
  if (comp) {
    // compensated epilogue: packed gemm operands, 128 x 64 tiles only
    if constexpr (BN != 64) {
      return cudaErrorInvalidValue;
    } else {
      if (fused || a.conv) return cudaErrorInvalidValue;
      using Cfg = TcCfg<BN, TF32, false, NP, 2>;
      cudaError_t e = prepare_variant<BN, TF32, false, NP>();
      if (e != cudaSuccess) return e;
      e = launch_dependent(tc_gemm_comp_kernel<BN, TF32, NP>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
      if (e != cudaSuccess) return e;
      return cudaGetLastError();
    }
  }
  if (fused) {
    if constexpr (NP != 2) {
      return cudaErrorInvalidValue;
    } else {
      using Cfg = TcCfg<BN, TF32, true>;
      cudaError_t e = prepare_variant<BN, TF32, true>();
      if (e != cudaSuccess) return e;
      if (a.conv && a.vecA && a.conv_box_c == 16)
        e = launch_dependent(tc_gemm_fused_kernel<BN, TF32, 64>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
      else
        e = launch_dependent(tc_gemm_fused_kernel<BN, TF32, 128>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
      if (e != cudaSuccess) return e;
    }
  } else {
    using Cfg = TcCfg<BN, TF32, false, NP>;
    cudaError_t e = prepare_variant<BN, TF32, false, NP>();
    if (e != cudaSuccess) return e;
    if (a.conv) {
      // packed convolution: tmA maps the split image's planes for im2col loads
      if (a.conv_box_c == 32) {
        if constexpr (NP == 2)
          e = launch_dependent(tc_conv_kernel<BN, TF32, NP, 32>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
        else
          return cudaErrorInvalidValue;
      } else if constexpr (TF32) {
        return cudaErrorInvalidValue;   // tf32 planes are always interleaved
      } else if (a.conv_box_c == 64) {
        e = launch_dependent(tc_conv_kernel<BN, false, NP, 64>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
      } else {
        e = launch_dependent(tc_conv_kernel<BN, false, NP, 16>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
      }
    } else {
      e = launch_dependent(tc_gemm_kernel<BN, TF32, NP>, grid, Cfg::THREADS, Cfg::SMEM, s, tmA, tmB, a);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t tc_gemm_launch(const TcLaunch& l, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const TcArgs& a, cudaStream_t s) {
  if (l.cluster == 2) {
    if (l.fused || l.comp || a.conv) return cudaErrorInvalidValue;   // pairs: packed gemm operands only
    return tc_pair_launch(l.bn, l.prec, l.grid, tmA, tmB, a, s);
  }
  if (l.bn == 32) {
    if (l.fused || l.comp) return cudaErrorInvalidValue;   // the narrow tile: packed convolutions only
    return launch_narrow(l.grid, l.prec, tmA, tmB, a, s);
  }
  if (l.prec == Prec::TF32) {
    if (l.bn == 64) return launch_variant<64, true>(l.grid, l.fused, l.comp, tmA, tmB, a, s);
    if (l.bn == 128) return launch_variant<128, true>(l.grid, l.fused, l.comp, tmA, tmB, a, s);
  } else if (l.prec == Prec::BF16X6) {
    if (l.bn == 64) return launch_variant<64, false, 3>(l.grid, l.fused, l.comp, tmA, tmB, a, s);
    if (l.bn == 128) return launch_variant<128, false, 3>(l.grid, l.fused, l.comp, tmA, tmB, a, s);
  } else {
    if (l.bn == 64) return launch_variant<64, false>(l.grid, l.fused, l.comp, tmA, tmB, a, s);
    if (l.bn == 128) return launch_variant<128, false>(l.grid, l.fused, l.comp, tmA, tmB, a, s);
  }
  return cudaErrorInvalidValue;
}

template <int BN, bool TF32, int NP = 2>
static cudaError_t launch_grouped_variant(int grid, const GroupedArgs& a, cudaStream_t s) {
  using Cfg = TcCfg<BN, TF32, false, NP, 1>;
  cudaError_t e = prepare_variant<BN, TF32, false, NP>();
  if (e != cudaSuccess) return e;
  e = launch_dependent(tc_grouped_kernel<BN, TF32, NP>, grid, Cfg::THREADS, Cfg::SMEM, s, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t tc_grouped_launch(int bn, Prec prec, int grid, const GroupedArgs& a, cudaStream_t s) {
  if (prec == Prec::TF32) {
    if (bn == 64) return launch_grouped_variant<64, true>(grid, a, s);
    if (bn == 128) return launch_grouped_variant<128, true>(grid, a, s);
  } else if (prec == Prec::BF16X6) {
    if (bn == 64) return launch_grouped_variant<64, false, 3>(grid, a, s);
    if (bn == 128) return launch_grouped_variant<128, false, 3>(grid, a, s);
  } else {
    if (bn == 64) return launch_grouped_variant<64, false>(grid, a, s);
    if (bn == 128) return launch_grouped_variant<128, false>(grid, a, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t splitk_reduce_launch(int M, int N, int splits, const float* partial, float beta,
                                 float* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // 128 threads cover 512 columns of a row; rows spread over blockIdx.y
  const int gx = (N + 511) / 512;
  const int gy = std::max(1, std::min(M, std::max(1, 8192 / gx)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gx, gy);
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, splitk_reduce_kernel, M, N, splits, partial, beta, C, ldc);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace gb
