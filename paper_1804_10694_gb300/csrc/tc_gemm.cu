// Split-precision tensor-core gemm for sm_103a: C = alpha * A * B + beta * C
// with FP32 semantics, computed as three bf16 (or tf32) tensor-core products
// per k-step, hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory.
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
//     tcgen05.mma into a TMEM accumulator (two buffers, so the epilogue of one
//     accumulation block overlaps the MMAs of the next);
//   * full vs partial tiles: TMA zero-fills the out-of-range part of edge
//     tiles on load, so the main loop never branches; only the epilogue
//     masks rows/columns, and full tiles take a vectorised store path;
//   * accumulation blocks: every kb k-chunks the epilogue warps fold the TMEM
//     partial sum into FP32 registers with round-to-nearest adds, which bounds
//     how many products the tensor core's own accumulation chains together.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = MMA issuer and
// TMEM owner, warps 2..5 = epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"
#include "scale.cuh"

namespace gb {

// Tile and pipeline geometry of one kernel variant.  A k-chunk is one
// swizzle span of every row, 128 bytes.  Instantiated for tile widths 64 and
// 128.  A 256-wide tile (two epilogue warpgroups of 128 columns each, which
// this geometry supports) measured 1.1-1.2 PFLOP/s on GB300 against 1.6 for
// 128, with the 128-byte swizzle (2-deep ring) and with the 64-byte swizzle
// (4-deep ring) alike, so it is not offered.
template <int BN, bool TF32>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int SW = 128;                       // bytes of one row per k-chunk
  static constexpr int A_PLANE = BM * SW;
  static constexpr int B_PLANE = BN * SW;
  static constexpr int STAGE = 2 * A_PLANE + 2 * B_PLANE;
  static constexpr int STAGES = BN == 64 ? 4 : BN == 128 ? 3 : 2;
  static constexpr int BK = SW / (TF32 ? 4 : 2);       // elements per k-chunk
  static constexpr int KSTEPS = SW / 32;               // MMAs (32-byte K slices) per chunk and product
  static constexpr int EPI_WG = BN == 256 ? 2 : 1;     // epilogue warpgroups
  static constexpr int EPI_COLS = BN / EPI_WG;         // columns per epilogue thread
  static constexpr int TMEM_COLS = 2 * BN;             // two accumulator buffers
  static constexpr int EPI_PITCH = 33;                 // floats per staged row (bank-conflict free)
  static constexpr int EPI_BYTES = 4 * EPI_WG * 32 * EPI_PITCH * 4;   // one 32x32 buffer per epilogue warp
  static constexpr int BAR_BYTES = 256;
  static constexpr int SMEM = STAGES * STAGE + EPI_BYTES + BAR_BYTES + 1024;
  static constexpr int THREADS = 64 + 128 * EPI_WG;
  static_assert(SMEM <= 232448, "shared memory budget");
  static_assert(TMEM_COLS <= 512, "tensor memory budget");
};

// One unit of work of a CTA: an output tile (tm, tn) of problem `prob` and
// the range [c0, c1) of 128-byte k-chunks it covers (all of K unless split).
struct Work {
  int prob, tm, tn, ks, c0, c1;
};

// Per-problem values the epilogue needs.
struct EpiView {
  int M, N;
  float* C;
  int64_t ldc;
  float alpha, beta;
  const unsigned* amaxA;
  const unsigned* amaxB;
  float* partial;
  int split_k;
};

__device__ __forceinline__ void raster(int t, int tiles_m, int tiles_n, int group_m, int& tm, int& tn) {
  const int group_tiles = group_m * tiles_n;
  const int g = t / group_tiles;
  const int first_m = g * group_m;
  const int rows_in_group = min(tiles_m - first_m, group_m);
  const int r = t % group_tiles;
  tm = first_m + r % rows_in_group;
  tn = r / rows_in_group;
}

// Scheduling policy of one gemm: units are (split, tile) pairs.
struct SingleSched {
  const CUtensorMap* tmA;
  const CUtensorMap* tmB;
  const TcArgs* a;
  __device__ int units() const { return a->num_units; }
  __device__ int kb() const { return a->kb; }
  __device__ int* err() const { return a->err; }
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
    return v;
  }
};

// Scheduling policy of a grouped launch: units are the tiles of all problems,
// listed problem after problem (problems ordered longest-K first on the host,
// each problem's tiles in grouped raster order); the table gives a unit's
// problem, tile coordinates and k-chunk count in one 16-byte load.
struct GroupedSched {
  const GroupedArgs* a;
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
    return v;
  }
};

template <int BN, bool TF32, class Sched>
__device__ __forceinline__ void tc_gemm_body(const Sched& sc) {
  using Cfg = TcCfg<BN, TF32>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (sbase - raw);
  int* const err = sc.err();
  const int nunits = sc.units();
  const int kb = sc.kb();

  // barrier block after the stage ring
  float* epi_buf = reinterpret_cast<float*>(smem + STAGES * Cfg::STAGE);
  uint8_t* bar_area = smem + STAGES * Cfg::STAGE + Cfg::EPI_BYTES;
  const uint32_t bar0 = sbase + STAGES * Cfg::STAGE + Cfg::EPI_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_area + 8 * (2 * STAGES + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 128 * Cfg::EPI_WG);
    }
    mbar_init(drain_bar, 1);
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

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      uint32_t last_phase[STAGES];
      bool issued[STAGES];
      for (int s = 0; s < STAGES; ++s) issued[s] = false, last_phase[s] = 0;
      bool ok = true;
      int last_prob = -1;
      Work wn = nunits > 0 ? sc.work(min(static_cast<int>(blockIdx.x), nunits - 1)) : Work{};
      for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        const Work w = wn;                         // next unit's entry loads early
        if (u + static_cast<int>(gridDim.x) < nunits) wn = sc.work(u + gridDim.x);
        const CUtensorMap* mA = sc.mapA(w.prob);
        const CUtensorMap* mB = sc.mapB(w.prob);
        if (w.prob != last_prob) {
          tma_prefetch_desc(mA);
          tma_prefetch_desc(mB);
          last_prob = w.prob;
        }
        for (int c = w.c0; c < w.c1; ++c) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t fb = full_bar(stage);
          mbar_arrive_expect_tx(fb, Cfg::STAGE);
          const uint32_t sA = sbase + stage * Cfg::STAGE;
          const int kx = c * Cfg::BK;
          tma_load_3d(sA, mA, fb, kx, w.tm * Cfg::BM, 0);
          tma_load_3d(sA + Cfg::A_PLANE, mA, fb, kx, w.tm * Cfg::BM, 1);
          tma_load_3d(sA + 2 * Cfg::A_PLANE, mB, fb, kx, w.tn * BN, 0);
          tma_load_3d(sA + 2 * Cfg::A_PLANE + Cfg::B_PLANE, mB, fb, kx, w.tn * BN, 1);
          issued[stage] = true;
          last_phase[stage] = phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
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
      uint32_t stage = 0, phase = 0, ab = 0, aphase = 0;
      bool ok = true;
      bool any = false;
      Work wn = nunits > 0 ? sc.work(min(static_cast<int>(blockIdx.x), nunits - 1)) : Work{};
      for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        const Work w = wn;
        if (u + static_cast<int>(gridDim.x) < nunits) wn = sc.work(u + gridDim.x);
        for (int cb = w.c0; ok && cb < w.c1; cb += kb) {
          const int ce = min(cb + kb, w.c1);
          if (!mbar_wait(acce_bar(ab), aphase ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + ab * BN;
          for (int c = cb; c < ce; ++c) {
            if (!mbar_wait(full_bar(stage), phase, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sAhi = sbase + stage * Cfg::STAGE;
            const uint32_t sAlo = sAhi + Cfg::A_PLANE;
            const uint32_t sBhi = sAhi + 2 * Cfg::A_PLANE;
            const uint32_t sBlo = sBhi + Cfg::B_PLANE;
#pragma unroll
            for (int kk = 0; kk < Cfg::KSTEPS; ++kk) {
              const uint32_t off = kk * 32;   // 32 bytes = one MMA's K slice
              const uint64_t dAhi = sdesc_k<Cfg::SW>(sAhi + off);
              const uint64_t dAlo = sdesc_k<Cfg::SW>(sAlo + off);
              const uint64_t dBhi = sdesc_k<Cfg::SW>(sBhi + off);
              const uint64_t dBlo = sdesc_k<Cfg::SW>(sBlo + off);
              const uint32_t acc = (c > cb || kk > 0) ? 1u : 0u;
              if (TF32) {
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
          ab ^= 1u;
          if (ab == 0) aphase ^= 1u;
        }
      }
      if (any) {
        // every MMA this thread issued has finished before TMEM is released
        umma_commit(drain_bar);
        mbar_wait_drain(drain_bar, 0);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int EC = Cfg::EPI_COLS;
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int half = (warp - 2) >> 2;       // column group of this warpgroup
    uint32_t ab = 0, aphase = 0;
    bool ok = true;
    Work wn = nunits > 0 ? sc.work(min(static_cast<int>(blockIdx.x), nunits - 1)) : Work{};
    for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      const Work w = wn;
      if (u + static_cast<int>(gridDim.x) < nunits) wn = sc.work(u + gridDim.x);
      float S[EC];
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
            tmem_base + (static_cast<uint32_t>(q * 32) << 16) + ab * BN + half * EC;
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
        }
        tc_fence_before();
        mbar_arrive(acce_bar(ab));
        ab ^= 1u;
        if (ab == 0) aphase ^= 1u;
      }
      if (!ok) break;
      const EpiView v = sc.epi(w.prob);
      if (blk == 0 || v.alpha == 0.0f) {
        // K == 0 or alpha == 0 (grouped problems only): C = beta * C; the
        // planes of such a problem are not packed, so their TMEM sum is unused
#pragma unroll
        for (int i = 0; i < EC; ++i) S[i] = 0.0f;
      }

      // undo the block scaling, acc * 2^(eA + eB).  With e != 0 alpha is
      // applied before the power of two, so that a result in range is not
      // lost to an overflow of the unscaled sum (the power of two is exact).
      const int col0 = w.tn * BN + half * EC;
      const int e = block_exponent(v.amaxA[w.tm]) + block_exponent(v.amaxB[col0 / kScaleBlock]);
      float alpha = v.alpha;
      float beta = v.beta;
      if (v.split_k > 1 || e != 0) {
#pragma unroll
        for (int i = 0; i < EC; ++i) S[i] = e != 0 ? scale_pow2(alpha * S[i], e) : alpha * S[i];
        alpha = 1.0f;
      }
      // destination: C, or this split's partial-sum plane (the reduction
      // kernel adds beta * C)
      float* dst = v.C;
      int64_t ldd = v.ldc;
      if (v.split_k > 1) {
        dst = v.partial + static_cast<int64_t>(w.ks) * v.M * v.N;
        ldd = v.N;
        beta = 0.0f;
      }
      // Two store paths, chosen per 32-column chunk and uniform per warp.
      // Aligned rows and a full chunk: each thread stores its own row with
      // float4 accesses (C loads of the chunk issued first).  Otherwise
      // (unaligned ldc, partial chunk or rows): the warp stages the 32x32
      // chunk of its rows (lane = row) in a padded shared buffer, then walks
      // it one row at a time (lane = column), so that every global access of
      // the warp covers 128 contiguous bytes of one row whatever the alignment.
      float* buf = epi_buf + (warp - 2) * 32 * Cfg::EPI_PITCH;
      const int row0 = w.tm * 128 + q * 32;
      const int nrows = min(32, v.M - row0);
      const bool rows_vec = nrows == 32 && (ldd & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
#pragma unroll
      for (int j = 0; j < EC / 32; ++j) {
        const int cb = col0 + j * 32;
        if (nrows <= 0 || cb >= v.N) break;   // uniform across the warp
        if (rows_vec && cb + 32 <= v.N) {
          float4* c4 = reinterpret_cast<float4*>(dst + static_cast<int64_t>(row0 + lane) * ldd + cb);
          float4 old[8];
          if (beta != 0.0f) {
#pragma unroll
            for (int i = 0; i < 8; ++i) old[i] = c4[i];
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float* sv = &S[j * 32 + 4 * i];
            float4 o;
            if (beta != 0.0f) {
              o.x = fmaf(alpha, sv[0], beta * old[i].x);
              o.y = fmaf(alpha, sv[1], beta * old[i].y);
              o.z = fmaf(alpha, sv[2], beta * old[i].z);
              o.w = fmaf(alpha, sv[3], beta * old[i].w);
            } else {
              o.x = alpha * sv[0];
              o.y = alpha * sv[1];
              o.z = alpha * sv[2];
              o.w = alpha * sv[3];
            }
            c4[i] = o;
          }
          continue;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) buf[lane * Cfg::EPI_PITCH + i] = S[j * 32 + i];
        __syncwarp();
        const bool col_ok = cb + lane < v.N;
        float* base = dst + static_cast<int64_t>(row0) * ldd + cb + lane;
#pragma unroll
        for (int r0 = 0; r0 < 32; r0 += 8) {
          float old[8];
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) {
            const int r = r0 + rr;
            old[rr] = (beta != 0.0f && col_ok && r < nrows) ? base[r * ldd] : 0.0f;
          }
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) {
            const int r = r0 + rr;
            if (col_ok && r < nrows) {
              const float sv = buf[r * Cfg::EPI_PITCH + lane];
              base[r * ldd] = beta != 0.0f ? fmaf(alpha, sv, beta * old[rr]) : alpha * sv;
            }
          }
        }
        __syncwarp();
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

template <int BN, bool TF32>
__global__ void __launch_bounds__(TcCfg<BN, TF32>::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs a) {
  SingleSched sc{&tmA, &tmB, &a};
  tc_gemm_body<BN, TF32>(sc);
}

template <int BN, bool TF32>
__global__ void __launch_bounds__(TcCfg<BN, TF32>::THREADS, 1) tc_grouped_kernel(const GroupedArgs a) {
  GroupedSched sc{&a};
  tc_gemm_body<BN, TF32>(sc);
}

// Split-K fix-up: C = sum_s partial[s] + beta * C, where each partial already
// holds alpha * (its share of A*B); partials are summed in increasing s (a
// fixed order, so results do not depend on timing).
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ partial,
                                     float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t total = static_cast<int64_t>(M) * N;
  const int64_t plane = total;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float s = partial[idx];
    for (int k = 1; k < splits; ++k) s += partial[k * plane + idx];
    const int64_t r = idx / N, c = idx % N;
    float* cp = C + r * ldc + c;
    *cp = beta != 0.0f ? s + beta * *cp : s;
  }
}

int tc_smem_bytes(int bn, Prec prec) {
  if (prec == Prec::TF32) return bn == 64 ? TcCfg<64, true>::SMEM : TcCfg<128, true>::SMEM;
  return bn == 64 ? TcCfg<64, false>::SMEM : TcCfg<128, false>::SMEM;
}

int tc_chunk_bytes(int bn) {
  (void)bn;   // every variant steps in 128-byte chunks (see TcCfg)
  return 128;
}

// The dynamic shared memory limit of every kernel variant is raised once per
// device and thread, outside any stream capture: plans call tc_prepare when
// they are created, launches call it again (a no-op after the first time).
template <int BN, bool TF32>
static cudaError_t prepare_variant() {
  using Cfg = TcCfg<BN, TF32>;
  static thread_local int configured_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device != dev) {
    e = cudaFuncSetAttribute(tc_gemm_kernel<BN, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tc_grouped_kernel<BN, TF32>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  return cudaSuccess;
}

cudaError_t tc_prepare(int bn, Prec prec) {
  if (prec == Prec::TF32) {
    if (bn == 64) return prepare_variant<64, true>();
    if (bn == 128) return prepare_variant<128, true>();
  } else {
    if (bn == 64) return prepare_variant<64, false>();
    if (bn == 128) return prepare_variant<128, false>();
  }
  return cudaErrorInvalidValue;
}

template <int BN, bool TF32>
static cudaError_t launch_variant(int grid, const CUtensorMap& tmA, const CUtensorMap& tmB,
                                  const TcArgs& a, cudaStream_t s) {
  using Cfg = TcCfg<BN, TF32>;
  cudaError_t e = prepare_variant<BN, TF32>();
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<BN, TF32><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(tmA, tmB, a);
  return cudaGetLastError();
}

cudaError_t tc_gemm_launch(const TcLaunch& l, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const TcArgs& a, cudaStream_t s) {
  if (l.prec == Prec::TF32) {
    if (l.bn == 64) return launch_variant<64, true>(l.grid, tmA, tmB, a, s);
    if (l.bn == 128) return launch_variant<128, true>(l.grid, tmA, tmB, a, s);
  } else {
    if (l.bn == 64) return launch_variant<64, false>(l.grid, tmA, tmB, a, s);
    if (l.bn == 128) return launch_variant<128, false>(l.grid, tmA, tmB, a, s);
  }
  return cudaErrorInvalidValue;
}

template <int BN, bool TF32>
static cudaError_t launch_grouped_variant(int grid, const GroupedArgs& a, cudaStream_t s) {
  using Cfg = TcCfg<BN, TF32>;
  cudaError_t e = prepare_variant<BN, TF32>();
  if (e != cudaSuccess) return e;
  tc_grouped_kernel<BN, TF32><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tc_grouped_launch(int bn, Prec prec, int grid, const GroupedArgs& a, cudaStream_t s) {
  if (prec == Prec::TF32) {
    if (bn == 64) return launch_grouped_variant<64, true>(grid, a, s);
    if (bn == 128) return launch_grouped_variant<128, true>(grid, a, s);
  } else {
    if (bn == 64) return launch_grouped_variant<64, false>(grid, a, s);
    if (bn == 128) return launch_grouped_variant<128, false>(grid, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t splitk_reduce_launch(int M, int N, int splits, const float* partial, float beta,
                                 float* C, int64_t ldc, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(M) * N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  splitk_reduce_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(M, N, splits, partial, beta, C,
                                                               ldc);
  return cudaGetLastError();
}

}  // namespace gb
