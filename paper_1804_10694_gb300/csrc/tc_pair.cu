// The split-precision gemm on pairs of SMs: C = alpha * A * B + beta * C with
// FP32 semantics, each output tile 256 x BN computed by a cluster of two
// CTAs with the fifth-generation tensor core's CTA-pair MMA (tcgen05,
// cta_group::2).
//
// The paper's gemm recipe is two-level tiling with register blocking
// (Section I; Section VI-A): the larger the tile a compute unit holds, the
// fewer operand bytes it moves per multiply-add.  On sm_103a the widest tile
// one MMA can produce is 256 x 256, spread over two SMs: the leader CTA
// (cluster rank 0) issues an MMA that reads A's rows 0..127 from its own
// shared memory and rows 128..255 from its peer's, B's first BN/2 columns
// from its own and the other BN/2 from its peer's, and writes each CTA's
// 128 rows of the FP32 accumulator into that CTA's tensor memory.  Against
// the single-CTA 128 x 128 tile, a 256 x 256 pair tile halves the shared
// memory bytes read per MMA (each SM supplies 128 rows of A and 128 of B for
// twice the products) and the L2 -> SM operand traffic per flop.
//
// Pipeline (both CTAs run the same roles on the same units of work):
//   warp 0, one thread: TMA producer.  Each CTA loads its own half of every
//     operand tile into its own ring stage, after its own stage-empty
//     barrier completed; every load signals the LEADER's stage-full barrier
//     (one arrival: the leader's expect_tx of both CTAs' bytes).
//   warp 1: allocates the pair's tensor memory (both CTAs); in the leader,
//     one thread waits for each stage, issues the pair MMAs (three products
//     per 32-byte K slice: lo*hi, hi*lo, hi*hi; or the six of BF16x6) and
//     commits them to the stage-empty barriers and, every kb chunks, to the
//     accumulator-full barriers of BOTH CTAs (multicast commit).
//   warps 4..: epilogue, in each CTA: wait for the accumulator, fold it into
//     FP32 registers, release it (one arrival per warp on the leader's
//     accumulator-empty barrier), then undo the block scaling and apply
//     alpha/beta for the CTA's 128 rows (the same epilogue as the single-CTA
//     kernel).
// Every wait is bounded; both CTAs meet at a cluster barrier before the
// tensor memory is released.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <utility>

#include "epilogue.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "scale.cuh"
#include "tile_order.cuh"

namespace gb {

// Geometry of one pair-kernel variant: output tile 256 x BN, 128 rows per
// CTA; each CTA stages 128 rows of A and BN/2 rows of (K-major) B per
// 128-byte k-chunk and plane.
template <int BN, bool TF32, int NP>
struct PairCfg {
  static_assert(BN == 128 || BN == 256, "pair tile width");
  static_assert(NP == 2 || (NP == 3 && !TF32), "three planes: bf16 only");
  static constexpr int BM = 128;                 // rows of A (and C) per CTA
  static constexpr int BNH = BN / 2;             // rows of K-major B per CTA
  static constexpr int SW = 128;                 // bytes of one row per k-chunk
  static constexpr int A_PLANE = BM * SW;
  static constexpr int B_PLANE = BNH * SW;
  static constexpr int STAGE = NP * (A_PLANE + B_PLANE);
  static constexpr int BK = SW / (TF32 ? 4 : 2); // elements per k-chunk
  static constexpr int KSTEPS = SW / 32;         // MMAs (32-byte K slices) per chunk and product
  // warpgroup 0: warp 0 the TMA producer, warp 1 the MMA issuer, warps 2-3
  // idle; then one epilogue warpgroup per 128 accumulator columns (a thread
  // folds 128 columns in registers)
  static constexpr int EPI_WG = BN / 128;
  static constexpr int EPI_WARP0 = 4;
  static constexpr int EPI_COLS = BN / EPI_WG;
  static constexpr int ACC_COLS = NP == 3 ? 2 * BN : BN;   // TMEM columns of one accumulator buffer
  static constexpr int NACC = 512 / ACC_COLS >= 4 ? 4 : 512 / ACC_COLS;
  static constexpr int TMEM_COLS = NACC * ACC_COLS;
  static constexpr int EPI_PITCH = 33;
  static constexpr int EPI_BYTES = 4 * EPI_WG * 32 * EPI_PITCH * 4;
  static constexpr int BAR_BYTES = 256;
  // ring as deep as shared memory allows (at most 6 stages)
  static constexpr int RING_BUDGET = 232448 - 1024 - EPI_BYTES - BAR_BYTES;
  static constexpr int STAGES = RING_BUDGET / STAGE > 6 ? 6 : RING_BUDGET / STAGE;
  static constexpr int OFF_EPI = STAGES * STAGE;
  static constexpr int OFF_BAR = OFF_EPI + EPI_BYTES;
  static constexpr int SMEM = OFF_BAR + BAR_BYTES + 1024;
  static constexpr int THREADS = 128 + 128 * EPI_WG;
  // Registers: a CTA of more than 256 threads is compiled for at most 168 a
  // thread (384 x 168 = the 64 K register file), too few for a thread that
  // holds 128 sums.  With two epilogue warpgroups, warpgroup 0 gives
  // registers back (setmaxnreg) and the epilogue warpgroups take them:
  // 128 x REGS_CTRL + 256 x REGS_EPI = 384 x 168, exactly the launch's pool.
  static constexpr int REGS_LAUNCH = 168;
  static constexpr int REGS_CTRL = 72;
  static constexpr int REGS_EPI = (THREADS * REGS_LAUNCH - 128 * REGS_CTRL) / (128 * EPI_WG);
  static_assert(EPI_WG == 1 || (THREADS == 384 && REGS_EPI == 216 &&
                                128 * REGS_CTRL + 256 * REGS_EPI == 384 * REGS_LAUNCH),
                "register split adds up to the launch's pool");
  static_assert(STAGES >= 2, "ring depth");
  static_assert(SMEM <= 232448, "shared memory budget");
  static_assert(TMEM_COLS <= 512, "tensor memory budget");
  static_assert(8 * (2 * STAGES + 2 * NACC + 1) + 8 <= BAR_BYTES, "barrier block");
};

// Units are (split, pair tile) pairs; a.tiles_m counts 256-row pair tiles
// and a.tm0 is the first 128-row block of the launch (even).
template <int BN, bool TF32, int NP>
__global__ void __launch_bounds__(PairCfg<BN, TF32, NP>::THREADS, 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const TcArgs a) {
  using Cfg = PairCfg<BN, TF32, NP>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr int NACC = Cfg::NACC;
  constexpr int EC = Cfg::EPI_COLS;
  extern __shared__ uint8_t smem_raw[];
  // both CTAs run the same code with the same dynamic shared memory, so the
  // 1024-aligned base (and every stage) has the same offset in both: the
  // pair MMA addresses the peer's operands at the leader's offsets
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (sbase - raw);
  const uint32_t rank = cluster_ctarank();   // 0: leader (issues the MMAs), 1: peer
  const int pair0 = static_cast<int>(cluster_id_x());
  const int npairs = static_cast<int>(num_clusters_x());
  int* const err = a.err;
  const int nunits = a.num_units;
  const int kb = a.kb;

  float* epi_buf = reinterpret_cast<float*>(smem + Cfg::OFF_EPI);
  const uint32_t bar0 = sbase + Cfg::OFF_BAR;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };                      // leader's counts
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };          // each CTA's own
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };       // each CTA's own
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + NACC + b); };  // leader's counts
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 2 * NACC);
  constexpr int NBAR = 2 * STAGES + 2 * NACC + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cfg::OFF_BAR + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);    // the leader producer's arrive (with both CTAs' bytes)
      mbar_init(empty_bar(s), 1);   // the leader's commit
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(accf_bar(b), 1);                          // the leader's commit
      mbar_init(acce_bar(b), 2 * 4 * Cfg::EPI_WG);        // one arrival per epilogue warp, both CTAs
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_slot), Cfg::TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync();   // both CTAs' barriers initialised and tensor memory allocated
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  if (warp == 0 && lane == 0) {   // kernel parameters: fetched meanwhile
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  // The prologue above overlaps the packing kernel.  Every role but the TMA
  // producer waits here until that kernel has completed and its writes are
  // visible; with a.readyA set (that kernel packs both operands and marks
  // each block ready; all of its CTAs have started when this launch starts)
  // the producer instead waits for each block of the planes it loads.
  if (warp != 0 || a.readyA == nullptr) griddep_wait();
  // the stream's next kernel may be scheduled now (it waits for this launch
  // to complete before it touches anything)
  griddep_launch_dependents();

  auto work = [&](int u) {
    Work w;
    const int t = u % a.num_tiles;
    w.prob = 0;
    w.ks = u / a.num_tiles;
    raster(t, a.tiles_m, a.tiles_n, a.group_m, w.tm, w.tn);
    w.c0 = w.ks * a.chunks_per_split;
    w.c1 = min(w.c0 + a.chunks_per_split, a.chunks_total);
    return w;
  };
  // the 128-row block of A and C this CTA covers in pair tile tm
  auto row_block = [&](int tm) { return a.tm0 + 2 * tm + static_cast<int>(rank); };

  if (warp < Cfg::EPI_WARP0) {
    // all four warps of warpgroup 0 give registers back, then take their roles
    if constexpr (Cfg::EPI_WG > 1) warpgroup_regs_dec<Cfg::REGS_CTRL>();
    if (warp == 0) {
      // ------------------------------------------------------------ producer
      if (lane == 0) {
        const bool hints = a.group_m > 1;   // consecutive waves keep the same rows of A
        const uint64_t polA = l2_policy_evict_last();
        const uint32_t full0_leader = mapa_shared(full_bar(0), 0);
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        uint32_t stage = 0, phase = 0;
        uint32_t last_phase[STAGES];
        bool issued[STAGES];
        for (int s = 0; s < STAGES; ++s) issued[s] = false, last_phase[s] = 0;
        bool ok = true;
        int ready_a = -1, ready_b = -1;   // the last blocks seen ready
        for (int u = pair0; ok && u < nunits; u += npairs) {
          const Work w = work(u);
          const int rowA = row_block(w.tm) * Cfg::BM;
          const int rowB = w.tn * BN + static_cast<int>(rank) * Cfg::BNH;
          if (a.readyA != nullptr) {
            // the blocks of A's rows and B's columns this CTA loads; a block
            // wholly past M or N (this CTA's half of the last pair tile) has
            // no planes and no counter: its loads only zero-fill
            const int ba = row_block(w.tm), bb = rowB / kScaleBlock;
            if (ba != ready_a || bb != ready_b) {
              if ((ba * kScaleBlock < a.M && !wait_flag_bit(a.readyA + ba, kBlockReady, abort_flag, err)) ||
                  (bb * kScaleBlock < a.N && !wait_flag_bit(a.readyB + bb, kBlockReady, abort_flag, err))) {
                ok = false;
                break;
              }
              fence_proxy_async_global();
              ready_a = ba, ready_b = bb;
            }
          }
          for (int c = w.c0; c < w.c1; ++c) {
            if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, err)) {
              ok = false;
              break;
            }
            const uint32_t sA = sbase + stage * Cfg::STAGE;
            const uint32_t sB = sA + NP * Cfg::A_PLANE;
            const int kx = c * Cfg::BK;
            if (rank == 0) {
              const uint32_t fb = full_bar(stage);
              mbar_arrive_expect_tx(fb, 2u * Cfg::STAGE);
  #pragma unroll
              for (int z = 0; z < NP; ++z) {
                if (hints) tma_load_3d_hint(sA + z * Cfg::A_PLANE, &tmA, fb, kx, rowA, z, polA);
                else tma_load_3d(sA + z * Cfg::A_PLANE, &tmA, fb, kx, rowA, z);
              }
  #pragma unroll
              for (int z = 0; z < NP; ++z) tma_load_3d(sB + z * Cfg::B_PLANE, &tmB, fb, kx, rowB, z);
            } else {
              const uint32_t fb = full0_leader + 8u * stage;   // the leader's stage barrier
  #pragma unroll
              for (int z = 0; z < NP; ++z) {
                if (hints) tma_load_3d_pair_hint(sA + z * Cfg::A_PLANE, &tmA, fb, kx, rowA, z, polA);
                else tma_load_3d_pair(sA + z * Cfg::A_PLANE, &tmA, fb, kx, rowA, z);
              }
  #pragma unroll
              for (int z = 0; z < NP; ++z) tma_load_3d_pair(sB + z * Cfg::B_PLANE, &tmB, fb, kx, rowB, z);
            }
            issued[stage] = true;
            last_phase[stage] = phase;
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok && rank == 0) {
          // abort: let the copies signalled here land before shared memory is released
          for (int s = 0; s < STAGES; ++s)
            if (issued[s]) mbar_wait_drain(full_bar(s), last_phase[s]);
        }
      }
    } else if (warp == 1) {
      // ------------------------------------------------------------ MMA issuer (leader)
      if (lane == 0 && rank == 0) {
        constexpr uint32_t idesc = idesc_f32acc(TF32, 256, BN);
        uint32_t stage = 0, phase = 0, ab = 0, aphase = 0;
        bool ok = true;
        bool any = false;
        for (int u = pair0; ok && u < nunits; u += npairs) {
          const Work w = work(u);
          for (int cb = w.c0; ok && cb < w.c1; cb += kb) {
            const int ce = min(cb + kb, w.c1);
            if (!mbar_wait_cluster(acce_bar(ab), aphase ^ 1u, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem_base + ab * Cfg::ACC_COLS;
            for (int c = cb; c < ce; ++c) {
              if (!mbar_wait_cluster(full_bar(stage), phase, abort_flag, err)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sAhi = sbase + stage * Cfg::STAGE;
              const uint32_t sAlo = sAhi + Cfg::A_PLANE;
              const uint32_t sBhi = sAhi + NP * Cfg::A_PLANE;
              const uint32_t sBlo = sBhi + Cfg::B_PLANE;
  #pragma unroll
              for (int kk = 0; kk < Cfg::KSTEPS; ++kk) {
                const uint32_t off = kk * 32;   // 32 bytes = one MMA's K slice
                const uint64_t dAhi = sdesc_k_sw128(sAhi + off);
                const uint64_t dAlo = sdesc_k_sw128(sAlo + off);
                const uint64_t dBhi = sdesc_k_sw128(sBhi + off);
                const uint64_t dBlo = sdesc_k_sw128(sBlo + off);
                const uint32_t acc = (c > cb || kk > 0) ? 1u : 0u;
                if constexpr (NP == 3) {
                  // planes hi, mid, lo: the five smaller products into the
                  // second accumulator (smallest first), hi*hi into the first
                  const uint32_t d2 = d + BN;
                  const uint64_t dAl2 = sdesc_k_sw128(sAhi + 2 * Cfg::A_PLANE + off);
                  const uint64_t dBl2 = sdesc_k_sw128(sBhi + 2 * Cfg::B_PLANE + off);
                  umma_bf16_pair(d2, dAl2, dBhi, idesc, acc);
                  umma_bf16_pair(d2, dAlo, dBlo, idesc, 1u);
                  umma_bf16_pair(d2, dAhi, dBl2, idesc, 1u);
                  umma_bf16_pair(d2, dAlo, dBhi, idesc, 1u);
                  umma_bf16_pair(d2, dAhi, dBlo, idesc, 1u);
                  umma_bf16_pair(d, dAhi, dBhi, idesc, acc);
                } else if (TF32) {
                  umma_tf32_pair(d, dAlo, dBhi, idesc, acc);
                  umma_tf32_pair(d, dAhi, dBlo, idesc, 1u);
                  umma_tf32_pair(d, dAhi, dBhi, idesc, 1u);
                } else {
                  umma_bf16_pair(d, dAlo, dBhi, idesc, acc);
                  umma_bf16_pair(d, dAhi, dBlo, idesc, 1u);
                  umma_bf16_pair(d, dAhi, dBhi, idesc, 1u);
                }
              }
              any = true;
              umma_commit_pair(empty_bar(stage), 0x3);   // the stage is free in both CTAs
              if (++stage == STAGES) {
                stage = 0;
                phase ^= 1u;
              }
            }
            if (!ok) break;
            umma_commit_pair(accf_bar(ab), 0x3);         // both CTAs' halves are ready
            if (++ab == NACC) {
              ab = 0;
              aphase ^= 1u;
            }
          }
        }
        if (any) {
          // every MMA issued has finished before tensor memory is released
          umma_commit_pair(drain_bar, 0x1);
          mbar_wait_drain(drain_bar, 0);
        }
      }
      __syncwarp();
    }
  } else {
    // ------------------------------------------------------------ epilogue (both CTAs)
    if constexpr (Cfg::EPI_WG > 1) warpgroup_regs_inc<Cfg::REGS_EPI>();
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int half = (warp - Cfg::EPI_WARP0) >> 2;   // column group of this warpgroup
    // the leader's accumulator-empty barriers, as this CTA reaches them
    const uint32_t acce0 = rank == 0 ? acce_bar(0) : mapa_shared(acce_bar(0), 0);
    uint32_t ab = 0, aphase = 0;
    bool ok = true;
    for (int u = pair0; ok && u < nunits; u += npairs) {
      const Work w = work(u);
      EpiView v;
      v.M = a.M, v.N = a.N, v.C = a.C, v.ldc = a.ldc, v.alpha = a.alpha, v.beta = a.beta;
      v.amaxA = a.amaxA, v.amaxB = a.amaxB, v.partial = a.partial, v.split_k = a.split_k;
      v.amaxA_stride = 1;
      const int rb = row_block(w.tm);
      const int col0 = w.tn * BN + half * EC;
      const int e = block_exponent(a.amaxA[rb]) + block_exponent(a.amaxB[col0 / kScaleBlock]);
      {
        // warm L2 with the part of C this thread will read (beta != 0)
        const int prow = rb * 128 + q * 32 + lane;
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
      int blk = 0;
      for (int cb = w.c0; cb < w.c1; cb += kb, ++blk) {
        const bool waited = mbar_wait_cluster(accf_bar(ab), aphase, abort_flag, err);
        if (!__all_sync(0xffffffffu, waited)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr =
            tmem_base + (static_cast<uint32_t>(q * 32) << 16) + ab * Cfg::ACC_COLS + half * EC;
        // 16 columns a load: a thread holds EC = 128 sums, and the load's
        // registers must fit beside them
#pragma unroll
        for (int j = 0; j < EC / 16; ++j) {
          uint32_t r[16];
          tmem_ld_32x32b_x16(taddr + j * 16, r);
          tmem_wait_ld();
          if (blk == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) S[j * 16 + i] = __uint_as_float(r[i]);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) S[j * 16 + i] += __uint_as_float(r[i]);
          }
          if constexpr (NP == 3) {
            tmem_ld_32x32b_x16(taddr + BN + j * 16, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) S[j * 16 + i] += __uint_as_float(r[i]);
          }
        }
        // every lane's loads are done; then one arrival for the warp
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (rank == 0) mbar_arrive(acce_bar(ab));
          else mbar_arrive_cluster(acce0 + 8u * ab);
        }
        if (++ab == NACC) {
          ab = 0;
          aphase ^= 1u;
        }
      }
      if (!ok) break;
      if (blk == 0 || v.alpha == 0.0f) {
#pragma unroll
        for (int i = 0; i < EC; ++i) S[i] = 0.0f;
      }
      epilogue_store<EC, Cfg::EPI_PITCH>(S, v, e, w.ks, rb * 128 + q * 32, col0, lane,
                                         epi_buf + (warp - Cfg::EPI_WARP0) * 32 * Cfg::EPI_PITCH);
    }
  }

  // both CTAs are done with the pair's tensor memory and with each other's
  // barriers before either releases them
  tc_fence_before();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, Cfg::TMEM_COLS);
  }
  // every role of this CTA is past its last read of the block maxima (the
  // cluster barrier above)
  clear_execution_state(a.state, a.state_words);
}

// ------------------------------------------------------------------- launch
template <int BN, bool TF32, int NP>
static cudaError_t prepare_pair_variant(int* max_pairs) {
  using Cfg = PairCfg<BN, TF32, NP>;
  static std::mutex mu;
  static int configured[64], pairs[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!configured[dev]) {
    e = cudaFuncSetAttribute(tc_gemm_pair_kernel<BN, TF32, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg::SMEM);
    if (e != cudaSuccess) return e;
    // pairs of SMs that can hold one cluster each at the same time
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(Cfg::THREADS);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, tc_gemm_pair_kernel<BN, TF32, NP>, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    pairs[dev] = n;
    configured[dev] = 1;
  }
  if (max_pairs) *max_pairs = pairs[dev];
  return cudaSuccess;
}

cudaError_t tc_pair_prepare(int bn, Prec prec, int* max_pairs) {
  if (prec == Prec::TF32) {
    if (bn == 128) return prepare_pair_variant<128, true, 2>(max_pairs);
    if (bn == 256) return prepare_pair_variant<256, true, 2>(max_pairs);
  } else if (prec == Prec::BF16X6) {
    if (bn == 128) return prepare_pair_variant<128, false, 3>(max_pairs);
    if (bn == 256) return prepare_pair_variant<256, false, 3>(max_pairs);
  } else {
    if (bn == 128) return prepare_pair_variant<128, false, 2>(max_pairs);
    if (bn == 256) return prepare_pair_variant<256, false, 2>(max_pairs);
  }
  return cudaErrorInvalidValue;
}

// Clusters of two CTAs, launched as a programmatic dependent of the previous
// kernel (the packing pass) like the single-CTA kernel.
template <int BN, bool TF32, int NP>
static cudaError_t launch_pair_variant(int grid, const CUtensorMap& tmA, const CUtensorMap& tmB,
                                       const TcArgs& a, cudaStream_t s) {
  using Cfg = PairCfg<BN, TF32, NP>;
  cudaError_t e = prepare_pair_variant<BN, TF32, NP>(nullptr);
  if (e != cudaSuccess) return e;
  if (grid < 2 || grid % 2 != 0) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Cfg::THREADS);
  cfg.dynamicSmemBytes = static_cast<size_t>(Cfg::SMEM);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, tc_gemm_pair_kernel<BN, TF32, NP>, tmA, tmB, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t tc_pair_launch(int bn, Prec prec, int grid, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const TcArgs& a, cudaStream_t s) {
  if (prec == Prec::TF32) {
    if (bn == 128) return launch_pair_variant<128, true, 2>(grid, tmA, tmB, a, s);
    if (bn == 256) return launch_pair_variant<256, true, 2>(grid, tmA, tmB, a, s);
  } else if (prec == Prec::BF16X6) {
    if (bn == 128) return launch_pair_variant<128, false, 3>(grid, tmA, tmB, a, s);
    if (bn == 256) return launch_pair_variant<256, false, 3>(grid, tmA, tmB, a, s);
  } else {
    if (bn == 128) return launch_pair_variant<128, false, 2>(grid, tmA, tmB, a, s);
    if (bn == 256) return launch_pair_variant<256, false, 2>(grid, tmA, tmB, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gb
