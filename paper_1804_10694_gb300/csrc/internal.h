// Declarations shared by the library's translation units (not part of the
// public C ABI, which is include/gemm.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace gb {

// ---------------------------------------------------------------- precision
// BF16: two bf16 planes (hi, lo), three products; BF16X6: three bf16 planes
// (hi, mid, lo), six products; TF32: two tf32 planes, three products.
enum class Prec : int { F32 = 0, BF16 = 1, TF32 = 2, BF16X6 = 3 };

inline bool prec_bf16(Prec p) { return p == Prec::BF16 || p == Prec::BF16X6; }
inline int prec_elem_bytes(Prec p) { return prec_bf16(p) ? 2 : 4; }
// Planes each operand is split into.
inline int prec_planes(Prec p) { return p == Prec::BF16X6 ? 3 : 2; }
// Elements of one 128-byte k-chunk (one swizzle span) per precision.
inline int prec_chunk_elems(Prec p) { return prec_bf16(p) ? 64 : 32; }
// Row pitch of the packed planes: K rounded up so that a row is 16-byte aligned.
inline int64_t packed_k_pitch(Prec p, int64_t K) {
  const int64_t q = prec_bf16(p) ? 8 : 4;
  return (K + q - 1) / q * q;
}

constexpr int kScaleBlock = 128;   // rows of A / columns of B sharing one exponent
// Set in a block's pack counter once the block's planes (and maximum) are
// final: by the CTA that completed the block, after re-splitting it if its
// exponent is not zero.
constexpr unsigned kBlockReady = 0x80000000u;

// --------------------------------------------------- tensor-core kernel args
struct TcArgs {
  int M, N, K;
  int tm0;       // first row tile of this launch (a row panel); 0 for the whole matrix
  int tiles_m, tiles_n, num_tiles, num_units;
  int split_k, chunks_total, chunks_per_split;
  int kb;        // k-chunks accumulated in TMEM before the epilogue folds them in
                 // (bounded: the tensor core's own FP32 accumulation is not
                 // round-to-nearest, so long chains in TMEM lose accuracy)
  int group_m;   // raster: tiles grouped along M
  float alpha, beta;
  float* C;
  int64_t ldc;
  const unsigned* amaxA;   // per 128-row block of A: bit pattern of max |a|
  const unsigned* amaxB;   // per 128-column block of B
  float* partial;          // split-K partial sums [split][M][N], null when split_k == 1
  int* err;
  // fused-split variant only: A itself (row-major FP32, split inside the kernel)
  const float* A;
  int64_t lda;
  int vecA;                // A 16-byte aligned and lda % 4 == 0: float4 loads
  // direct convolution: A is the patch matrix of the NHWC image at A
  // (conv_N images of conv_H x conv_W x conv_C pixels) for an odd conv_R x
  // conv_S filter with same zero padding; one block exponent for the whole
  // image (amaxA[0]).  Fused variant: gathered from the FP32 image while
  // staging.  Packed variant (conv_C % 16 == 0, bf16 planes): the image is
  // split once into planes stacked as 2 conv_N images, and the kernel loads
  // 16-channel im2col boxes of them (plane z = images z conv_N ...).
  int conv, conv_N, conv_H, conv_W, conv_C, conv_R, conv_S;
  int conv_box_c;          // fused variant: channels per TMA im2col box (32, or 16), when vecA
  int* unit_ctr;           // packed convolution: units taken so far (zero before the launch)
  // per-execution state (block maxima, pack counters, unit counter) that the
  // last CTA of the launch clears, followed by its done counter; 0 words:
  // nothing to clear (the caller clears the state itself)
  unsigned* state;
  int state_words;
  // per-block pack counters of A's 128-row and B's 128-column blocks, when
  // the packing kernel right before this launch packs both (it sets
  // kBlockReady in each): the TMA producer then waits for the blocks each
  // unit loads instead of for the whole packing kernel (null: it waits for
  // that kernel, griddepcontrol.wait)
  const unsigned* readyA;
  const unsigned* readyB;
};

struct TcLaunch {
  int bn;          // tile N (64 or 128; 128 or 256 for a CTA pair; 32 for a narrow convolution)
  Prec prec;       // BF16, BF16X6 or TF32
  int grid;
  bool fused;      // A split inside the gemm kernel (only B is packed)
  int cluster;     // 1, or 2: a 256-row tile on a pair of SMs (tc_pair_launch)
  bool comp = false;   // compensated epilogue (single-CTA packed kernels only)
};

// Packed convolutions with at most 32 output features may run 128 x 32
// tiles (TcLaunch.bn = 32): CTAs of that kernel a SM holds at once (2, or 1
// for a precision whose ring does not fit twice).
int tc_narrow_ctas_per_sm(Prec prec);
// Returns the dynamic shared memory a tensor-core kernel variant needs.
int tc_smem_bytes(int bn, Prec prec, bool fused = false);
// Bytes of one row per k-chunk of the kernel variant with tile width bn (the
// swizzle width of its operand tiles: 128, or 64 for bn = 256).
int tc_chunk_bytes(int bn);
// Raise the shared-memory limit of a tile-width/precision variant on the
// current device (call outside stream capture; idempotent).
cudaError_t tc_prepare(int bn, Prec prec, bool fused = false);
cudaError_t tc_gemm_launch(const TcLaunch& l, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const TcArgs& a, cudaStream_t s);
// CTA-pair variants (tile 256 x bn, bn 128 or 256; clusters of two CTAs,
// tcgen05 cta_group::2): raise the shared-memory limit and report how many
// clusters can be resident at once (call outside stream capture), and
// launch (grid = 2 x clusters; a.tiles_m in 256-row tiles, a.tm0 even; tmB's
// box holds bn/2 rows).
cudaError_t tc_pair_prepare(int bn, Prec prec, int* max_pairs);
cudaError_t tc_pair_launch(int bn, Prec prec, int grid, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const TcArgs& a, cudaStream_t s);
// C = sum_s partial[s] + beta * C over the split-K partial sums (alpha is
// already inside the partials).
cudaError_t splitk_reduce_launch(int M, int N, int splits, const float* partial, float beta,
                                 float* C, int64_t ldc, cudaStream_t s);

// ------------------------------------------------------------ SIMT kernel
// transA: A stored K x M (lda >= M); transB: B stored N x K (ldb >= K).
cudaError_t simt_gemm_launch(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                             int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                             int64_t ldc, cudaStream_t s, bool transA = false, bool transB = false);
// C = beta * C (K == 0 or alpha == 0), C write-only when beta == 0.
cudaError_t scale_c_launch(int64_t M, int64_t N, float beta, float* C, int64_t ldc, cudaStream_t s);

// ------------------------------------------------------------ split / pack
// Packing (split.cu), both operands in one launch: the unscaled planes and
// the per-block max |x| bit patterns (A: blocks of 128 rows, into amaxA; B,
// transposed: blocks of 128 columns, into amaxB); amax* hold the block
// maxima and cnt* one counter per block (items done), both zero on entry.
// The CTA that completes a block re-splits it with its exponent when the
// block lies outside the safe range.  A (or B) may be null to pack only the
// other operand.
// A: M x K (lda) -> planesA [P][M][pitch];  B: K x N (ldb) -> planesB [P][N][pitch],
// P = prec_planes(prec).
// transA: A is stored K x M (lda >= M); transB: B is stored N x K (ldb >= K).
cudaError_t pack_launch(Prec prec, const float* A, int64_t M, int64_t K, int64_t lda, const float* B,
                        int64_t N, int64_t ldb, unsigned* amaxA, unsigned* amaxB, unsigned* cntA,
                        unsigned* cntB, void* planesA, void* planesB, int64_t pitch, int sms,
                        cudaStream_t s, bool transA = false, bool transB = false);
// Fused-split preparation, one launch: A's block maxima only (no planes:
// the gemm kernel splits A itself) and B packed as by pack_launch.
cudaError_t pack_fused_launch(Prec prec, const float* A, int64_t M, int64_t K, int64_t lda,
                              const float* B, int64_t N, int64_t ldb, unsigned* amaxA,
                              unsigned* amaxB, unsigned* cntB, void* planesB, int64_t pitch, int sms,
                              cudaStream_t s, int64_t K_b = -1, bool transB = false);
// A row panel of A (rows rows, starting at a 128-row block) packed into the
// planes of the whole matrix at planesA (already offset to the panel's
// first row; plane_stride = elements from one plane to the next).
cudaError_t pack_rows_panel_launch(Prec prec, const float* A, int64_t rows, int64_t K, int64_t lda,
                                   unsigned* amaxA, unsigned* cntA, void* planesA,
                                   int64_t plane_stride, int64_t pitch, int sms, cudaStream_t s);
int pack_first_items(int64_t M, int64_t N, int64_t pitch);
// Packed convolution: split the NHWC image X (elems FP32 values, elems % 4
// == 0, X 16-byte aligned) into bf16 planes [plane][elems], or (interleave,
// BF16 or TF32, C % 16 == 0) one image whose 16-channel groups hold hi then lo,
// under one exponent from its max |x|, folded into amax[0] (zero on entry).
// Two launches.
cudaError_t image_split_launch(Prec prec, const float* X, int64_t elems, unsigned* amax, void* planes,
                               int sms, cudaStream_t s, bool interleave = false);

// ------------------------------------------------------------ grouped
// Static description of one problem of a grouped gemm, device resident
// (written once when the plan is created).  The tensor maps come first: a
// tensor map in global memory must be 64-byte aligned.
struct alignas(128) GroupedProblem {
  CUtensorMap tmA;          // hi/lo planes of A
  CUtensorMap tmB;          // hi/lo planes of B (transposed)
  void* planesA;
  void* planesB;
  unsigned* amaxA;
  unsigned* amaxB;
  unsigned* cntA;           // per block: pack items done
  unsigned* cntB;
  int64_t pitch, lda, ldb, ldc;
  int M, N, K, chunks, tiles_m, tiles_n;
};

// Per-execution values of one problem (rewritten when they change).
struct GroupedPtrs {
  const float* A;
  const float* B;
  float* C;
  float alpha, beta;
};

// One output tile of a grouped launch, precomputed on the host so that a CTA
// finds its next tile with a single 16-byte load.
struct GroupedUnit {
  int prob, tm, tn, chunks;
};

struct GroupedArgs {
  const GroupedProblem* probs;
  const GroupedPtrs* ptrs;
  const GroupedUnit* units;   // num_units entries, problems longest-K first
  int G, num_units, kb, group_m;
  int* err;
  int* unit_ctr;              // units taken so far (zero before the launch)
  unsigned* state;            // per-execution state cleared by the launch's last CTA
  int state_words;            // (followed by its done counter)
};

cudaError_t tc_grouped_launch(int bn, Prec prec, int grid, const GroupedArgs& a, cudaStream_t s);
// Packing of every problem in one launch (items found through the prefix
// sums of pack_first_items); the block maxima and counters must be zero.
cudaError_t grouped_pack_launch(Prec p, const GroupedProblem* probs, const GroupedPtrs* ptrs,
                                const int* first_prefix, int first_total, int G, int sms, cudaStream_t s);

}  // namespace gb
