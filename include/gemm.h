/*
 * gb300-sgemm: C ABI of a GB300 (sm_103a) library for generalized matrix
 * multiplication in FP32 semantics,
 *
 *                 C = alpha * A * B + beta * C
 *
 * the computation the Tiramisu paper (arXiv 1804.10694) uses as its running
 * example and benchmarks as sgemm (Section I; Section VI-A).  The tensor-core
 * modes compute each product as three split-precision tensor-core products
 * (bf16 or tf32 hi/lo parts, FP32 accumulation, per-block power-of-two
 * scaling), or, in BF16X6, as six bf16 products of a three-way split (hi,
 * mid, lo: hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi); the SIMT mode
 * is a plain FP32 CUDA-core kernel.
 *
 * Conventions for every call below:
 *   - Layout: row-major.  A is M x K with lda >= K, B is K x N with ldb >= N,
 *     C is M x N with ldc >= N (leading dimensions in elements).  A and B must
 *     not overlap C.
 *   - Memory: matrix pointers are DEVICE pointers owned by the caller (except
 *     gemm_f32_host); the library never frees them.  Plans own their
 *     workspace (packed operand planes, block exponents, split-K partials,
 *     descriptor tables, CUDA graphs) and release it in *_destroy.
 *   - BLAS special cases: M == 0 or N == 0 is a no-op; K == 0 or alpha == 0
 *     gives C = beta * C without reading A or B; beta == 0 makes C
 *     write-only (NaN/Inf in the old C do not propagate).
 *   - Streams: every compute call is asynchronous and ordered on the given
 *     stream (0 = legacy default stream).  A device fault in a kernel shows up
 *     as GEMM_ERR_CUDA on a later call; a kernel that gave up waiting on
 *     its own pipeline raises the device error word read by
 *     gemm_device_error().
 *   - Errors: no exception crosses the ABI.  Invalid arguments are rejected
 *     with GEMM_ERR_INVALID_ARG before anything is launched.  The text of the
 *     last error of the calling thread is returned by gemm_last_error().
 *   - Threads: calls are thread-safe; a plan must not be executed
 *     concurrently on two streams (its workspace is shared).
 */
#ifndef GB300_SGEMM_GEMM_H
#define GB300_SGEMM_GEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as CUDA's cudaStream_t (a CUstream handle); 0 = default stream. */
typedef struct CUstream_st* gemm_stream_t;

typedef enum {
  GEMM_OK = 0,
  GEMM_ERR_INVALID_ARG = 1,      /* bad size, leading dimension, pointer or handle */
  GEMM_ERR_ALIGNMENT = 2,        /* pointer alignment the call requires is not met */
  GEMM_ERR_ALLOC = 3,            /* device or host allocation failed */
  GEMM_ERR_CUDA = 4,             /* a CUDA runtime/driver call failed */
  GEMM_ERR_UNSUPPORTED_DEVICE = 5, /* tensor-core modes need compute capability 10.3 */
  GEMM_ERR_TIMEOUT = 6,          /* a kernel gave up waiting on its own pipeline */
  GEMM_ERR_IO = 7                /* file could not be read, written or parsed */
} gemm_status;

typedef enum {
  GEMM_MODE_AUTO = 0,     /* BF16X3 on sm_103, else error */
  GEMM_MODE_F32_SIMT = 1, /* plain FP32 CUDA-core kernel (reference form) */
  GEMM_MODE_BF16X3 = 2,   /* split-precision bf16 x3 tensor-core kernel */
  GEMM_MODE_TF32X3 = 3,   /* split-precision tf32 x3 tensor-core kernel */
  GEMM_MODE_BF16X6 = 4    /* three-way bf16 split, six tensor-core products: the
                           * error of an FP32 dot product at about twice the
                           * tensor work of BF16X3; packed operands only */
} gemm_mode;

typedef enum {
  GEMM_SELECT_DEFAULT = 0,    /* built-in heuristic: the candidate of least estimated time */
  GEMM_SELECT_MODEL = 1,      /* argmin of the loaded MLP cost model (else heuristic) */
  GEMM_SELECT_TABLE = 2,      /* loaded autotune table, exact shape match (else heuristic) */
  GEMM_SELECT_EXHAUSTIVE = 3  /* time every candidate now, keep the fastest */
} gemm_select;

/* Plan options (bit flags of gemm_plan_create_opts). */
typedef enum {
  GEMM_OPT_NONE = 0,
  GEMM_OPT_COMPENSATED = 1   /* compensated epilogue: the per-fold partial sums are
                              * added with their rounding errors kept (TwoSum) */
} gemm_option;

typedef struct gemm_plan_s* gemm_plan_t;
typedef struct gemm_grouped_plan_s* gemm_grouped_plan_t;

/* Tile configuration of the tensor-core kernels (one entry of the candidate
 * table that the autotuner and the cost model choose from; the paper tunes
 * tile size and unroll factor, Section VI-A; the table itself is this
 * library's). */
typedef struct {
  int block_n;     /* output tile width */
  int stages;      /* depth of the shared-memory operand ring */
  int split_k;     /* number of K partitions (partials reduced in fixed order) */
  int kb;          /* k-chunks accumulated in tensor memory per epilogue fold (1..8) */
  int group_m;     /* raster: output tiles walked in groups spanning this many
                    * 128-row blocks along M (group_m / 2 CTA-pair tile rows) */
  int fused;       /* 1: A is split inside the gemm kernel (no packed copy of A);
                    *    0: A is packed into hi/lo planes by a separate pass */
  int cluster;     /* CTAs per output tile: 1 (tile 128 x block_n on one SM), or
                    * 2 (tile 256 x block_n on a pair of SMs, one tensor-core
                    * operation over both: tcgen05 cta_group::2) */
} gemm_config;
/* BF16X3 and TF32X3 share one table of 216 entries: ids 0..71 single-CTA
 * packed (block_n 128 or 64), ids 72..143 CTA pairs (block_n 256 or 128,
 * packed), ids 144..215 the fused twins of ids 0..71.  BF16X6 has ids
 * 0..143 (packed and pairs; no fused kernel), each with stages = 2. */

/* ---------------------------------------------------------------- gemm -- */

/* C = alpha*A*B + beta*C on the default stream, mode AUTO, default tiles.
 * Definition: paper Section I.  Plans are created and cached internally per
 * (shape, leading dimensions, mode, stream); the cache holds 16 plans, and a
 * plan it drops is destroyed once its last execution has completed (polled
 * with an event on later calls: no call waits on the device).  Creating or
 * dropping a cached plan allocates or frees device memory, so a call that
 * would do either while its stream is being captured into a graph fails with
 * GEMM_ERR_INVALID_ARG: make the call once before the capture, or capture
 * an explicit plan (gemm_plan_create / gemm_plan_execute), which also keeps
 * the captured workspace alive for as long as the graph needs it. */
gemm_status gemm_f32(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                     const float* B, int64_t ldb, float beta, float* C, int64_t ldc);

/* As gemm_f32 with an explicit mode, tile-selection policy and stream. */
gemm_status gemm_f32_ex(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                        int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                        int64_t ldc, gemm_mode mode, gemm_select sel, gemm_stream_t stream);

/* C = alpha * op(A) op(B) + beta * C with BLAS-style transposes: op(A) is
 * M x K and op(B) is K x N.  transA != 0: A is stored K x M row-major
 * (lda >= M), op(A) = A^T; transB != 0: B is stored N x K (ldb >= K),
 * op(B) = B^T.  The packing pass (tensor-core modes) and the F32_SIMT
 * kernel's tile loads read each layout directly (no transposed copy), so the
 * results are bit-identical to the untransposed call on the transposed
 * matrices; a fused-split configuration chosen for a transposed A runs as
 * its packed twin. */
gemm_status gemm_f32_t(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                       int64_t ldc, gemm_mode mode, gemm_select sel, gemm_stream_t stream);

/* As gemm_f32_ex, but A, B and C are HOST pointers (pageable or pinned): the
 * call copies A, B (and C when beta != 0) to device buffers it keeps per
 * thread, computes, copies C back and synchronizes the stream before
 * returning.  Only the M x N (M x K, K x N) elements are copied; padding
 * beyond a row's length in the host buffers is never written.  With
 * page-locked A and C, at least 512 rows, no split-K and the environment
 * variable GEMM_HOST_PANELS (default 16) above 1, B is copied and packed once
 * and row panels of A and C stream through two copy streams while earlier
 * panels compute. */
gemm_status gemm_f32_host(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                          int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                          int64_t ldc, gemm_mode mode, gemm_stream_t stream);

/* ---------------------------------------------------------------- plans -- */

/* Create a plan for one shape: picks the tile configuration (policy `sel`),
 * allocates the packed-operand workspace and encodes the TMA descriptors.
 * Errors: INVALID_ARG (negative sizes, ld below row length), ALLOC, CUDA,
 * UNSUPPORTED_DEVICE. */
gemm_status gemm_plan_create(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                             int64_t ldc, gemm_mode mode, gemm_select sel, gemm_plan_t* out);

/* Create a plan with an explicit candidate configuration id (see
 * gemm_config_count / gemm_config_get). */
gemm_status gemm_plan_create_config(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                                    int64_t ldc, gemm_mode mode, int config_id, gemm_plan_t* out);

/* As gemm_plan_create (config_id < 0: chosen by `sel`) or
 * gemm_plan_create_config (config_id >= 0), with options.
 * GEMM_OPT_COMPENSATED, the higher-accuracy epilogue of the tensor-core
 * modes: the tensor core accumulates the products of a fold (kb k-chunks) in
 * TMEM, an FP32 sum whose rounding is not to nearest and whose error grows
 * with the fold's length, and the epilogue adds the per-fold partial sums
 * into FP32 registers.  With this option the fold is one k-chunk (the
 * configuration's kb is not used), and every addition of a fold into the
 * registers is an error-free transformation (Knuth's TwoSum: the rounded sum
 * and its exact rounding error); the errors are summed in a second register
 * per output and added back once, so that the sum over the folds carries
 * about one rounding instead of one per fold.  What remains is the error
 * of the split (the operands' low parts, the dropped products) and of the
 * tensor core's sum within one k-chunk.  The option runs the single-CTA
 * packed kernel with 128 x 64 tiles, whose epilogue threads hold each
 * output's sum and error in registers: any other configuration (wider,
 * fused-split or CTA-pair) runs as the 128 x 64 packed tile with the same
 * split-K and raster group, and gemm_plan_info reports that configuration.
 * It has no effect in F32_SIMT mode and is not available for convolutions.  Errors:
 * as gemm_plan_create; INVALID_ARG for unknown option bits.  The paper has
 * no counterpart (it computes in FP32 throughout); this is the
 * higher-accuracy variant of the split-precision method. */
gemm_status gemm_plan_create_opts(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                                  int64_t ldc, gemm_mode mode, gemm_select sel, int config_id,
                                  unsigned opts, gemm_plan_t* out);

/* As gemm_plan_create, with the transposes of gemm_f32_t. */
gemm_status gemm_plan_create_t(int transA, int transB, int64_t M, int64_t N, int64_t K, int64_t lda,
                               int64_t ldb, int64_t ldc, gemm_mode mode, gemm_select sel,
                               gemm_plan_t* out);

/* Direct convolution with an odd R x S filter (1..11 each), stride 1, "same"
 * zero padding pR = (R-1)/2, pS = (S-1)/2 (the paper benchmarks convolutions
 * with filters specialised from 3x3 to 11x11, Section VI), as an implicit
 * gemm: the patch matrix of the image (M = batch*H*W output pixels by R*S*C
 * taps x channels) is never formed.
 *   out[n][h][w][k] = alpha * sum_{r,s,c} in[n][h+r-pR][w+s-pS][c] * f[r][s][c][k]
 *                     + beta * out[n][h][w][k]      (in = 0 outside the image)
 * Execute with gemm_plan_execute(plan, alpha, in, f, beta, out, stream):
 *   in:  NHWC FP32 [batch][H][W][C], channels contiguous, 16-byte aligned;
 *   f:   RSCK FP32 [R][S][C][K] (= the gemm's B, R*S*C x K row-major);
 *   out: NHWC FP32 [batch][H][W][K] (= the gemm's C, ld K).
 * All device memory owned by the caller.  Modes BF16X3, TF32X3, BF16X6
 * (AUTO = BF16X3).  Two paths, chosen by the configuration:
 *   packed (a configuration with fused == 0; C a multiple of 16): each
 *     execution splits the image once into planes in the plan's workspace
 *     (planes x batch*H*W*C values; for BF16X3 with C not a multiple of 64,
 *     and always for TF32X3, the two planes interleaved by 16-channel
 *     groups), and the kernel loads the patch tiles from them by TMA im2col
 *     boxes of one tap (64 channels for BF16X3/BF16X6 when C is a multiple
 *     of 64, else one 16-channel group: its hi and lo together, or one
 *     plane's for BF16X6);
 *   fused-split (fused == 1; BF16X3 and TF32X3, C a multiple of 4): the
 *     kernel stages FP32 patch tiles (TMA im2col boxes of 32 or 16 channels
 *     when C is a multiple of 16, else gathered by its threads) and splits
 *     them itself.
 * config_id < 0 picks the default: packed where it applies (C a multiple of
 * 16; BF16X6 has no fused-split kernel), else fused-split; a default packed
 * plan with at most 32 output features (K <= 32) and no split-K runs
 * 128 x 32 tiles, two CTAs a SM where shared memory holds two.  One power-of-two exponent covers
 * the whole image (its max |x|); B is scaled per 128 output channels as in
 * the gemm.
 * Errors: INVALID_ARG (sizes, filter sizes, C % 4, mode, a packed
 * configuration where the packed path does not apply), ALIGNMENT (at
 * execute: input not 16-byte aligned), ALLOC, CUDA, UNSUPPORTED_DEVICE (no
 * tcgen05, or no im2col tensor maps for a packed plan). */
gemm_status gemm_conv_plan_create(int64_t batch, int64_t H, int64_t W, int64_t C, int64_t K, int R,
                                  int S, gemm_mode mode, int config_id, gemm_plan_t* out);

/* gemm_conv_plan_create with R = S = 3 (zero padding 1). */
gemm_status gemm_conv3x3_plan_create(int64_t batch, int64_t H, int64_t W, int64_t C, int64_t K,
                                     gemm_mode mode, int config_id, gemm_plan_t* out);

/* Run the plan: split/pack of A and B, the gemm kernel, and the split-K
 * reduction when split_k > 1, all on `stream`.  No host synchronization, so
 * the call may be captured into a CUDA graph. */
gemm_status gemm_plan_execute(gemm_plan_t plan, float alpha, const float* A, const float* B,
                              float beta, float* C, gemm_stream_t stream);

/* Resolved mode, configuration id (-1 for SIMT) and workspace bytes. */
gemm_status gemm_plan_info(gemm_plan_t plan, int* mode, int* config_id, size_t* workspace_bytes);

gemm_status gemm_plan_destroy(gemm_plan_t plan);

/* Stage timing with CUDA events recorded on the execution stream: for the
 * next `max_records` executions of a tensor-core plan, events are recorded at
 * the start of packing, around the main gemm kernel and at the end (split-K
 * reduction).  0 turns timing off and frees the events.  Not for use while a
 * stream is being captured into a graph. */
gemm_status gemm_plan_profile(gemm_plan_t plan, int max_records);

/* Waits for the recorded executions and returns their count and the summed
 * milliseconds of packing, main kernel and reduction. */
gemm_status gemm_plan_profile_read(gemm_plan_t plan, int* records, float* pack_ms, float* main_ms,
                                   float* reduce_ms);

/* --------------------------------------------------------- grouped gemm -- */

/* Plan for G independent problems C_g = alpha_g*A_g*B_g + beta_g*C_g with
 * their own shapes and leading dimensions (arrays of G entries, caller's
 * order).  The tensor-core modes run every problem in ONE persistent kernel
 * launch (after one launch that takes all block maxima and one that writes all
 * hi/lo planes); tiles are walked problem by problem, longest K first.  The
 * tile width and TMEM fold length are chosen by `sel`: DEFAULT uses a
 * heuristic (tile width with less padding waste), EXHAUSTIVE times the
 * candidates on synthetic data now (the project's autotuner).  SIMT mode runs
 * one plain FP32 launch per problem.  The plan owns its packed planes,
 * problem tables and CUDA graph. */
gemm_status gemm_grouped_plan_create(int G, const int64_t* M, const int64_t* N, const int64_t* K,
                                     const int64_t* lda, const int64_t* ldb, const int64_t* ldc,
                                     gemm_mode mode, gemm_select sel, gemm_grouped_plan_t* out);

/* As gemm_grouped_plan_create with an explicit tile width (64 or 128) and TMEM
 * fold length kb (1..8). */
gemm_status gemm_grouped_plan_create_config(int G, const int64_t* M, const int64_t* N,
                                            const int64_t* K, const int64_t* lda,
                                            const int64_t* ldb, const int64_t* ldc, gemm_mode mode,
                                            int block_n, int kb, gemm_grouped_plan_t* out);

/* Execute: alpha/beta are HOST arrays of G scalars, A/B/C HOST arrays of G
 * DEVICE pointers (caller's order).  The first call captures the launches
 * into a CUDA graph, later calls replay it; the per-problem pointers and
 * scalars are uploaded (stream-ordered, before the replay) only when they
 * change.  No host synchronisation. */
gemm_status gemm_grouped_execute(gemm_grouped_plan_t plan, const float* alpha, const float* const* A,
                                 const float* const* B, const float* beta, float* const* C,
                                 gemm_stream_t stream);

/* Same computation without the graph: launches directly on `stream`. */
gemm_status gemm_grouped_execute_eager(gemm_grouped_plan_t plan, const float* alpha,
                                       const float* const* A, const float* const* B,
                                       const float* beta, float* const* C, gemm_stream_t stream);

/* Tile width, TMEM fold length, total output tiles, workspace bytes. */
gemm_status gemm_grouped_plan_info(gemm_grouped_plan_t plan, int* block_n, int* kb, int* tiles,
                                   size_t* workspace_bytes);

gemm_status gemm_grouped_plan_destroy(gemm_grouped_plan_t plan);

/* ------------------------------------------------------------ autotuning -- */

/* Autotune (the paper chooses tile sizes by search, Section VI-A; the
 * candidate table and this call are this library's): for each of the G
 * shapes, given as G rows of six numbers (M, N, K, lda, ldb, ldc) in
 * `shapes` (G x 6 int64, row-major; leading dimensions as for gemm_f32_ex),
 * time every distinct candidate configuration of `mode` on synthetic uniform
 * data stored with those leading dimensions: after two warm-ups, `reps`
 * CUDA-event-timed batches of three back-to-back executions (C = A B +
 * 0.5 C), the median time per execution.  Leading dimensions are part of a
 * shape because they select code paths (TMA or cp.async staging of A, float4
 * or staged stores of C).  Appends one CSV row per (shape, configuration) to
 * out_path ("M,N,K,lda,ldb,ldc,mode,config_id,median_ms,block_n,split_k,kb,
 * group_m,fused"; header written to a new file; an existing file must carry
 * that header, else GEMM_ERR_IO; NULL = no file) and records the fastest
 * configuration per shape in the process-wide table used by
 * GEMM_SELECT_TABLE, keyed by all six numbers.  Errors: INVALID_ARG (a bad
 * shape, before anything runs), IO, ALLOC, CUDA.  Synchronises the device. */
gemm_status gemm_autotune(const int64_t* shapes, int G, gemm_mode mode, int reps, const char* out_path);

/* Load timing rows (the CSV above; rows of the earlier 11-column format
 * without leading dimensions are read as tight shapes) into the tuned table. */
gemm_status gemm_autotune_load(const char* path);

/* Fastest configuration and its median time for a shape (sizes and leading
 * dimensions) in the tuned table (GEMM_ERR_INVALID_ARG if it was never
 * tuned). */
gemm_status gemm_autotune_best(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                               gemm_mode mode, int* config_id, float* ms);

/* The configuration id a plan created now would get for this shape under
 * policy `sel` (defined by this library, like the policies themselves):
 * DEFAULT = the built-in heuristic (the packed candidate with the least
 * estimated time: waves of units x (per-unit prologue + k-chunks x chunk cost
 * + epilogue) + the split-K fix-up, constants fitted to this library's
 * autotuner timings on GB300), TABLE = the tuned table's entry for the
 * exact six numbers (else the heuristic), MODEL = the loaded cost model's
 * argmin (runs on the GPU; else the heuristic), EXHAUSTIVE = time every
 * candidate now.  -1 for F32_SIMT or an empty problem.  DEFAULT and TABLE
 * need no device (the heuristic assumes 152 SMs without one). */
gemm_status gemm_select_config(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                               gemm_mode mode, gemm_select sel, int* config_id);

/* ------------------------------------------------------------ cost model -- */

/* Number of input features of the cost model (17).  The cost model, its
 * features and its training are this library's (the learned replacement of
 * the paper's tile-size search, Section VI-A); they have no paper passage of
 * their own. */
int gemm_costmodel_feature_count(void);

/* Features of one (shape, configuration) pair for an `sms`-SM device, written
 * to out[gemm_costmodel_feature_count()]: log2 M, N, K; tile width / 128;
 * log2 split-K; fold length / 8; log2 raster group; log2 tiles; log2(1 +
 * waves); fill of the last wave; padded-work fraction; log2 arithmetic
 * intensity; log2 k-chunks per split; 1 for TF32X3; 1 for a fused
 * configuration; 1 for BF16X6; 1 for a CTA-pair configuration (a 256-row
 * tile on two SMs, whose waves count SM pairs). */
gemm_status gemm_costmodel_features(int64_t M, int64_t N, int64_t K, gemm_mode mode, int config_id,
                                    int sms, float* out);

/* Train the MLP cost model (features -> 64 -> ReLU -> 64 -> ReLU -> 1,
 * predicting normalised log time) on the GPU from autotuner timing rows:
 * `epochs` full-batch Adam steps, weights initialised from `seed`.  The model
 * becomes the process-wide model used by GEMM_SELECT_MODEL and is written to
 * out_model (text; NULL = not saved).  final_loss (optional) receives the
 * training MSE in normalised units. */
gemm_status gemm_costmodel_train(const char* timings_path, int epochs, uint64_t seed,
                                 const char* out_model, float* final_loss);

/* Load a saved cost model (GEMM_ERR_IO if the file is missing or malformed). */
gemm_status gemm_costmodel_load(const char* path);

/* Configuration with the smallest predicted time for a shape (one batched
 * forward pass over the distinct candidates on the GPU) and that time. */
gemm_status gemm_costmodel_predict(int64_t M, int64_t N, int64_t K, gemm_mode mode, int* config_id,
                                   float* pred_ms);

/* The training kernels alone, for checking them: loss and gradient of the MSE
 * at parameters theta (flat layout W1[64][F], b1[64], W2[64][64], b2[64],
 * w3[64], b3; F = gemm_costmodel_feature_count()) over n samples X[n][F] with
 * targets t[n]; HOST pointers, computed on the GPU. */
gemm_status gemm_mlp_loss_grad(int n, const float* theta, const float* X, const float* t, float* loss,
                               float* grad);

/* One Adam update on the GPU of P parameters (HOST arrays updated in place;
 * step counts from 1). */
gemm_status gemm_mlp_adam_step(int P, float* theta, const float* grad, float* m, float* v, int step,
                               float lr, float beta1, float beta2, float eps);

/* --------------------------------------------------- tile configurations -- */

/* Number of candidate configurations for a tensor-core mode (0 for SIMT). */
int gemm_config_count(gemm_mode mode);
gemm_status gemm_config_get(gemm_mode mode, int config_id, gemm_config* out);
/* Heuristic default configuration id for a shape. */
int gemm_config_default(gemm_mode mode, int64_t M, int64_t N, int64_t K);

/* ----------------------------------------------------------- diagnostics -- */

/* Text of the calling thread's last error ("" if none).  Valid until the
 * thread's next library call. */
const char* gemm_last_error(void);

/* Reads and clears the current device's kernel error words (the regular
 * entry points' word and, if it ran on this device, the allocation-free
 * path's own word): GEMM_OK, or GEMM_ERR_TIMEOUT if a kernel abandoned a
 * pipeline wait since the last call.  Synchronizes the device. */
gemm_status gemm_device_error(void);

/* Self-test of failure detection: launches one kernel whose pipeline wait can
 * never complete (an mbarrier nothing arrives on) and checks that the bounded
 * wait gives up after its limit (about 2 s), that the kernel returns, and that
 * the error is reported.  Returns GEMM_ERR_TIMEOUT (the expected outcome) and
 * leaves the device error word cleared; anything else is a failure. */
gemm_status gemm_selftest_wait_timeout(void);

/* Number of streaming multiprocessors of the current device. */
int gemm_device_sm_count(void);

/* The packing stage alone (the paper's "array packing", Section I), exposed
 * so that it can be checked bit for bit: splits the FP32 matrix X (rows x cols,
 * leading dimension ld, device memory) into hi/lo planes
 * planes[2][rows][pitch] (bf16 for BF16X3, tf32 values in 32-bit containers
 * for TF32X3; pitch = cols rounded up to 8 resp. 4; BF16X6 writes three bf16
 * planes hi, mid, lo, planes[3][rows][pitch]) and writes the per-block
 * max |x| bit patterns to amax[0 .. nblk), nblk = ceil(rows/128); blocks
 * outside the safe range are split with their exponent.  `transpose` != 0
 * treats X as a K x N matrix B and writes planes[2][N][pitch], with
 * nblk = ceil(N/128) blocks of 128 columns.  amax must hold 2 * nblk words,
 * zeroed by the caller (the second half counts pack items per block).  All
 * pointers are device pointers. */
gemm_status gemm_split_pack(gemm_mode mode, int transpose, int64_t rows, int64_t cols,
                            const float* X, int64_t ld, void* planes, int64_t pitch,
                            unsigned* amax, gemm_stream_t stream);

/* ------------------------------------------------- allocation-free path -- */

/* C = alpha*A*B + beta*C with the BF16x3 tensor-core kernel, for callers that
 * cannot allocate device memory: for example a thread capturing a stream in a
 * mode where allocation is illegal, a framework whose caching allocator holds
 * (nearly) all of device memory, or a latency-critical path that cannot
 * afford the device synchronisation cudaMalloc/cudaFree may imply.  The paper
 * has no counterpart: it is an interface convenience of this library.
 *
 * The call allocates nothing.  Its scratch (packed hi/lo operand planes,
 * block maxima and per-block pack counters) is a fixed 64 MiB static device
 * array that every GPU which loads this code holds until the process exits;
 * a problem needing more, 4 * (M + N) * roundup(K, 8) bytes plus
 * 8 * (ceil(M/128) + ceil(N/128)) for the maxima and counters (each part
 * rounded up to 256 bytes), is rejected with
 * GEMM_ERR_INVALID_ARG (for square problems the limit is about
 * M = N = K = 2896).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset on a device, do not call this entry point
 * on that device again.  A pipeline wait that gives up in this path's kernel
 * is recorded in its own device error word, read and cleared by
 * gemm_device_error().  All calls share the array and each call
 * overwrites it, so calls that overlap on the GPU (other streams, other host
 * threads) race.  Pointers, layout, special cases and errors are as for
 * gemm_f32_ex; no split-K is used and the call never synchronises. */
gemm_status gemm_f32_bf16x3_noalloc(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                                    int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                                    int64_t ldc, gemm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_SGEMM_GEMM_H */
