// Host runtime behind the C ABI (include/gemm.h): argument validation, BLAS
// special cases, per-device state, the candidate tile-configuration table,
// plans (workspace + TMA descriptors), the internal plan cache and the
// host-buffer entry point.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/gemm.h"
#include "internal.h"
#include "runtime.h"

namespace gb {

// ------------------------------------------------------------------ errors
static thread_local std::string t_last_error;

gemm_status fail(gemm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

gemm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(GEMM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void clear_error() { t_last_error.clear(); }

// ------------------------------------------------------------ device state
struct DeviceState {
  bool init = false;
  int sms = 0;
  int cc_major = 0, cc_minor = 0;
  int* err_word = nullptr;
};

static std::mutex g_dev_mutex;
static DeviceState g_devices[64];
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn g_encode = nullptr;
using EncodeIm2colFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const int*, const int*,
                                    cuuint32_t, cuuint32_t, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeIm2colFn g_encode_im2col = nullptr;

gemm_status device_state(DeviceState** out, int* dev_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "device index %d", dev);
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  DeviceState& d = g_devices[dev];
  if (!d.init) {
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
    cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    if ((e = cudaMalloc(&d.err_word, sizeof(int))) != cudaSuccess)
      return fail(GEMM_ERR_ALLOC, "cudaMalloc(error word): %s", cudaGetErrorString(e));
    if ((e = cudaMemset(d.err_word, 0, sizeof(int))) != cudaSuccess)
      return cuda_fail(e, "cudaMemset(error word)");
    d.init = true;
  }
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeTiled entry point not found");
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  if (!g_encode_im2col) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeIm2col", &fn, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && fn)
      g_encode_im2col = reinterpret_cast<EncodeIm2colFn>(fn);
    else
      cudaGetLastError();   // the convolution then stages its patches with cp.async
  }
  *out = &d;
  if (dev_out) *dev_out = dev;
  return GEMM_OK;
}

bool device_has_tcgen05(const DeviceState& d) { return d.cc_major == 10 && d.cc_minor == 3; }

// ------------------------------------------------------ configuration table
// Longest run of k-chunks the tensor core may accumulate in TMEM before the
// epilogue folds the partial sum into FP32 registers.  Measured on GB300 at
// K = 8192: accumulating all 128 chunks in TMEM gives 2.8e-5 (bf16x3) and
// 5.7e-5 (tf32x3) relative Frobenius error, folding every 4 chunks 3.8e-6 and
// 9.2e-7; the extra error grows linearly with the run length.
constexpr int kMaxFoldChunks = 8;

// Candidates of the tensor-core kernels.  The same table serves BF16X3 and
// TF32X3 (the k-chunk is 64 bf16 or 32 tf32 elements, 128 bytes either way):
// ids 0..71 pack both operands and run one CTA per 128 x {128, 64} tile;
// ids 72..143 pack both operands and run a CTA pair per 256 x {256, 128}
// tile; ids 144..215 repeat ids 0..71 with A split inside the gemm kernel.
// BF16X6 has ids 0..143 (its kernels read packed planes of both operands),
// each with a two-deep ring: a stage holds six planes.
static const std::vector<gemm_config>& config_table() {
  static const std::vector<gemm_config> table = [] {
    std::vector<gemm_config> t;
    const int splits[] = {1, 2, 3, 4, 6, 8};
    const int kbs[] = {4, 2, 8};
    const int groups[] = {16, 1};
    // (fused, cluster): packed single CTAs, packed pairs, fused single CTAs
    const int kinds[3][2] = {{0, 1}, {0, 2}, {1, 1}};
    for (const auto& kind : kinds) {
      const int fused = kind[0], cluster = kind[1];
      const int widths[2][2] = {{128, 64}, {256, 128}};
      for (int bn : widths[cluster == 2 ? 1 : 0])
        for (int sk : splits)
          for (int kb : kbs)
            for (int g : groups) {
              gemm_config c;
              c.block_n = bn;
              c.stages = cluster == 2 ? (bn == 256 ? 3 : 4) : fused ? (bn == 64 ? 3 : 2) : (bn == 64 ? 4 : 3);
              c.split_k = sk;
              c.kb = kb;
              c.group_m = g;
              c.fused = fused;
              c.cluster = cluster;
              t.push_back(c);
            }
    }
    return t;
  }();
  return table;
}

int config_count(gemm_mode mode) {
  if (mode == GEMM_MODE_BF16X6) return (int)config_table().size() * 2 / 3;
  return (mode == GEMM_MODE_BF16X3 || mode == GEMM_MODE_TF32X3) ? (int)config_table().size() : 0;
}

bool config_get(int id, gemm_config* out) {
  const auto& t = config_table();
  if (id < 0 || id >= (int)t.size()) return false;
  *out = t[id];
  return true;
}

bool config_get(gemm_mode mode, int id, gemm_config* out) {
  if (id < 0 || id >= config_count(mode) || !config_get(id, out)) return false;
  if (mode == GEMM_MODE_BF16X6) out->stages = 2;
  return true;
}

// The packed configuration with these fields (single CTA or pair).
static int find_config(int bn, int sk, int kb, int g, int cluster = 1) {
  const auto& t = config_table();
  for (int i = 0; i < (int)t.size(); ++i)
    if (t[i].block_n == bn && t[i].split_k == sk && t[i].kb == kb && t[i].group_m == g && !t[i].fused &&
        t[i].cluster == cluster)
      return i;
  return 0;
}

// Built-in tile choice (no tuned table, no trained model): an estimate of
// each packed candidate's time, minimised over tile width (128 x 64 and
// 128 x 128 on one SM, 256 x 256 on a CTA pair) and split-K.  For one
// candidate, with `chunks` 128-byte k-chunks, `per` of them a split and
// `units` = tiles x splits on `slots` (SMs, or SM pairs):
//     waves x (kA0 + per x chunk cost + kEpi) + [splits > 1] (kFix0 + kFix1 x M N splits / 1e6),
// waves = ceil(units / slots).  Chunk costs relative to a 128 x 64 tile's
// (the six-product mode's kSix times as much), per-tile costs in the same
// unit (about a microsecond).  The constants were fitted on GB300 to the autotuner's
// timings (back-to-back executions, C = A B + 0.5 C) of 700 random shapes
// and 21 square ones in each of the three modes, minimising the mean regret
// against the fastest timed configuration (fit_estimate.py); on 103
// held-out shapes the regret is 4.8 % (BF16x3), 6.2 % (TF32x3) and 2.7 %
// (BF16x6), against 11.1 %, 11.4 % and 10.0 % for the previous rule
// (largest one-wave split-K of 128 x 128 tiles, a pair tile when it needs
// fewer waves).  The fold length stays 4 chunks (8 on a
// six-product pair tile, whose single accumulator buffer stalls the MMAs at
// every fold), the raster group 16.
namespace {
constexpr double kChunk64 = 1.0, kChunk128 = 1.5, kChunkPair = 2.0;   // per k-chunk of a unit
constexpr double kEpi64 = 3.3, kEpi128 = 7.2, kEpiPair = 28.8;        // per unit: epilogue
constexpr double kA0 = 3.6;                                           // per unit: prologue
constexpr double kFix0 = 4.0, kFix1 = 0.99;                           // split-K fix-up launch
constexpr double kSix = 1.6;                                          // six products a chunk
}  // namespace

int default_config(gemm_mode mode, int64_t M, int64_t N, int64_t K, int sms) {
  if (config_count(mode) == 0) return -1;
  const Prec p = prec_of_mode(mode);
  const bool six = mode == GEMM_MODE_BF16X6;
  const int64_t chunks = std::max<int64_t>(1, (K + prec_chunk_elems(p) - 1) / prec_chunk_elems(p));
  struct Tile {
    int bn, cluster;
    double chunk, epi;
  };
  const Tile cands[3] = {{64, 1, kChunk64, kEpi64}, {128, 1, kChunk128, kEpi128}, {256, 2, kChunkPair, kEpiPair}};
  const int splits[] = {1, 2, 3, 4, 6, 8};
  double best = 0.0;
  int pick = find_config(64, 1, 4, 16);
  bool have = false;
  for (const Tile& t : cands) {
    if (t.cluster == 2 && sms < 2) continue;
    const int64_t tiles = ((M + 128 * t.cluster - 1) / (128 * t.cluster)) * ((N + t.bn - 1) / t.bn);
    const int64_t slots = std::max(1, sms / t.cluster);
    const double chunk = t.chunk * (six ? kSix : 1.0);
    for (int sk : splits) {
      if (sk > 1 && sk > chunks) break;
      const int64_t per = (chunks + sk - 1) / sk;
      const int64_t splits_eff = (chunks + per - 1) / per;   // (no empty split)
      const int64_t waves = (tiles * splits_eff + slots - 1) / slots;
      double est = (double)waves * (kA0 + (double)per * chunk + t.epi);
      if (splits_eff > 1) est += kFix0 + kFix1 * (double)M * (double)N * (double)splits_eff * 1e-6;
      if (!have || est < best) {
        have = true;
        best = est;
        pick = find_config(t.bn, sk, six && t.cluster == 2 ? 8 : 4, 16, t.cluster);
      }
    }
  }
  return pick;
}

// -------------------------------------------------------------------- plans
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
static gemm_status encode_planes(CUtensorMap* map, Prec p, void* base, int64_t rows, int64_t K,
                                 int64_t pitch, int box_rows, int sw);

gemm_status device_err_word(int** out) {
  DeviceState* d;
  gemm_status st = device_state(&d, nullptr);
  if (st != GEMM_OK) return st;
  *out = d->err_word;
  return GEMM_OK;
}

gemm_status encode_planes_map(CUtensorMap* map, Prec p, void* base, int64_t rows, int64_t K,
                              int64_t pitch, int box_rows, int sw) {
  if (!g_encode) {
    DeviceState* d;
    gemm_status st = device_state(&d, nullptr);
    if (st != GEMM_OK) return st;
  }
  return encode_planes(map, p, base, rows, K, pitch, box_rows, sw);
}

static gemm_status encode_planes(CUtensorMap* map, Prec p, void* base, int64_t rows, int64_t K,
                                 int64_t pitch, int box_rows, int sw) {
  const int es = prec_elem_bytes(p);
  // the box is one k-chunk wide: sw bytes, the swizzle span of the kernel variant
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)prec_planes(p)};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * es), (cuuint64_t)(rows * pitch * es)};
  cuuint32_t box[3] = {(cuuint32_t)(sw / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt =
      prec_bf16(p) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = g_encode(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        sw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) rows=%lld K=%lld pitch=%lld",
                (int)r, (long long)rows, (long long)K, (long long)pitch);
  return GEMM_OK;
}

// FP32 A itself for the fused-split kernel: 128-byte-wide boxes (32 floats)
// of 128 rows, 128-byte swizzle, zero fill outside the matrix.  Needs a
// 16-byte aligned base and lda % 4 == 0.
static gemm_status encode_rows_f32(CUtensorMap* map, const float* A, int64_t M, int64_t K, int64_t lda) {
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)M, 1};
  cuuint64_t strides[2] = {(cuuint64_t)(lda * 4), (cuuint64_t)(M * lda * 4)};
  cuuint32_t box[3] = {32, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(A), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for A, M=%lld K=%lld lda=%lld", (int)r,
                (long long)M, (long long)K, (long long)lda);
  return GEMM_OK;
}

// The patch matrix of an R x S convolution (stride 1, zero padding (R-1)/2
// and (S-1)/2) over the NHWC image X, for TMA's im2col mode: each load
// brings 128 consecutive output pixels (row-major over N, H, W, wrapping
// rows and images) times box_c channels of one filter tap, zero outside the
// image; 128-byte swizzle for 32 channels (128-byte rows), 64-byte swizzle
// for 16 (64-byte rows).  Bounding box corners of -(S-1)/2 (along W) and
// -(R-1)/2 (along H), lower and upper alike, make the starting pixel of
// output (h, w) the input pixel (h - (R-1)/2, w - (S-1)/2) and keep H x W
// starting pixels; the tap adds (r, s).
static gemm_status encode_im2col(CUtensorMap* map, const float* X, int64_t batch, int64_t H, int64_t W,
                                 int64_t C, int R, int S, int box_c) {
  if (!g_encode_im2col) return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "cuTensorMapEncodeIm2col unavailable");
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)batch};
  cuuint64_t strides[3] = {(cuuint64_t)(C * 4), (cuuint64_t)(W * C * 4), (cuuint64_t)(H * W * C * 4)};
  const int lower[2] = {-(S / 2), -(R / 2)}, upper[2] = {-(S / 2), -(R / 2)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode_im2col(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(X), dims, strides,
                               lower, upper, (cuuint32_t)box_c, 128, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               box_c == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeIm2col failed (%d)", (int)r);
  return GEMM_OK;
}

// The same patch matrix over the bf16 planes of a split image (packed
// convolution): the planes are stacked as planes x batch images of H x W x C
// values, and each load brings 128 output pixels times box_c channels of one
// tap: 64 (128-byte rows, 128-byte swizzle) or 16 (32-byte rows, 32-byte
// swizzle); plane z's pixels are images z batch onward, whose zero padding
// TMA supplies image by image.  box_c = 32: the two planes interleaved by
// 16-channel groups, one image of 2C channels, boxes of one group's hi and
// lo (64-byte rows, 64-byte swizzle).
static gemm_status encode_im2col_planes(CUtensorMap* map, Prec prec, const void* planes, int planes_n,
                                        int64_t batch, int64_t H, int64_t W, int64_t C, int R, int S,
                                        int box_c) {
  if (!g_encode_im2col) return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "cuTensorMapEncodeIm2col unavailable");
  const bool ilv = box_c == 32;
  const int64_t Ct = ilv ? 2 * C : C;   // channels of one stacked image
  const int64_t es = prec_elem_bytes(prec);
  const int64_t box_bytes = box_c * es;   // 32, 64 or 128: the swizzle span
  cuuint64_t dims[4] = {(cuuint64_t)Ct, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(ilv ? batch : planes_n * batch)};
  cuuint64_t strides[3] = {(cuuint64_t)(Ct * es), (cuuint64_t)(W * Ct * es), (cuuint64_t)(H * W * Ct * es)};
  const int lower[2] = {-(S / 2), -(R / 2)}, upper[2] = {-(S / 2), -(R / 2)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode_im2col(map, prec_bf16(prec) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               4, const_cast<void*>(planes), dims,
                               strides, lower, upper, (cuuint32_t)box_c, 128, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE,
                               box_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                               : box_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                 : CU_TENSOR_MAP_SWIZZLE_32B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeIm2col failed (%d) for the image planes", (int)r);
  return GEMM_OK;
}

gemm_status validate_shape_t(bool transA, bool transB, int64_t M, int64_t N, int64_t K, int64_t lda,
                             int64_t ldb, int64_t ldc) {
  if (M < 0 || N < 0 || K < 0) return fail(GEMM_ERR_INVALID_ARG, "negative size M=%lld N=%lld K=%lld",
                                           (long long)M, (long long)N, (long long)K);
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX)
    return fail(GEMM_ERR_INVALID_ARG, "size above 2^31-1");
  const int64_t row_a = transA ? M : K, row_b = transB ? K : N;
  if (lda < std::max<int64_t>(row_a, 1))
    return fail(GEMM_ERR_INVALID_ARG, "lda=%lld < max(%s,1)", (long long)lda, transA ? "M" : "K");
  if (ldb < std::max<int64_t>(row_b, 1))
    return fail(GEMM_ERR_INVALID_ARG, "ldb=%lld < max(%s,1)", (long long)ldb, transB ? "K" : "N");
  if (ldc < std::max<int64_t>(N, 1)) return fail(GEMM_ERR_INVALID_ARG, "ldc=%lld < max(N,1)", (long long)ldc);
  return GEMM_OK;
}

gemm_status validate_shape(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc) {
  if (M < 0 || N < 0 || K < 0) return fail(GEMM_ERR_INVALID_ARG, "negative size M=%lld N=%lld K=%lld",
                                           (long long)M, (long long)N, (long long)K);
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX)
    return fail(GEMM_ERR_INVALID_ARG, "size above 2^31-1");
  if (lda < std::max<int64_t>(K, 1)) return fail(GEMM_ERR_INVALID_ARG, "lda=%lld < max(K,1)", (long long)lda);
  if (ldb < std::max<int64_t>(N, 1)) return fail(GEMM_ERR_INVALID_ARG, "ldb=%lld < max(N,1)", (long long)ldb);
  if (ldc < std::max<int64_t>(N, 1)) return fail(GEMM_ERR_INVALID_ARG, "ldc=%lld < max(N,1)", (long long)ldc);
  return GEMM_OK;
}

static gemm_status resolve_mode(gemm_mode mode, const DeviceState& d, gemm_mode* out) {
  if (mode == GEMM_MODE_AUTO) mode = GEMM_MODE_BF16X3;
  if (mode != GEMM_MODE_F32_SIMT && !mode_is_split(mode))
    return fail(GEMM_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
  if (mode != GEMM_MODE_F32_SIMT && !device_has_tcgen05(d))
    return fail(GEMM_ERR_UNSUPPORTED_DEVICE,
                "tensor-core modes need compute capability 10.3 (device is %d.%d)", d.cc_major,
                d.cc_minor);
  *out = mode;
  return GEMM_OK;
}

gemm_status plan_create_impl(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                             gemm_mode mode, int config_id, gemm_select sel, gemm_plan_t* out,
                             bool transA, bool transB, int64_t conv_image_elems, unsigned opts) {
  if (!out) return fail(GEMM_ERR_INVALID_ARG, "null plan output pointer");
  *out = nullptr;
  const bool comp = (opts & GEMM_OPT_COMPENSATED) != 0;
  if (comp && conv_image_elems >= 0)
    return fail(GEMM_ERR_INVALID_ARG, "the compensated epilogue is for gemm plans, not convolutions");
  gemm_status st = validate_shape_t(transA, transB, M, N, K, lda, ldb, ldc);
  if (st != GEMM_OK) return st;
  DeviceState* dev;
  int devidx;
  if ((st = device_state(&dev, &devidx)) != GEMM_OK) return st;
  gemm_mode m;
  if ((st = resolve_mode(mode, *dev, &m)) != GEMM_OK) return st;

  std::unique_ptr<gemm_plan_s, void (*)(gemm_plan_t)> p(new gemm_plan_s(), plan_destroy_impl);
  p->M = M, p->N = N, p->K = K, p->lda = lda, p->ldb = ldb, p->ldc = ldc;
  p->transA = transA, p->transB = transB;
  p->mode = m;
  p->device = devidx;
  p->sms = dev->sms;
  p->err_word = dev->err_word;
  if (m == GEMM_MODE_F32_SIMT || M == 0 || N == 0 || K == 0) {
    p->config_id = -1;
    *out = p.release();
    return GEMM_OK;
  }
  p->prec = prec_of_mode(m);
  if (config_id < 0) {
    config_id = select_config(m, M, N, K, lda, ldb, ldc, sel, dev->sms);
    if (config_id < 0) return fail(GEMM_ERR_INVALID_ARG, "no configuration for mode");
  }
  if (!config_get(m, config_id, &p->cfg))
    return fail(GEMM_ERR_INVALID_ARG, "configuration id %d out of range for mode %d", config_id, (int)m);
  if (transA && p->cfg.fused) {
    // the fused kernel stages rows of A: a transposed A runs as the packed twin
    config_id = find_config(p->cfg.block_n, p->cfg.split_k, p->cfg.kb, p->cfg.group_m);
    config_get(m, config_id, &p->cfg);
  }
  if (comp && (p->cfg.fused || p->cfg.cluster == 2 || p->cfg.block_n != 64)) {
    // the compensated epilogue runs in the single-CTA packed kernel with
    // 128 x 64 tiles: any other configuration runs as that tile with the
    // same split-K and raster group
    config_id = find_config(64, p->cfg.split_k, p->cfg.kb, p->cfg.group_m);
    config_get(m, config_id, &p->cfg);
  }
  if ((opts & kOptNarrowConv) && conv_image_elems >= 0 && !p->cfg.fused && p->cfg.cluster == 1)
    p->cfg.block_n = 32;   // a packed convolution with few output features: 128 x 32 tiles
  const int cluster = p->cfg.cluster == 2 ? 2 : 1;
  if (cluster == 2 && conv_image_elems >= 0)
    return fail(GEMM_ERR_INVALID_ARG, "configuration %d runs on CTA pairs: not for convolutions", config_id);
  p->config_id = config_id;

  const Prec pr = p->prec;
  const int es = prec_elem_bytes(pr);
  p->pitch = packed_k_pitch(pr, K);
  // split-K and the fold length are defined in 128-byte k-chunks; the kernel
  // variant may step in narrower chunks (sw bytes), ratio kc of them per 128
  const int64_t chunks = (K + prec_chunk_elems(pr) - 1) / prec_chunk_elems(pr);
  int sk = std::max(1, std::min<int>(p->cfg.split_k, (int)chunks));
  const int64_t per = (chunks + sk - 1) / sk;
  sk = (int)((chunks + per - 1) / per);   // no empty split
  const int bn = p->cfg.block_n;
  const int sw = tc_chunk_bytes(bn);
  const int kc = 128 / sw;
  const int64_t kchunk = sw / es;                       // elements per kernel chunk
  const int64_t chunks_kernel = (K + kchunk - 1) / kchunk;
  // (a CTA pair's tile is 256 rows high)
  const int64_t tiles_m = (M + 128 * cluster - 1) / (128 * cluster), tiles_n = (N + bn - 1) / bn;

  // workspace: A planes (packed variant) | B planes | amax A | amax B | split-K partials
  const bool fused = p->cfg.fused != 0;
  const int np = prec_planes(pr);
  const bool conv_packed = conv_image_elems >= 0 && !fused;
  const size_t bytesA = fused ? 0
                        : conv_packed ? (size_t)np * conv_image_elems * es
                                      : (size_t)np * M * p->pitch * es;
  const size_t bytesB = (size_t)np * N * p->pitch * es;
  const size_t nblkA = (size_t)(M + kScaleBlock - 1) / kScaleBlock;
  const size_t nblkB = (size_t)(N + kScaleBlock - 1) / kScaleBlock;
  size_t off = 0;
  const size_t offA = off; off = align_up(off + bytesA, 256);
  const size_t offB = off; off = align_up(off + bytesB, 256);
  // per-execution state: maxima and pack counters of both operands, then one
  // unit counter (the packed convolution's dynamic tile order), then the
  // gemm launch's done counter; zeroed once here, and after each execution
  // by the last CTA of its gemm launch
  const int state_words = (int)(2 * (nblkA + nblkB) + 1);
  const size_t offAmax = off; off = align_up(off + (state_words + 1) * sizeof(unsigned), 256);
  const size_t offPart = off;
  if (sk > 1) off = align_up(off + (size_t)sk * M * N * sizeof(float), 256);
  p->ws_bytes = off;
  cudaError_t e = cudaMalloc(&p->ws, p->ws_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "cudaMalloc(%zu bytes) for the plan workspace: %s", p->ws_bytes,
                cudaGetErrorString(e));
  }
  char* w = static_cast<char*>(p->ws);
  p->planesA = fused ? nullptr : w + offA;
  p->planesB = w + offB;
  p->amaxA = reinterpret_cast<unsigned*>(w + offAmax);
  p->amaxB = p->amaxA + nblkA;
  p->amax_bytes = (state_words + 1) * sizeof(unsigned);   // maxima, block counters, unit and done counters
  if ((e = cudaMemset(p->amaxA, 0, p->amax_bytes)) != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMemset(plan state)");
  }
  p->cntA = p->amaxB + nblkB;
  p->cntB = p->cntA + nblkA;
  p->unit_ctr = reinterpret_cast<int*>(p->cntB + nblkB);
  p->partial = sk > 1 ? reinterpret_cast<float*>(w + offPart) : nullptr;

  // (a packed convolution's A map, over the image planes, is made by its creator)
  if (!fused && !conv_packed &&
      (st = encode_planes(&p->tmA, pr, p->planesA, M, K, p->pitch, 128, sw)) != GEMM_OK)
    return st;
  // (each CTA of a pair loads half of the tile's rows of B)
  if ((st = encode_planes(&p->tmB, pr, p->planesB, N, K, p->pitch, bn / cluster, sw)) != GEMM_OK) return st;

  TcArgs& a = p->args;
  a.M = (int)M, a.N = (int)N, a.K = (int)K;
  a.tiles_m = (int)tiles_m, a.tiles_n = (int)tiles_n;
  a.num_tiles = (int)(tiles_m * tiles_n);
  a.split_k = sk;
  a.num_units = a.num_tiles * sk;
  a.chunks_total = (int)chunks_kernel;
  a.chunks_per_split = (int)(per * kc);
  // (the compensated epilogue folds every k-chunk: the tensor core's own
  // accumulation chain is then one chunk long, and the register sum of the
  // folds is compensated)
  a.kb = (comp ? 1 : std::max(1, std::min(p->cfg.kb, kMaxFoldChunks))) * kc;
  // group_m counts 128-row blocks of C, so a raster group spans the same
  // rows of A in both kernels: 16 blocks are 16 single-CTA tile rows or 8
  // CTA-pair tile rows.  (At 8192^3 on pairs, groups of 4, 6, 8, 12, 16
  // and 32 pair rows ran within 2.5 % of one another; of 4, 8 and 16, 8
  // read the least from DRAM: 2.81 GB a launch against 3.46 and 3.17 GB.)
  a.group_m = std::max(1, std::min<int>(p->cfg.group_m / cluster, (int)tiles_m));
  a.ldc = ldc;
  a.amaxA = p->amaxA;
  a.amaxB = p->amaxB;
  a.partial = p->partial;
  a.err = dev->err_word;
  a.lda = lda;
  a.state = p->amaxA;
  a.state_words = state_words;
  p->launch.bn = bn;
  p->launch.prec = pr;
  p->launch.fused = fused;
  p->launch.cluster = cluster;
  p->launch.comp = comp;
  if (cluster == 2) {
    // one cluster per SM pair that can hold one at a time
    if ((e = tc_pair_prepare(bn, pr, &p->max_pairs)) != cudaSuccess) return cuda_fail(e, "pair kernel attribute");
    p->launch.grid = 2 * (int)std::min<int64_t>(a.num_units, p->max_pairs);
  } else {
    const int per_sm = bn == 32 ? tc_narrow_ctas_per_sm(pr) : 1;
    p->launch.grid = (int)std::min<int64_t>(a.num_units, (int64_t)dev->sms * per_sm);
    if ((e = tc_prepare(bn, pr, fused)) != cudaSuccess) return cuda_fail(e, "kernel attribute");
  }
  *out = p.release();
  return GEMM_OK;
}

gemm_status plan_execute_impl(gemm_plan_t p, float alpha, const float* A, const float* B, float beta,
                              float* C, cudaStream_t s) {
  if (!p) return fail(GEMM_ERR_INVALID_ARG, "null plan");
  const int64_t M = p->M, N = p->N, K = p->K;
  if (M == 0 || N == 0) return GEMM_OK;
  if (!C) return fail(GEMM_ERR_INVALID_ARG, "null C");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device)
    return fail(GEMM_ERR_INVALID_ARG, "plan was created on device %d, current device is %d",
                p->device, dev);
  cudaError_t e;
  if (K == 0 || alpha == 0.0f) {
    if ((e = scale_c_launch(M, N, beta, C, p->ldc, s)) != cudaSuccess)
      return cuda_fail(e, "scale_c launch");
    return GEMM_OK;
  }
  if (!A || !B) return fail(GEMM_ERR_INVALID_ARG, "null A or B");
  if (p->mode == GEMM_MODE_F32_SIMT) {
    if ((e = simt_gemm_launch(M, N, K, alpha, A, p->lda, B, p->ldb, beta, C, p->ldc, s, p->transA,
                              p->transB)) != cudaSuccess)
      return cuda_fail(e, "simt gemm launch");
    return GEMM_OK;
  }
  const bool prof = p->prof_n < p->prof_max;
  cudaEvent_t* ev = prof ? &p->prof_events[4 * p->prof_n] : nullptr;
  if (prof) cudaEventRecord(ev[0], s);
  // (the block maxima and counters are zero: the previous execution's gemm
  // launch cleared them)
  if (p->args.conv) {
    // one exponent for the whole image: its max, scanned as a single row
    if (reinterpret_cast<uintptr_t>(A) % 16 != 0)
      return fail(GEMM_ERR_ALIGNMENT, "the convolution's input image must be 16-byte aligned");
    const int64_t elems = (int64_t)p->conv_batch * p->args.conv_H * p->args.conv_W * p->args.conv_C;
    if (!p->launch.fused) {
      // packed: the image split once into planes, then B packed alone
      e = image_split_launch(p->prec, A, elems, p->amaxA, p->planesA, p->sms, s, p->args.conv_box_c == 32);
      if (e == cudaSuccess)
        e = pack_launch(p->prec, nullptr, 0, K, K, B, N, p->ldb, p->amaxA, p->amaxB, p->cntA, p->cntB,
                        nullptr, p->planesB, p->pitch, p->sms, s);
    } else {
      e = pack_fused_launch(p->prec, A, 1, elems, elems, B, N, p->ldb, p->amaxA, p->amaxB, p->cntB,
                            p->planesB, p->pitch, p->sms, s, K);
    }
  } else if (p->launch.fused)
    e = pack_fused_launch(p->prec, A, M, K, p->lda, B, N, p->ldb, p->amaxA, p->amaxB, p->cntB,
                          p->planesB, p->pitch, p->sms, s, -1, p->transB);
  else
    e = pack_launch(p->prec, A, M, K, p->lda, B, N, p->ldb, p->amaxA, p->amaxB, p->cntA, p->cntB,
                    p->planesA, p->planesB, p->pitch, p->sms, s, p->transA, p->transB);
  if (e != cudaSuccess) return cuda_fail(e, "pack launch");
  TcArgs a = p->args;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.A = A;
  a.vecA = (p->lda % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0) ? 1 : 0;
  if (!p->args.conv && !p->launch.fused) {
    // the packing kernel just launched packs both operands and marks each
    // block ready: the gemm's loads of a block may start once it is
    a.readyA = p->cntA;
    a.readyB = p->cntB;
  }
  if (a.conv && p->launch.fused) {
    // TMA im2col staging when C is a multiple of 16: boxes of 32 channels
    // (128-byte rows) when every k-chunk holds whole taps (C a multiple of
    // the chunk, so K = R*S*C has no partial chunk), else boxes of 16
    // (64-byte rows; the kernel variant for them zeroes the part of a last
    // chunk past K); other channel counts are gathered by the split threads
    a.vecA = (g_encode_im2col && a.conv_C % 16 == 0) ? 1 : 0;
    a.conv_box_c = a.conv_C % prec_chunk_elems(p->prec) == 0 ? 32 : 16;
  }
  CUtensorMap tmAf;   // fused variant: A staged by TMA when its rows are 16-byte aligned
  const CUtensorMap* mapA = &p->tmA;
  if (p->launch.fused) {
    std::memset(&tmAf, 0, sizeof tmAf);
    if (a.vecA) {
      gemm_status st = a.conv ? encode_im2col(&tmAf, A, p->conv_batch, a.conv_H, a.conv_W, a.conv_C,
                                              a.conv_R, a.conv_S, a.conv_box_c)
                              : encode_rows_f32(&tmAf, A, M, K, p->lda);
      if (st != GEMM_OK) return st;
    }
    mapA = &tmAf;
  }
  if (prof) cudaEventRecord(ev[1], s);
  if ((e = tc_gemm_launch(p->launch, *mapA, p->tmB, a, s)) != cudaSuccess)
    return cuda_fail(e, "tensor-core gemm launch");
  if (prof) cudaEventRecord(ev[2], s);
  if (a.split_k > 1) {
    if ((e = splitk_reduce_launch(a.M, a.N, a.split_k, a.partial, beta, C, p->ldc, s)) != cudaSuccess)
      return cuda_fail(e, "split-K reduce launch");
  }
  if (prof) {
    cudaEventRecord(ev[3], s);
    ++p->prof_n;
  }
  return GEMM_OK;
}

static void profile_release(gemm_plan_t p) {
  for (cudaEvent_t e : p->prof_events) cudaEventDestroy(e);
  p->prof_events.clear();
  p->prof_max = p->prof_n = 0;
}

void plan_destroy_impl(gemm_plan_t p) {
  if (!p) return;
  profile_release(p);
  if (p->ws) cudaFree(p->ws);
  if (p->last_use) cudaEventDestroy(p->last_use);
  delete p;
}

// --------------------------------------------------------------- plan cache
struct CacheKey {
  int dev;
  int64_t M, N, K, lda, ldb, ldc;
  int mode, sel, trans;
  uintptr_t stream;
  bool operator<(const CacheKey& o) const {
    return std::tie(dev, M, N, K, lda, ldb, ldc, mode, sel, trans, stream) <
           std::tie(o.dev, o.M, o.N, o.K, o.lda, o.ldb, o.ldc, o.mode, o.sel, o.trans, o.stream);
  }
  bool operator==(const CacheKey& o) const { return !(*this < o) && !(o < *this); }
};

static std::mutex g_cache_mutex;
static std::map<CacheKey, gemm_plan_t> g_cache;
static std::list<CacheKey> g_lru;
// Plans the cache has dropped whose last execution may still be queued:
// each is destroyed once its last-use event has completed, found by polling
// (cudaEventQuery) on later cache calls.  Nothing waits on the device, so
// an eviction stalls no stream and is legal next to other streams' captures.
static std::list<gemm_plan_t> g_retired;
constexpr size_t kCacheMax = 16;

// (g_cache_mutex held)
static void reap_retired() {
  for (auto it = g_retired.begin(); it != g_retired.end();) {
    gemm_plan_t p = *it;
    const cudaError_t q = p->last_use ? cudaEventQuery(p->last_use) : cudaSuccess;
    if (q == cudaErrorNotReady) {
      ++it;
      continue;
    }
    if (q != cudaSuccess) cudaGetLastError();   // a sticky fault is reported by the next call
    plan_destroy_impl(p);
    it = g_retired.erase(it);
  }
}

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

gemm_status cached_plan(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                        gemm_mode mode, gemm_select sel, cudaStream_t s, gemm_plan_t* out,
                        bool transA, bool transB) {
  int dev = 0;
  cudaGetDevice(&dev);
  CacheKey key{dev, M, N, K, lda, ldb, ldc, (int)mode, (int)sel, (transA ? 1 : 0) | (transB ? 2 : 0),
               reinterpret_cast<uintptr_t>(s)};
  // (the capture status is read first: while this thread's stream is being
  // captured, no event of an eager execution is queried)
  const bool capturing = stream_capturing(s);
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  if (!capturing) reap_retired();
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    g_lru.remove(key);
    g_lru.push_front(key);
    ++it->second->cache_users;
    *out = it->second;
    return GEMM_OK;
  }
  // a new plan allocates its workspace, and an eviction may free one: neither
  // belongs inside a stream capture
  if (capturing)
    return fail(GEMM_ERR_INVALID_ARG,
                "no cached plan for this shape and stream while the stream is being captured: "
                "call once before the capture, or capture an explicit plan (gemm_plan_create)");
  gemm_plan_t p = nullptr;
  gemm_status st = plan_create_impl(M, N, K, lda, ldb, ldc, mode, -1, sel, &p, transA, transB);
  if (st != GEMM_OK) return st;
  cudaError_t e = cudaEventCreateWithFlags(&p->last_use, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    p->last_use = nullptr;
    plan_destroy_impl(p);
    return cuda_fail(e, "cudaEventCreate");
  }
  if (g_cache.size() >= kCacheMax) {
    const CacheKey victim = g_lru.back();
    g_lru.pop_back();
    gemm_plan_t v = g_cache[victim];
    g_cache.erase(victim);
    if (v->cache_users == 0)
      g_retired.push_back(v);    // destroyed once its last execution has completed
    else
      v->cache_evicted = true;   // another call holds it: its last holder retires it
    reap_retired();
  }
  g_cache[key] = p;
  g_lru.push_front(key);
  ++p->cache_users;
  *out = p;
  return GEMM_OK;
}

// Marks the end of one eager execution of a cached plan on stream s (an
// execution captured into a graph is not tracked: the graph's owner must
// keep the plan alive, which only an explicit plan guarantees).
static void note_use(gemm_plan_t p, cudaStream_t s) {
  if (p && p->last_use && !stream_capturing(s)) cudaEventRecord(p->last_use, s);
}

void release_cached_plan(gemm_plan_t p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  if (--p->cache_users == 0 && p->cache_evicted) g_retired.push_back(p);
}

// Holds a plan of the internal cache for the duration of one call, so that
// another thread's insertion cannot destroy it meanwhile.
struct CachedPlanUse {
  gemm_plan_t p;
  explicit CachedPlanUse(gemm_plan_t plan) : p(plan) {}
  ~CachedPlanUse() { release_cached_plan(p); }
  CachedPlanUse(const CachedPlanUse&) = delete;
  CachedPlanUse& operator=(const CachedPlanUse&) = delete;
};

// ----------------------------------------------------- host-buffer entry
// gemm_f32_host keeps per-thread device copies of A, B, C and two copy
// streams.  Large tensor-core problems are pipelined over row panels of A
// and C: B is copied and packed first, then panel i's copy in (A rows and,
// when beta != 0, C rows) overlaps panel i-1's pack + gemm, which overlaps
// panel i-2's copy of C back to the host.
struct HostBuffers {
  int dev = -1;
  float *A = nullptr, *B = nullptr, *C = nullptr;
  size_t nA = 0, nB = 0, nC = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  std::vector<cudaEvent_t> ev;
  void release() {
    if (A) cudaFree(A);
    if (B) cudaFree(B);
    if (C) cudaFree(C);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (h2d) cudaStreamDestroy(h2d);
    if (d2h) cudaStreamDestroy(d2h);
    A = B = C = nullptr;
    nA = nB = nC = 0;
    ev.clear();
    h2d = d2h = nullptr;
  }
  ~HostBuffers() { release(); }
};
static thread_local HostBuffers t_host;

static gemm_status grow(float** p, size_t* cap, size_t n) {
  if (*cap >= n) return GEMM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, n * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "cudaMalloc(%zu bytes) for host-call buffers", n * sizeof(float));
  }
  *cap = n;
  return GEMM_OK;
}

// rows x cols floats between row-major buffers with leading dimension ld
// (only the logical matrix moves; padding columns are never touched)
static cudaError_t copy_rows(float* dst, const float* src, int64_t rows, int64_t cols, int64_t ld,
                             cudaMemcpyKind kind, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (ld == cols) return cudaMemcpyAsync(dst, src, (size_t)rows * cols * 4, kind, s);
  return cudaMemcpy2DAsync(dst, (size_t)ld * 4, src, (size_t)ld * 4, (size_t)cols * 4, (size_t)rows, kind, s);
}

// Panels of the host-buffer pipeline (GEMM_HOST_PANELS, default 16; 1 turns
// the pipeline off).  On 8192^3 with pinned buffers 1/2/4/8/16/32 panels took
// 7.5/5.7/5.0/4.66/4.53/4.67 ms per call with beta != 0 (4.19/4.25/4.43 ms
// for 8/16/32 with beta = 0).  The host link carries 211 GB/s host to device
// alone but 171 + 170 GB/s with both directions busy, so with beta != 0 the
// floor is about 4.1 ms: the copies back of C panels overlap the copies in.
static int host_panels() {
  static const int n = [] {
    const char* v = std::getenv("GEMM_HOST_PANELS");
    const int x = v ? std::atoi(v) : 16;
    return x < 1 ? 1 : (x > 64 ? 64 : x);
  }();
  return n;
}

// Page-locked (or registered) host memory: only such buffers copy
// asynchronously, so only they gain from the panel pipeline (pageable copies
// are staged by the driver and ran slower with more panels).
static bool page_locked(const void* ptr) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

static gemm_status host_streams(int nevents) {
  cudaError_t e;
  if (!t_host.h2d && (e = cudaStreamCreateWithFlags(&t_host.h2d, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  if (!t_host.d2h && (e = cudaStreamCreateWithFlags(&t_host.d2h, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  while ((int)t_host.ev.size() < nevents) {
    cudaEvent_t x;
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    t_host.ev.push_back(x);
  }
  return GEMM_OK;
}

// Pipelined path: tensor-core plan without split-K, M spanning >= 2 panels.
static gemm_status host_gemm_panels(gemm_plan_t p, float alpha, const float* A, const float* B,
                                    float beta, float* C, cudaStream_t s) {
  const int64_t M = p->M, N = p->N, K = p->K, lda = p->lda, ldb = p->ldb, ldc = p->ldc;
  const int64_t tiles_m = (M + 127) / 128;
  const int npan = (int)std::min<int64_t>(host_panels(), tiles_m);
  // 128-row tiles per panel; even for a CTA-pair plan (its tiles are 256 rows)
  const int64_t cl = p->launch.cluster == 2 ? 2 : 1;
  const int64_t tiles_per = ((tiles_m + npan - 1) / npan + cl - 1) / cl * cl;
  gemm_status st = host_streams(2 + 2 * npan);
  if (st != GEMM_OK) return st;
  cudaEvent_t* ev = t_host.ev.data();
  cudaError_t e;
  // the copies start after whatever the caller queued on s
  if ((e = cudaEventRecord(ev[0], s)) || (e = cudaStreamWaitEvent(t_host.h2d, ev[0], 0)) ||
      (e = cudaStreamWaitEvent(t_host.d2h, ev[0], 0)))
    return cuda_fail(e, "stream ordering");
  if ((e = copy_rows(t_host.B, B, K, N, ldb, cudaMemcpyHostToDevice, t_host.h2d)) ||
      (e = cudaEventRecord(ev[1], t_host.h2d)))
    return cuda_fail(e, "copy B to device");
  for (int i = 0; i < npan; ++i) {   // all panel copies in, queued behind B
    const int64_t r0 = i * tiles_per * 128, r1 = std::min(M, (i + 1) * tiles_per * 128);
    if (r0 >= r1) break;
    if ((e = copy_rows(t_host.A + r0 * lda, A + r0 * lda, r1 - r0, K, lda, cudaMemcpyHostToDevice,
                       t_host.h2d)))
      return cuda_fail(e, "copy A panel to device");
    if (beta != 0.0f && (e = copy_rows(t_host.C + r0 * ldc, C + r0 * ldc, r1 - r0, N, ldc,
                                       cudaMemcpyHostToDevice, t_host.h2d)))
      return cuda_fail(e, "copy C panel to device");
    if ((e = cudaEventRecord(ev[2 + i], t_host.h2d))) return cuda_fail(e, "event");
  }
  // B packed once
  if ((e = cudaStreamWaitEvent(s, ev[1], 0)) ||
      (e = cudaMemsetAsync(p->amaxA, 0, p->amax_bytes, s)) ||
      (e = pack_launch(p->prec, nullptr, 0, K, 1, t_host.B, N, ldb, nullptr, p->amaxB, nullptr,
                       p->cntB, nullptr, p->planesB, p->pitch, p->sms, s)))
    return cuda_fail(e, "pack B");
  for (int i = 0; i < npan; ++i) {
    const int64_t t0 = i * tiles_per, t1 = std::min(tiles_m, (i + 1) * tiles_per);
    if (t0 >= t1) break;
    const int64_t r0 = t0 * 128, r1 = std::min(M, t1 * 128);
    if ((e = cudaStreamWaitEvent(s, ev[2 + i], 0)) ||
        (e = pack_rows_panel_launch(p->prec, t_host.A + r0 * lda, r1 - r0, K, lda, p->amaxA + t0,
                                    p->cntA + t0,
                                    static_cast<char*>(p->planesA) + r0 * p->pitch * prec_elem_bytes(p->prec),
                                    M * p->pitch, p->pitch, p->sms, s)))
      return cuda_fail(e, "pack A panel");
    TcArgs a = p->args;
    a.alpha = alpha;
    a.beta = beta;
    a.C = t_host.C;
    a.tm0 = (int)t0;
    // this panel's blocks of A are packed by the launch just before, B's
    // before the first panel: each is marked ready in its counter
    a.readyA = p->cntA;
    a.readyB = p->cntB;
    // the maxima are read by every panel's gemm: only the last one clears them
    if (t1 < tiles_m) a.state_words = 0;
    a.tiles_m = (int)((t1 - t0 + cl - 1) / cl);   // in the plan's tile height
    a.num_tiles = a.tiles_m * a.tiles_n;
    a.num_units = a.num_tiles;   // split_k == 1
    a.group_m = std::max(1, std::min(a.group_m, a.tiles_m));
    TcLaunch l = p->launch;
    l.grid = cl == 2 ? 2 * std::min(a.num_units, p->max_pairs) : std::min(a.num_units, p->sms);
    if ((e = tc_gemm_launch(l, p->tmA, p->tmB, a, s)) || (e = cudaEventRecord(ev[2 + npan + i], s)) ||
        (e = cudaStreamWaitEvent(t_host.d2h, ev[2 + npan + i], 0)) ||
        (e = copy_rows(C + r0 * ldc, t_host.C + r0 * ldc, r1 - r0, N, ldc, cudaMemcpyDeviceToHost,
                       t_host.d2h)))
      return cuda_fail(e, "panel gemm / copy back");
  }
  if ((e = cudaStreamSynchronize(t_host.d2h)) || (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "synchronize");
  return GEMM_OK;
}

gemm_status host_gemm_impl(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                           const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                           gemm_mode mode, cudaStream_t s) {
  gemm_status st = validate_shape(M, N, K, lda, ldb, ldc);
  if (st != GEMM_OK) return st;
  if (M == 0 || N == 0) return GEMM_OK;
  if (!C || (K > 0 && alpha != 0.0f && (!A || !B))) return fail(GEMM_ERR_INVALID_ARG, "null host pointer");
  int dev = 0;
  cudaGetDevice(&dev);
  if (t_host.dev != dev) {
    t_host.release();
    t_host.dev = dev;
  }
  const bool need_ab = K > 0 && alpha != 0.0f;
  const size_t nA = need_ab ? (size_t)(M - 1) * lda + K : 0;
  const size_t nB = need_ab ? (size_t)(K - 1) * ldb + N : 0;
  const size_t nC = (size_t)(M - 1) * ldc + N;
  if ((st = grow(&t_host.A, &t_host.nA, std::max<size_t>(nA, 1))) != GEMM_OK) return st;
  if ((st = grow(&t_host.B, &t_host.nB, std::max<size_t>(nB, 1))) != GEMM_OK) return st;
  if ((st = grow(&t_host.C, &t_host.nC, nC)) != GEMM_OK) return st;
  gemm_plan_t p = nullptr;
  if ((st = cached_plan(M, N, K, lda, ldb, ldc, mode, GEMM_SELECT_DEFAULT, s, &p, false, false)) != GEMM_OK)
    return st;
  const CachedPlanUse hold(p);
  // (every path below synchronises its streams before returning, so the plan
  // is idle once the call ends; the event still marks its last use on s)
  struct NoteUse {
    gemm_plan_t p;
    cudaStream_t s;
    ~NoteUse() { note_use(p, s); }
  } note{p, s};
  if (need_ab && p->mode != GEMM_MODE_F32_SIMT && p->args.split_k == 1 && !p->launch.fused &&
      host_panels() > 1 &&
      M >= 4 * 128 && page_locked(A) && page_locked(C))
    return host_gemm_panels(p, alpha, A, B, beta, C, s);
  cudaError_t e;
  if (need_ab) {
    if ((e = copy_rows(t_host.A, A, M, K, lda, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "copy A to device");
    if ((e = copy_rows(t_host.B, B, K, N, ldb, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "copy B to device");
  }
  if (beta != 0.0f) {
    if ((e = copy_rows(t_host.C, C, M, N, ldc, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "copy C to device");
  }
  if ((st = plan_execute_impl(p, alpha, t_host.A, t_host.B, beta, t_host.C, s)) != GEMM_OK) return st;
  if ((e = copy_rows(C, t_host.C, M, N, ldc, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "copy C to host");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return GEMM_OK;
}

}  // namespace gb

// =================================================================== C ABI
using namespace gb;

extern "C" {

gemm_status gemm_f32_ex(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                        gemm_mode mode, gemm_select sel, gemm_stream_t stream) {
  clear_error();
  gemm_status st = validate_shape(M, N, K, lda, ldb, ldc);
  if (st != GEMM_OK) return st;
  if (M == 0 || N == 0) return GEMM_OK;
  if (!C || (K > 0 && alpha != 0.0f && (!A || !B))) return fail(GEMM_ERR_INVALID_ARG, "null pointer");
  gemm_plan_t p = nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if ((st = cached_plan(M, N, K, lda, ldb, ldc, mode, sel, s, &p, false, false)) != GEMM_OK) return st;
  const CachedPlanUse hold(p);
  st = plan_execute_impl(p, alpha, A, B, beta, C, s);
  note_use(p, s);
  return st;
}

gemm_status gemm_f32_t(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                       int64_t ldc, gemm_mode mode, gemm_select sel, gemm_stream_t stream) {
  clear_error();
  gemm_status st = validate_shape_t(transA != 0, transB != 0, M, N, K, lda, ldb, ldc);
  if (st != GEMM_OK) return st;
  if (M == 0 || N == 0) return GEMM_OK;
  if (!C || (K > 0 && alpha != 0.0f && (!A || !B))) return fail(GEMM_ERR_INVALID_ARG, "null pointer");
  gemm_plan_t p = nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if ((st = cached_plan(M, N, K, lda, ldb, ldc, mode, sel, s, &p, transA != 0, transB != 0)) != GEMM_OK)
    return st;
  const CachedPlanUse hold(p);
  st = plan_execute_impl(p, alpha, A, B, beta, C, s);
  note_use(p, s);
  return st;
}

gemm_status gemm_plan_create_t(int transA, int transB, int64_t M, int64_t N, int64_t K, int64_t lda,
                               int64_t ldb, int64_t ldc, gemm_mode mode, gemm_select sel,
                               gemm_plan_t* out) {
  clear_error();
  return plan_create_impl(M, N, K, lda, ldb, ldc, mode, -1, sel, out, transA != 0, transB != 0);
}

gemm_status gemm_f32(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                     const float* B, int64_t ldb, float beta, float* C, int64_t ldc) {
  return gemm_f32_ex(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, GEMM_MODE_AUTO,
                     GEMM_SELECT_DEFAULT, nullptr);
}

gemm_status gemm_f32_host(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                          const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                          gemm_mode mode, gemm_stream_t stream) {
  clear_error();
  return host_gemm_impl(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, mode,
                        reinterpret_cast<cudaStream_t>(stream));
}

gemm_status gemm_plan_create(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                             gemm_mode mode, gemm_select sel, gemm_plan_t* out) {
  clear_error();
  return plan_create_impl(M, N, K, lda, ldb, ldc, mode, -1, sel, out);
}

gemm_status gemm_plan_create_opts(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                                  int64_t ldc, gemm_mode mode, gemm_select sel, int config_id,
                                  unsigned opts, gemm_plan_t* out) {
  clear_error();
  if (opts & ~static_cast<unsigned>(GEMM_OPT_COMPENSATED))
    return fail(GEMM_ERR_INVALID_ARG, "unknown plan option bits 0x%x", opts);
  return plan_create_impl(M, N, K, lda, ldb, ldc, mode, config_id < 0 ? -1 : config_id, sel, out, false,
                          false, -1, opts);
}

gemm_status gemm_plan_create_config(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                                    int64_t ldc, gemm_mode mode, int config_id, gemm_plan_t* out) {
  clear_error();
  if (config_id < 0 && mode != GEMM_MODE_F32_SIMT)
    return fail(GEMM_ERR_INVALID_ARG, "negative configuration id");
  return plan_create_impl(M, N, K, lda, ldb, ldc, mode, config_id, GEMM_SELECT_DEFAULT, out);
}

// Largest filter side of the direct convolution (the paper specialises 3x3
// to 11x11); TMA's im2col corners of a 4-D map reach -128.
constexpr int kMaxFilter = 11;

gemm_status gemm_conv_plan_create(int64_t batch, int64_t H, int64_t W, int64_t C, int64_t K, int R,
                                   int S, gemm_mode mode, int config_id, gemm_plan_t* out) {
  clear_error();
  if (!out) return fail(GEMM_ERR_INVALID_ARG, "null plan output pointer");
  *out = nullptr;
  if (batch < 1 || H < 1 || W < 1 || C < 1 || K < 1)
    return fail(GEMM_ERR_INVALID_ARG, "convolution sizes must be positive");
  if (R < 1 || S < 1 || R > kMaxFilter || S > kMaxFilter || R % 2 == 0 || S % 2 == 0)
    return fail(GEMM_ERR_INVALID_ARG, "filter %d x %d: sizes must be odd, 1..%d", R, S, kMaxFilter);
  if (C % 4 != 0) return fail(GEMM_ERR_INVALID_ARG, "input channels C=%lld must be a multiple of 4", (long long)C);
  const int64_t taps = (int64_t)R * S;
  if (H > 65535 || W > 65535 || C > (1 << 20) || batch * H * W > INT32_MAX || taps * C > INT32_MAX)
    return fail(GEMM_ERR_INVALID_ARG, "convolution too large");
  if (mode == GEMM_MODE_AUTO) mode = GEMM_MODE_BF16X3;
  if (mode != GEMM_MODE_BF16X3 && mode != GEMM_MODE_TF32X3 && mode != GEMM_MODE_BF16X6)
    return fail(GEMM_ERR_INVALID_ARG, "the convolution runs in BF16X3, TF32X3 or BF16X6 mode");
  // Packed path (C a multiple of 16): the image is split once into planes
  // and the kernel loads im2col boxes of them.  Fused path (the other
  // cases): the FP32 patches are staged and split inside the kernel, once
  // per tap.
  const bool pack_shape = C % 16 == 0;
  if (mode == GEMM_MODE_BF16X6 && !pack_shape)
    return fail(GEMM_ERR_INVALID_ARG, "the BF16X6 convolution needs C a multiple of 16 (C=%lld)",
                (long long)C);
  const int64_t M = batch * H * W, Kd = taps * C;
  gemm_config c;
  if (config_id >= 0) {
    if (!config_get(mode, config_id, &c))
      return fail(GEMM_ERR_INVALID_ARG, "configuration %d out of range", config_id);
    if (c.cluster == 2)
      return fail(GEMM_ERR_INVALID_ARG, "configuration %d runs on CTA pairs: not for convolutions", config_id);
    if (!c.fused && !pack_shape)
      return fail(GEMM_ERR_INVALID_ARG,
                  "configuration %d is packed: the convolution runs packed only with C a multiple of 16",
                  config_id);
  }
  DeviceState* dev;
  gemm_status st0 = device_state(&dev, nullptr);   // also resolves the tensor-map encoders
  if (st0 != GEMM_OK) return st0;
  const bool can_pack = pack_shape && g_encode_im2col != nullptr;
  if (!can_pack && (mode == GEMM_MODE_BF16X6 || (config_id >= 0 && !c.fused)))
    return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "the packed convolution needs TMA im2col tensor maps");
  const bool default_choice = config_id < 0;
  if (config_id < 0) {
    // default: the gemm heuristic's choice for this shape (tile width by K,
    // split-K when the tiles do not fill the GPU), as its packed or its
    // fused-split twin
    const int guess = default_config(mode, M, K, Kd, dev->sms);
    gemm_config d;
    config_get(mode, guess, &d);
    const bool want_fused = !can_pack;
    for (int id = 0; id < config_count(mode); ++id) {
      config_get(mode, id, &c);
      if ((c.fused != 0) == want_fused && c.cluster == 1 && c.block_n == d.block_n && c.split_k == d.split_k &&
          c.kb == d.kb && c.group_m == d.group_m) {
        config_id = id;
        break;
      }
    }
    if (config_id < 0) return fail(GEMM_ERR_INVALID_ARG, "no configuration for the convolution");
  }
  config_get(mode, config_id, &c);
  const bool packed_conv = !c.fused;
  const int64_t elems = batch * H * W * C;
  // the default plan of a packed convolution with at most 32 output
  // features and no split-K takes the narrow tile (128 x 32, two CTAs a SM)
  const unsigned narrow = default_choice && packed_conv && K <= 32 && c.split_k == 1 ? kOptNarrowConv : 0u;
  gemm_plan_t p = nullptr;
  gemm_status st = plan_create_impl(M, K, Kd, Kd, K, K, mode, config_id, GEMM_SELECT_DEFAULT, &p, false,
                                    false, packed_conv ? elems : -1, narrow);
  if (st != GEMM_OK) return st;
  // packed: channels per im2col box (32: the two planes interleaved by
  // 16-channel groups, the only layout of tf32 planes)
  const Prec pr = prec_of_mode(mode);
  const int box_c = pr == Prec::TF32 ? 32 : C % 64 == 0 ? 64 : prec_planes(pr) == 2 ? 32 : 16;
  if (packed_conv && (st = encode_im2col_planes(&p->tmA, p->prec, p->planesA, prec_planes(p->prec), batch, H,
                                                W, C, R, S, box_c)) != GEMM_OK) {
    plan_destroy_impl(p);
    return st;
  }
  p->conv_batch = (int)batch;
  p->args.conv = 1;
  p->args.conv_N = (int)batch;
  p->args.conv_box_c = packed_conv ? box_c : 0;
  p->args.unit_ctr = packed_conv ? p->unit_ctr : nullptr;
  p->args.conv_H = (int)H;
  p->args.conv_W = (int)W;
  p->args.conv_C = (int)C;
  p->args.conv_R = R;
  p->args.conv_S = S;
  *out = p;
  return GEMM_OK;
}

gemm_status gemm_conv3x3_plan_create(int64_t batch, int64_t H, int64_t W, int64_t C, int64_t K,
                                     gemm_mode mode, int config_id, gemm_plan_t* out) {
  return gemm_conv_plan_create(batch, H, W, C, K, 3, 3, mode, config_id, out);
}

gemm_status gemm_plan_execute(gemm_plan_t plan, float alpha, const float* A, const float* B,
                              float beta, float* C, gemm_stream_t stream) {
  clear_error();
  return plan_execute_impl(plan, alpha, A, B, beta, C, reinterpret_cast<cudaStream_t>(stream));
}

gemm_status gemm_plan_info(gemm_plan_t plan, int* mode, int* config_id, size_t* workspace_bytes) {
  clear_error();
  if (!plan) return fail(GEMM_ERR_INVALID_ARG, "null plan");
  if (mode) *mode = (int)plan->mode;
  if (config_id) *config_id = plan->config_id;
  if (workspace_bytes) *workspace_bytes = plan->ws_bytes;
  return GEMM_OK;
}

gemm_status gemm_plan_destroy(gemm_plan_t plan) {
  clear_error();
  plan_destroy_impl(plan);
  return GEMM_OK;
}

gemm_status gemm_plan_profile(gemm_plan_t plan, int max_records) {
  clear_error();
  if (!plan || max_records < 0) return fail(GEMM_ERR_INVALID_ARG, "bad plan or record count");
  profile_release(plan);
  if (max_records == 0) return GEMM_OK;
  plan->prof_events.resize((size_t)4 * max_records);
  for (auto& e : plan->prof_events) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) {
      e = nullptr;
      profile_release(plan);
      return cuda_fail(r, "cudaEventCreate");
    }
  }
  plan->prof_max = max_records;
  plan->prof_n = 0;
  return GEMM_OK;
}

gemm_status gemm_plan_profile_read(gemm_plan_t plan, int* records, float* pack_ms, float* main_ms,
                                   float* reduce_ms) {
  clear_error();
  if (!plan) return fail(GEMM_ERR_INVALID_ARG, "null plan");
  float tp = 0, tm = 0, tr = 0;
  for (int i = 0; i < plan->prof_n; ++i) {
    cudaEvent_t* ev = &plan->prof_events[4 * i];
    cudaError_t r = cudaEventSynchronize(ev[3]);
    if (r != cudaSuccess) return cuda_fail(r, "cudaEventSynchronize");
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    cudaEventElapsedTime(&c, ev[2], ev[3]);
    tp += a, tm += b, tr += c;
  }
  if (records) *records = plan->prof_n;
  if (pack_ms) *pack_ms = tp;
  if (main_ms) *main_ms = tm;
  if (reduce_ms) *reduce_ms = tr;
  return GEMM_OK;
}

int gemm_config_count(gemm_mode mode) { return config_count(mode); }

gemm_status gemm_config_get(gemm_mode mode, int config_id, gemm_config* out) {
  clear_error();
  if (!out) return fail(GEMM_ERR_INVALID_ARG, "null output");
  if (config_count(mode) == 0) return fail(GEMM_ERR_INVALID_ARG, "mode has no configurations");
  if (!config_get(mode, config_id, out)) return fail(GEMM_ERR_INVALID_ARG, "configuration id out of range");
  return GEMM_OK;
}

int gemm_config_default(gemm_mode mode, int64_t M, int64_t N, int64_t K) {
  int sms = 152;
  DeviceState* d;
  if (device_state(&d, nullptr) == GEMM_OK) sms = d->sms;
  return default_config(mode == GEMM_MODE_AUTO ? GEMM_MODE_BF16X3 : mode, M, N, K, sms);
}

const char* gemm_last_error(void) { return t_last_error.c_str(); }

gemm_status gemm_device_error(void) {
  clear_error();
  DeviceState* d;
  int dev = 0;
  gemm_status st = device_state(&d, &dev);
  if (st != GEMM_OK) return st;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  int v = 0, vn = 0;
  if ((e = cudaMemcpy(&v, d->err_word, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read error word");
  // the allocation-free entry point keeps its own word (it allocates nothing)
  if ((e = noalloc_take_error(dev, &vn)) != cudaSuccess)
    return cuda_fail(e, "read the allocation-free path's error word");
  if (v != 0) {
    cudaMemset(d->err_word, 0, sizeof(int));
    return fail(GEMM_ERR_TIMEOUT, "a kernel abandoned a pipeline wait (error word %d)", v);
  }
  if (vn != 0)
    return fail(GEMM_ERR_TIMEOUT,
                "a kernel of the allocation-free path abandoned a pipeline wait (error word %d)", vn);
  return GEMM_OK;
}

int gemm_device_sm_count(void) {
  DeviceState* d;
  if (device_state(&d, nullptr) != GEMM_OK) return -1;
  return d->sms;
}

gemm_status gemm_split_pack(gemm_mode mode, int transpose, int64_t rows, int64_t cols, const float* X,
                            int64_t ld, void* planes, int64_t pitch, unsigned* amax,
                            gemm_stream_t stream) {
  clear_error();
  if (!mode_is_split(mode))
    return fail(GEMM_ERR_INVALID_ARG, "split_pack needs BF16X3, TF32X3 or BF16X6");
  const Prec p = prec_of_mode(mode);
  if (rows < 0 || cols < 0 || ld < std::max<int64_t>(cols, 1))
    return fail(GEMM_ERR_INVALID_ARG, "bad split_pack shape");
  if (rows == 0 || cols == 0) return GEMM_OK;
  if (!X || !planes || !amax) return fail(GEMM_ERR_INVALID_ARG, "null pointer");
  // K is the row length of the planes: cols of A, rows of B
  const int64_t K = transpose ? rows : cols;
  if (pitch != packed_k_pitch(p, K))
    return fail(GEMM_ERR_INVALID_ARG, "pitch must be %lld", (long long)packed_k_pitch(p, K));
  if (reinterpret_cast<uintptr_t>(planes) % 16)
    return fail(GEMM_ERR_ALIGNMENT, "planes must be 16-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int sms = gemm_device_sm_count();
  if (sms <= 0) return fail(GEMM_ERR_CUDA, "no device");
  cudaError_t e;
  // amax holds the maxima of nblk blocks followed by their nblk counters
  const int64_t nblk = ((transpose ? cols : rows) + kScaleBlock - 1) / kScaleBlock;
  if (!transpose)
    e = pack_launch(p, X, rows, cols, ld, nullptr, 0, 1, amax, nullptr, amax + nblk, nullptr, planes,
                    nullptr, pitch, sms, s);
  else
    e = pack_launch(p, nullptr, 0, rows, 1, X, cols, ld, nullptr, amax, nullptr, amax + nblk, nullptr,
                    planes, pitch, sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "pack launch");
  return GEMM_OK;
}

}  // extern "C"
