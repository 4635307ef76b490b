// gemm_f32_bf16x3_noalloc: the split-precision BF16x3 gemm for callers that
// cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- a host thread that is
// capturing a stream into a CUDA graph in a mode where allocation is illegal,
// a framework whose caching allocator already owns (nearly) all of device
// memory so that a library allocation fails or fragments it, a
// latency-critical path that cannot afford the implicit device
// synchronisation cudaMalloc/cudaFree may cause, or a plug-in host that only
// hands out input and output buffers.  The regular entry points keep their
// packed-operand workspace in plans, which they allocate.
//
// This path instead keeps its scratch (the hi/lo operand planes and the block
// maxima) in one file-scope __device__ array of fixed size.  The array is
// static device storage: every GPU whose context loads this module holds it
// until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device (with that device
// current) asks the runtime for the address with cudaGetSymbolAddress and
// keeps it; that first call should therefore come before any stream capture.
// The kept address belongs to the device's context as it was then: after a
// cudaDeviceReset (or any re-creation of the primary context) it is stale,
// so this path must not be called on that device again in the process.
// A pipeline wait that gives up in this path's gemm kernel is recorded in
// this path's own error word, which gemm_device_error() reads and clears.
// All calls share the one array and each call overwrites it (the block
// maxima are cleared at the start of every call): calls whose work overlaps
// on the GPU -- two streams, or two host threads -- race on it.
//
// The kernels are the library's regular split/pack and tensor-core kernels,
// launched with tile 128 x {64,128}, no split-K and a TMEM fold every 4
// k-chunks.  The call never synchronises.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/gemm.h"
#include "internal.h"
#include "runtime.h"

namespace gb {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB

// The scratch array and this path's own pipeline-timeout word.  The call
// never synchronises, so it never reads the word itself: gemm_device_error()
// reads and clears it (through noalloc_take_error below) together with the
// regular entry points' word.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ int g_noalloc_error_word;

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct NoAllocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch
  int* err = nullptr;                 // device address of g_noalloc_error_word
  int sms = 0;
  bool tcgen05 = false;
};

std::mutex g_mu;
NoAllocDevice g_dev[64];
EncodeFn g_encode_fn = nullptr;

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

gemm_status setup(int dev, NoAllocDevice** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDevice& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    void* w = nullptr;
    e = cudaGetSymbolAddress(&w, g_noalloc_error_word);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(error word)");
    int major = 0, minor = 0;
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "cudaDeviceGetAttribute");
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (!g_encode_fn) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeTiled entry point not found");
      g_encode_fn = reinterpret_cast<EncodeFn>(fn);
    }
    d.scratch = static_cast<unsigned char*>(p);
    d.err = static_cast<int*>(w);
    d.tcgen05 = major == 10 && minor == 3;
    d.ready = true;
  }
  *out = &d;
  return GEMM_OK;
}

gemm_status encode(CUtensorMap* map, void* base, int64_t rows, int64_t K, int64_t pitch, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, 2};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * 2), (cuuint64_t)(rows * pitch * 2)};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode_fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(GEMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GEMM_OK;
}

}  // namespace

cudaError_t noalloc_take_error(int dev, int* value) {
  *value = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64 || !g_dev[dev].ready) return cudaSuccess;   // never ran here
  }
  // copies to and from the symbol of the current device: nothing is allocated
  cudaError_t e = cudaMemcpyFromSymbol(value, g_noalloc_error_word, sizeof(int));
  if (e == cudaSuccess && *value != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_noalloc_error_word, &zero, sizeof(int));
  }
  return e;
}

}  // namespace gb

using namespace gb;

extern "C" gemm_status gemm_f32_bf16x3_noalloc(int64_t M, int64_t N, int64_t K, float alpha,
                                               const float* A, int64_t lda, const float* B,
                                               int64_t ldb, float beta, float* C, int64_t ldc,
                                               gemm_stream_t stream) {
  clear_error();
  gemm_status st = validate_shape(M, N, K, lda, ldb, ldc);
  if (st != GEMM_OK) return st;
  if (M == 0 || N == 0) return GEMM_OK;
  if (!C || (K > 0 && alpha != 0.0f && (!A || !B))) return fail(GEMM_ERR_INVALID_ARG, "null pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (K == 0 || alpha == 0.0f) {
    if ((e = scale_c_launch(M, N, beta, C, ldc, s)) != cudaSuccess) return cuda_fail(e, "scale_c launch");
    return GEMM_OK;
  }

  // scratch layout: A planes | B planes | block maxima of A | of B
  const int64_t pitch = packed_k_pitch(Prec::BF16, K);
  const size_t bytesA = round256((size_t)2 * M * pitch * 2);
  const size_t bytesB = round256((size_t)2 * N * pitch * 2);
  const size_t nblkA = (size_t)(M + kScaleBlock - 1) / kScaleBlock;
  const size_t nblkB = (size_t)(N + kScaleBlock - 1) / kScaleBlock;
  const size_t bytesAmax = 2 * (nblkA + nblkB) * sizeof(unsigned);   // maxima, then pack counters
  const size_t need = bytesA + bytesB + round256(bytesAmax);
  if (need > kNoAllocScratchBytes)
    return fail(GEMM_ERR_INVALID_ARG,
                "M=%lld N=%lld K=%lld needs %zu bytes of scratch; this entry point has a fixed "
                "maximum of %zu bytes (4*(M+N)*roundup(K,8) plus block maxima)",
                (long long)M, (long long)N, (long long)K, need, kNoAllocScratchBytes);

  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "device index %d", dev);
  NoAllocDevice* d = nullptr;
  if ((st = setup(dev, &d)) != GEMM_OK) return st;
  if (!d->tcgen05)
    return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "the BF16x3 kernel needs compute capability 10.3");

  unsigned char* planesA = d->scratch;
  unsigned char* planesB = planesA + bytesA;
  unsigned* amaxA = reinterpret_cast<unsigned*>(planesB + bytesB);
  unsigned* amaxB = amaxA + nblkA;

  if ((e = cudaMemsetAsync(amaxA, 0, bytesAmax, s)) != cudaSuccess) return cuda_fail(e, "clear block maxima");
  unsigned* cntA = amaxB + nblkB;
  if ((e = pack_launch(Prec::BF16, A, M, K, lda, B, N, ldb, amaxA, amaxB, cntA, cntA + nblkA, planesA,
                       planesB, pitch, d->sms, s)) != cudaSuccess)
    return cuda_fail(e, "pack");

  const int bn = N <= 64 ? 64 : 128;
  CUtensorMap tmA, tmB;
  if ((st = encode(&tmA, planesA, M, K, pitch, 128)) != GEMM_OK) return st;
  if ((st = encode(&tmB, planesB, N, K, pitch, bn)) != GEMM_OK) return st;

  TcArgs a{};
  a.M = (int)M, a.N = (int)N, a.K = (int)K;
  a.tiles_m = (int)((M + 127) / 128);
  a.tiles_n = (int)((N + bn - 1) / bn);
  a.num_tiles = a.tiles_m * a.tiles_n;
  a.split_k = 1;
  a.num_units = a.num_tiles;
  a.chunks_total = (int)((K + 63) / 64);
  a.chunks_per_split = a.chunks_total;
  a.kb = 4;
  a.group_m = std::min(16, a.tiles_m);
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.amaxA = amaxA;
  a.amaxB = amaxB;
  a.partial = nullptr;
  a.err = d->err;
  TcLaunch l{};
  l.bn = bn;
  l.prec = Prec::BF16;
  l.grid = std::min(a.num_units, d->sms);
  if ((e = tc_gemm_launch(l, tmA, tmB, a, s)) != cudaSuccess) return cuda_fail(e, "tensor-core gemm launch");
  return GEMM_OK;
}
