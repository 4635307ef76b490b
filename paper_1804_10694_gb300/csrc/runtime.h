// Host-side runtime structures shared by runtime.cpp and the tuning code.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/gemm.h"
#include "internal.h"

// Split precision of a tensor-core mode.
inline gb::Prec prec_of_mode(gemm_mode m) {
  return m == GEMM_MODE_TF32X3 ? gb::Prec::TF32 : m == GEMM_MODE_BF16X6 ? gb::Prec::BF16X6 : gb::Prec::BF16;
}
inline bool mode_is_split(gemm_mode m) {
  return m == GEMM_MODE_BF16X3 || m == GEMM_MODE_TF32X3 || m == GEMM_MODE_BF16X6;
}

struct gemm_plan_s {
  int64_t M = 0, N = 0, K = 0, lda = 0, ldb = 0, ldc = 0;
  bool transA = false, transB = false;   // A stored K x M, B stored N x K
  gemm_mode mode = GEMM_MODE_F32_SIMT;
  int config_id = -1;
  gemm_config cfg{};
  int device = 0;
  int sms = 0;
  int* err_word = nullptr;
  gb::Prec prec = gb::Prec::F32;
  int64_t pitch = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* planesA = nullptr;
  void* planesB = nullptr;
  unsigned* amaxA = nullptr;
  unsigned* amaxB = nullptr;
  size_t amax_bytes = 0;            // block maxima of A and B, then their pack counters
  unsigned* cntA = nullptr;
  unsigned* cntB = nullptr;
  int* unit_ctr = nullptr;          // after the counters: the packed convolution's unit counter
  int conv_batch = 0;               // direct convolution plans (args.conv): images per call
  float* partial = nullptr;
  CUtensorMap tmA{}, tmB{};
  gb::TcArgs args{};
  gb::TcLaunch launch{};
  int max_pairs = 0;                // CTA-pair plans: clusters resident at once
  // stage timing (gemm_plan_profile): four events per recorded execution,
  // at the start of packing, before and after the main kernel, at the end
  int prof_max = 0, prof_n = 0;
  std::vector<cudaEvent_t> prof_events;
  // internal plan cache (guarded by its mutex): calls holding the plan,
  // whether the cache has dropped it (the last holder then retires it), and
  // an event recorded on the plan's stream after each of its executions (a
  // retired plan is destroyed once that event has completed)
  int cache_users = 0;
  bool cache_evicted = false;
  cudaEvent_t last_use = nullptr;
};

namespace gb {

gemm_status fail(gemm_status st, const char* fmt, ...);
gemm_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
gemm_status validate_shape_t(bool transA, bool transB, int64_t M, int64_t N, int64_t K, int64_t lda,
                             int64_t ldb, int64_t ldc);
gemm_status validate_shape(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc);

int config_count(gemm_mode mode);
bool config_get(int id, gemm_config* out);
// The entry as it applies to a mode (false when the id is not one of the mode's).
bool config_get(gemm_mode mode, int id, gemm_config* out);
int default_config(gemm_mode mode, int64_t M, int64_t N, int64_t K, int sms);
// Configuration for a new plan under a selection policy (tuning code).
int select_config(gemm_mode mode, int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                  int64_t ldc, gemm_select sel, int sms);

// Internal plan option (beside the public GEMM_OPT_* bits): a packed
// convolution plan runs 128 x 32 tiles, two CTAs a SM.
constexpr unsigned kOptNarrowConv = 1u << 16;

// conv_image_elems >= 0: a packed convolution, whose A planes hold the
// split image (that many elements a plane) instead of M x pitch rows
gemm_status plan_create_impl(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                             gemm_mode mode, int config_id, gemm_select sel, gemm_plan_t* out,
                             bool transA = false, bool transB = false,
                             int64_t conv_image_elems = -1, unsigned opts = 0);
gemm_status plan_execute_impl(gemm_plan_t p, float alpha, const float* A, const float* B, float beta,
                              float* C, cudaStream_t s);
void plan_destroy_impl(gemm_plan_t p);

// The current device's kernel error word (allocated on first use).
gemm_status device_err_word(int** out);
// Reads and clears the allocation-free path's kernel error word of device
// `dev`, which must be the current device (value 0 if that path never ran
// there).  Allocates nothing.
cudaError_t noalloc_take_error(int dev, int* value);
// 3-D tensor map over hi/lo planes [2][rows][pitch] with box {sw bytes of K,
// box_rows, 1} and the sw-byte swizzle (128 or 64).
gemm_status encode_planes_map(CUtensorMap* map, Prec p, void* base, int64_t rows, int64_t K,
                              int64_t pitch, int box_rows, int sw);

// Grouped plans (grouped.cpp) and their tuning (autotune.cpp).
gemm_status grouped_create_impl(int G, const int64_t* M, const int64_t* N, const int64_t* K,
                                const int64_t* lda, const int64_t* ldb, const int64_t* ldc,
                                gemm_mode mode, int bn_override, int kb_override,
                                gemm_grouped_plan_t* out);
gemm_status grouped_execute_impl(gemm_grouped_plan_t p, const float* alpha, const float* const* A,
                                 const float* const* B, const float* beta, float* const* C,
                                 cudaStream_t s, bool use_graph);
void grouped_destroy_impl(gemm_grouped_plan_t p);
gemm_status grouped_tune_and_create(int G, const int64_t* M, const int64_t* N, const int64_t* K,
                                    const int64_t* lda, const int64_t* ldb, const int64_t* ldc,
                                    gemm_mode mode, gemm_grouped_plan_t* out);

// Uniform[-1, 1) fill from a counter-based hash (timing inputs of the tuner).
cudaError_t fill_uniform_launch(float* x, size_t n, uint64_t seed, cudaStream_t s);

}  // namespace gb
