// Shared declarations of the autotuner and the cost model.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/gemm.h"
#include "internal.h"

namespace gb {

// A candidate configuration as it behaves on one shape.  group_m is the
// configuration's raster group clamped to the shape's tile rows, a cost-model
// feature (the CTA-pair kernel walks groups of half the configuration's value
// in pair rows); candidates with equal effective fields launch the same
// kernel arguments.
struct EffConfig {
  int bn, split_k, chunks_per_split, kb, group_m, fused, cluster;
  int64_t tiles;
};

EffConfig effective_config(const gemm_config& c, Prec p, int64_t M, int64_t N, int64_t K);
// Candidate ids with pairwise different effective configurations on the shape.
std::vector<int> distinct_configs(gemm_mode mode, int64_t M, int64_t N, int64_t K);
// A tuned shape: sizes and leading dimensions.
struct Shape6 {
  int64_t M, N, K, lda, ldb, ldc;
};
bool table_lookup(gemm_mode mode, const Shape6& sh, int* cid, float* ms);
// One row of an autotuner CSV file (rows without leading dimensions, from
// files written before they were part of a shape, read as tight); 0 if the
// line is not a timing row.
struct TimingRow {
  Shape6 sh;
  int mode, cid;
  float ms;
};
int parse_timing_row(const char* line, TimingRow* r);
// Cost-model argmin over the distinct configurations (GEMM_ERR_INVALID_ARG
// when no model is loaded).
gemm_status costmodel_pick(gemm_mode mode, int64_t M, int64_t N, int64_t K, int* cid, float* ms);

constexpr int kFeatures = 17;
constexpr int kHidden = 64;
// Input features of the cost model for a (shape, configuration) pair.
void costmodel_features(gemm_mode mode, int64_t M, int64_t N, int64_t K, const gemm_config& c,
                        int sms, float* out);

}  // namespace gb
