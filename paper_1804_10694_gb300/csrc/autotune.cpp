// Autotuner and tile-configuration selection.  The paper autotunes the tile
// size and unroll factor of its sgemm for the machine it runs on (Section
// VI-A); here the tuned quantities are the tensor-core kernels' tile width,
// split-K, TMEM fold length and raster grouping.  For each shape every
// DISTINCT effective configuration (candidates that behave identically on the
// shape, e.g. split-K above the number of k-chunks, are timed once) is run
// after two warm-up executions in `reps` timed batches of three back-to-back
// executions (C = A B + 0.5 C), each batch between two CUDA events; the
// median time per execution is recorded.  Back to back, as a caller's loop
// runs them, each execution's launches overlap the end of the previous one
// (programmatic launches), which an event between executions would prevent:
// the fixed cost of a split-K fix-up launch, for one, is then what a loop of
// calls pays.  A shape is (M, N, K) with its leading
// dimensions (lda, ldb, ldc): they choose code paths (TMA or cp.async
// staging of A in the fused kernel, float4 or staged stores of C), so they
// are part of what is tuned.  Results are appended to a CSV file
// ("M,N,K,lda,ldb,ldc,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused")
// that the cost model trains on, and the fastest configuration per shape is
// kept in an in-memory table (GEMM_SELECT_TABLE), keyed by all six numbers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/gemm.h"
#include "internal.h"
#include "runtime.h"
#include "tuning.h"

namespace gb {

// --------------------------------------------------------- effective config
EffConfig effective_config(const gemm_config& c, Prec p, int64_t M, int64_t N, int64_t K) {
  EffConfig e;
  const int64_t chunks = std::max<int64_t>(1, (K + prec_chunk_elems(p) - 1) / prec_chunk_elems(p));
  int sk = (int)std::max<int64_t>(1, std::min<int64_t>(c.split_k, chunks));
  const int64_t per = (chunks + sk - 1) / sk;
  sk = (int)((chunks + per - 1) / per);
  const int cl = c.cluster == 2 ? 2 : 1;
  const int64_t tiles_m = (M + 128 * cl - 1) / (128 * cl);   // a CTA pair's tile is 256 rows
  e.bn = c.block_n;
  e.cluster = cl;
  e.split_k = sk;
  e.chunks_per_split = (int)per;
  e.kb = (int)std::min<int64_t>(c.kb, per);
  e.group_m = (int)std::max<int64_t>(1, std::min<int64_t>(c.group_m, tiles_m));
  e.tiles = tiles_m * ((N + c.block_n - 1) / c.block_n);
  e.fused = c.fused;
  return e;
}

std::vector<int> distinct_configs(gemm_mode mode, int64_t M, int64_t N, int64_t K) {
  std::vector<int> out;
  std::set<std::tuple<int, int, int, int, int, int>> seen;
  const Prec p = prec_of_mode(mode);
  gemm_config c;
  for (int id = 0; id < config_count(mode); ++id) {
    config_get(id, &c);
    const EffConfig e = effective_config(c, p, M, N, K);
    if (seen.insert(std::make_tuple(e.bn, e.split_k, e.kb, e.group_m, e.fused, e.cluster)).second)
      out.push_back(id);
  }
  return out;
}

// -------------------------------------------------------------- tuned table
namespace {
using TableKey = std::tuple<int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t>;
std::mutex g_table_mu;
std::map<TableKey, std::pair<int, float>> g_table;

void table_offer(gemm_mode mode, const Shape6& sh, int cid, float ms) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  const TableKey key = std::make_tuple((int)mode, sh.M, sh.N, sh.K, sh.lda, sh.ldb, sh.ldc);
  auto it = g_table.find(key);
  if (it == g_table.end() || ms < it->second.second) g_table[key] = {cid, ms};
}
}  // namespace

bool table_lookup(gemm_mode mode, const Shape6& sh, int* cid, float* ms) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto it = g_table.find(std::make_tuple((int)mode, sh.M, sh.N, sh.K, sh.lda, sh.ldb, sh.ldc));
  if (it == g_table.end()) return false;
  if (cid) *cid = it->second.first;
  if (ms) *ms = it->second.second;
  return true;
}

int parse_timing_row(const char* line, TimingRow* r) {
  int commas = 0;
  for (const char* c = line; *c; ++c) commas += *c == ',';
  long long M, N, K, lda, ldb, ldc;
  if (commas >= 13) {
    if (std::sscanf(line, "%lld,%lld,%lld,%lld,%lld,%lld,%d,%d,%f", &M, &N, &K, &lda, &ldb, &ldc,
                    &r->mode, &r->cid, &r->ms) != 9)
      return 0;
  } else if (commas == 10) {
    // rows written before leading dimensions were part of a shape: tight
    if (std::sscanf(line, "%lld,%lld,%lld,%d,%d,%f", &M, &N, &K, &r->mode, &r->cid, &r->ms) != 6) return 0;
    lda = K, ldb = N, ldc = N;
  } else {
    return 0;
  }
  r->sh = Shape6{M, N, K, lda, ldb, ldc};
  return 1;
}

// ------------------------------------------------------------------- timing
// Median time of `reps` executions of a plan with the given configuration.
gemm_status time_config(const Shape6& sh, gemm_mode mode, int cid, const float* A, const float* B,
                        float* C, int reps, float* median_ms) {
  gemm_plan_t p = nullptr;
  gemm_status st = plan_create_impl(sh.M, sh.N, sh.K, sh.lda, sh.ldb, sh.ldc, mode, cid,
                                    GEMM_SELECT_DEFAULT, &p);
  if (st != GEMM_OK) return st;
  reps = std::max(1, reps);
  std::vector<cudaEvent_t> ev(2 * reps, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) break;
  if (e == cudaSuccess) {
    constexpr int kBatch = 3;
    for (int w = 0; w < 2 && st == GEMM_OK; ++w) st = plan_execute_impl(p, 1.0f, A, B, 0.5f, C, nullptr);
    for (int r = 0; r < reps && st == GEMM_OK; ++r) {
      cudaEventRecord(ev[2 * r], nullptr);
      for (int b = 0; b < kBatch && st == GEMM_OK; ++b) st = plan_execute_impl(p, 1.0f, A, B, 0.5f, C, nullptr);
      cudaEventRecord(ev[2 * r + 1], nullptr);
    }
    if (st == GEMM_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) st = cuda_fail(e, "tuning run");
    if (st == GEMM_OK) {
      std::vector<float> t(reps);
      for (int r = 0; r < reps; ++r) {
        cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]);
        t[r] /= kBatch;
      }
      std::sort(t.begin(), t.end());
      *median_ms = reps % 2 ? t[reps / 2] : 0.5f * (t[reps / 2 - 1] + t[reps / 2]);
    }
  } else {
    st = cuda_fail(e, "cudaEventCreate");
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  plan_destroy_impl(p);
  return st;
}

namespace {

struct DeviceInputs {
  float *A = nullptr, *B = nullptr, *C = nullptr;
  ~DeviceInputs() {
    if (A) cudaFree(A);
    if (B) cudaFree(B);
    if (C) cudaFree(C);
  }
};

gemm_status make_inputs(const Shape6& sh, uint64_t seed, DeviceInputs* in) {
  // storage of row-major matrices with leading dimensions: (rows - 1) * ld + cols
  const size_t na = (size_t)std::max<int64_t>((sh.M - 1) * sh.lda + sh.K, 1);
  const size_t nb = (size_t)std::max<int64_t>((sh.K - 1) * sh.ldb + sh.N, 1);
  const size_t nc = (size_t)std::max<int64_t>((sh.M - 1) * sh.ldc + sh.N, 1);
  cudaError_t e;
  if ((e = cudaMalloc(&in->A, na * 4)) != cudaSuccess || (e = cudaMalloc(&in->B, nb * 4)) != cudaSuccess ||
      (e = cudaMalloc(&in->C, nc * 4)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "tuning inputs for %lldx%lldx%lld do not fit", (long long)sh.M,
                (long long)sh.N, (long long)sh.K);
  }
  if ((e = fill_uniform_launch(in->A, na, seed, nullptr)) != cudaSuccess ||
      (e = fill_uniform_launch(in->B, nb, seed + 1, nullptr)) != cudaSuccess ||
      (e = fill_uniform_launch(in->C, nc, seed + 2, nullptr)) != cudaSuccess)
    return cuda_fail(e, "fill tuning inputs");
  return GEMM_OK;
}

}  // namespace

// Time every distinct configuration of one shape; calls `row` for each.
template <class RowFn>
gemm_status tune_shape(const Shape6& sh, gemm_mode mode, int reps, RowFn row, int* best_cid,
                       float* best_ms) {
  DeviceInputs in;
  gemm_status st = make_inputs(sh, 0x5EEDull + (uint64_t)(sh.M * 31 + sh.N * 17 + sh.K), &in);
  if (st != GEMM_OK) return st;
  *best_cid = -1;
  *best_ms = 0.0f;
  for (int cid : distinct_configs(mode, sh.M, sh.N, sh.K)) {
    float ms = 0.0f;
    st = time_config(sh, mode, cid, in.A, in.B, in.C, reps, &ms);
    if (st != GEMM_OK) return st;
    row(cid, ms);
    table_offer(mode, sh, cid, ms);
    if (*best_cid < 0 || ms < *best_ms) *best_cid = cid, *best_ms = ms;
  }
  return GEMM_OK;
}

int select_config(gemm_mode mode, int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                  int64_t ldc, gemm_select sel, int sms) {
  const Shape6 sh{M, N, K, lda, ldb, ldc};
  int cid = -1;
  float ms = 0.0f;
  switch (sel) {
    case GEMM_SELECT_TABLE:
      if (table_lookup(mode, sh, &cid, &ms)) return cid;
      break;
    case GEMM_SELECT_MODEL:
      if (costmodel_pick(mode, M, N, K, &cid, &ms) == GEMM_OK && cid >= 0) return cid;
      break;
    case GEMM_SELECT_EXHAUSTIVE: {
      if (tune_shape(sh, mode, 5, [](int, float) {}, &cid, &ms) == GEMM_OK && cid >= 0) return cid;
      break;
    }
    default:
      break;
  }
  return default_config(mode, M, N, K, sms);
}

gemm_status grouped_tune_and_create(int G, const int64_t* M, const int64_t* N, const int64_t* K,
                                    const int64_t* lda, const int64_t* ldb, const int64_t* ldc,
                                    gemm_mode mode, gemm_grouped_plan_t* out) {
  // one buffer per operand kind holding every problem, uniform[-1, 1) data
  size_t na = 0, nb = 0, nc = 0;
  std::vector<size_t> oa(G), ob(G), oc(G);
  for (int i = 0; i < G; ++i) {
    oa[i] = na, ob[i] = nb, oc[i] = nc;
    na += (size_t)(M[i] > 0 ? (M[i] - 1) * lda[i] + K[i] : 0) + 64;
    nb += (size_t)(K[i] > 0 ? (K[i] - 1) * ldb[i] + N[i] : 0) + 64;
    nc += (size_t)(M[i] > 0 ? (M[i] - 1) * ldc[i] + N[i] : 0) + 64;
    na = (na + 3) / 4 * 4, nb = (nb + 3) / 4 * 4, nc = (nc + 3) / 4 * 4;
  }
  DeviceInputs in;
  cudaError_t e;
  if ((e = cudaMalloc(&in.A, na * 4)) != cudaSuccess || (e = cudaMalloc(&in.B, nb * 4)) != cudaSuccess ||
      (e = cudaMalloc(&in.C, nc * 4)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "grouped tuning inputs do not fit");
  }
  fill_uniform_launch(in.A, na, 11, nullptr);
  fill_uniform_launch(in.B, nb, 12, nullptr);
  fill_uniform_launch(in.C, nc, 13, nullptr);
  std::vector<const float*> pa(G), pb(G);
  std::vector<float*> pc(G);
  std::vector<float> alpha(G, 1.0f), beta(G, 1.0f);
  for (int i = 0; i < G; ++i) pa[i] = in.A + oa[i], pb[i] = in.B + ob[i], pc[i] = in.C + oc[i];

  gemm_grouped_plan_t best = nullptr;
  float best_ms = 0.0f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  gemm_status st = GEMM_OK;
  for (int bn : {128, 64}) {
    for (int kb : {4, 2, 8}) {
      gemm_grouped_plan_t p = nullptr;
      st = grouped_create_impl(G, M, N, K, lda, ldb, ldc, mode, bn, kb, &p);
      if (st != GEMM_OK) break;
      std::vector<float> t;
      for (int r = 0; r < 7 && st == GEMM_OK; ++r) {
        cudaEventRecord(e0, nullptr);
        st = grouped_execute_impl(p, alpha.data(), pa.data(), pb.data(), beta.data(), pc.data(),
                                  nullptr, false);
        cudaEventRecord(e1, nullptr);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r >= 2) t.push_back(ms);
      }
      if (st != GEMM_OK) {
        grouped_destroy_impl(p);
        break;
      }
      std::sort(t.begin(), t.end());
      const float med = t[t.size() / 2];
      if (!best || med < best_ms) {
        if (best) grouped_destroy_impl(best);
        best = p, best_ms = med;
      } else {
        grouped_destroy_impl(p);
      }
    }
    if (st != GEMM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GEMM_OK) {
    if (best) grouped_destroy_impl(best);
    return st;
  }
  *out = best;
  return GEMM_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

gemm_status gemm_autotune(const int64_t* shapes, int G, gemm_mode mode, int reps, const char* out_path) {
  clear_error();
  if (G < 0 || (G > 0 && !shapes)) return fail(GEMM_ERR_INVALID_ARG, "bad shape list");
  if (!mode_is_split(mode)) return fail(GEMM_ERR_INVALID_ARG, "autotune needs a tensor-core mode");
  for (int s = 0; s < G; ++s) {
    const int64_t* r = shapes + 6 * s;
    gemm_status st = validate_shape(r[0], r[1], r[2], r[3], r[4], r[5]);
    if (st != GEMM_OK) return fail(st, "shape %d: %s", s, gemm_last_error());
  }
  FILE* f = nullptr;
  if (out_path && *out_path) {
    // an existing file must hold rows of this format (its header names lda)
    if (FILE* old = std::fopen(out_path, "r")) {
      char head[512] = {0};
      const bool has = std::fgets(head, sizeof head, old) != nullptr;
      std::fclose(old);
      if (has && !std::strstr(head, "lda"))
        return fail(GEMM_ERR_IO, "%s holds timing rows without leading dimensions; use a new file",
                    out_path);
    }
    f = std::fopen(out_path, "a");
    if (!f) return fail(GEMM_ERR_IO, "cannot open %s for appending", out_path);
    std::fseek(f, 0, SEEK_END);
    if (std::ftell(f) == 0)
      std::fprintf(f, "M,N,K,lda,ldb,ldc,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused,cluster\n");
  }
  gemm_status st = GEMM_OK;
  for (int s = 0; s < G && st == GEMM_OK; ++s) {
    const int64_t* r = shapes + 6 * s;
    const Shape6 sh{r[0], r[1], r[2], r[3], r[4], r[5]};
    if (sh.M == 0 || sh.N == 0 || sh.K == 0) continue;
    int best = -1;
    float best_ms = 0;
    st = tune_shape(
        sh, mode, reps,
        [&](int cid, float ms) {
          if (!f) return;
          gemm_config c;
          config_get(cid, &c);
          std::fprintf(f, "%lld,%lld,%lld,%lld,%lld,%lld,%d,%d,%.6f,%d,%d,%d,%d,%d,%d\n", (long long)sh.M,
                       (long long)sh.N, (long long)sh.K, (long long)sh.lda, (long long)sh.ldb,
                       (long long)sh.ldc, (int)mode, cid, ms, c.block_n, c.split_k, c.kb, c.group_m,
                       c.fused, c.cluster);
        },
        &best, &best_ms);
    if (f) std::fflush(f);
  }
  if (f) std::fclose(f);
  return st;
}

gemm_status gemm_autotune_load(const char* path) {
  clear_error();
  if (!path) return fail(GEMM_ERR_INVALID_ARG, "null path");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(GEMM_ERR_IO, "cannot open %s", path);
  char line[512];
  int rows = 0;
  while (std::fgets(line, sizeof line, f)) {
    TimingRow r;
    if (!parse_timing_row(line, &r)) continue;
    if (r.cid < 0 || r.cid >= config_count((gemm_mode)r.mode)) continue;
    table_offer((gemm_mode)r.mode, r.sh, r.cid, r.ms);
    ++rows;
  }
  std::fclose(f);
  if (rows == 0) return fail(GEMM_ERR_IO, "no timing rows in %s", path);
  return GEMM_OK;
}

gemm_status gemm_autotune_best(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                               gemm_mode mode, int* config_id, float* ms) {
  clear_error();
  if (!table_lookup(mode, Shape6{M, N, K, lda, ldb, ldc}, config_id, ms))
    return fail(GEMM_ERR_INVALID_ARG, "shape not in the tuned table");
  return GEMM_OK;
}

gemm_status gemm_select_config(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                               gemm_mode mode, gemm_select sel, int* config_id) {
  clear_error();
  if (!config_id) return fail(GEMM_ERR_INVALID_ARG, "null output");
  gemm_status st = validate_shape(M, N, K, lda, ldb, ldc);
  if (st != GEMM_OK) return st;
  if (mode == GEMM_MODE_AUTO) mode = GEMM_MODE_BF16X3;
  if (mode != GEMM_MODE_F32_SIMT && !mode_is_split(mode))
    return fail(GEMM_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
  if (mode == GEMM_MODE_F32_SIMT || M == 0 || N == 0 || K == 0) {
    *config_id = -1;
    return GEMM_OK;
  }
  // the SM count of the current device; the heuristic assumes 152 without one
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  *config_id = select_config(mode, M, N, K, lda, ldb, ldc, sel, sms);
  clear_error();
  return *config_id >= 0 ? GEMM_OK : fail(GEMM_ERR_INVALID_ARG, "no configuration for mode");
}

}  // extern "C"
