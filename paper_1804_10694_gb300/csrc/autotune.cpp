// Autotuner and tile-configuration selection.  The paper autotunes the tile
// size and unroll factor of its sgemm for the machine it runs on (Section
// VI-A); here the tuned quantities are the tensor-core kernels' tile width,
// split-K, TMEM fold length and raster grouping.  For each shape every
// DISTINCT effective configuration (candidates that behave identically on the
// shape, e.g. split-K above the number of k-chunks, are timed once) is run
// `reps` times after two warm-up executions, each execution timed with CUDA
// events; the median is recorded.  Results are appended to a CSV file
// ("M,N,K,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused") that the cost
// model trains on, and the fastest configuration per shape is kept in an
// in-memory table (GEMM_SELECT_TABLE).
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
  const int64_t tiles_m = (M + 127) / 128;
  e.bn = c.block_n;
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
  std::set<std::tuple<int, int, int, int, int>> seen;
  const Prec p = prec_of_mode(mode);
  gemm_config c;
  for (int id = 0; id < config_count(mode); ++id) {
    config_get(id, &c);
    const EffConfig e = effective_config(c, p, M, N, K);
    if (seen.insert(std::make_tuple(e.bn, e.split_k, e.kb, e.group_m, e.fused)).second) out.push_back(id);
  }
  return out;
}

// -------------------------------------------------------------- tuned table
namespace {
std::mutex g_table_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t>, std::pair<int, float>> g_table;

void table_offer(gemm_mode mode, int64_t M, int64_t N, int64_t K, int cid, float ms) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto key = std::make_tuple((int)mode, M, N, K);
  auto it = g_table.find(key);
  if (it == g_table.end() || ms < it->second.second) g_table[key] = {cid, ms};
}
}  // namespace

bool table_lookup(gemm_mode mode, int64_t M, int64_t N, int64_t K, int* cid, float* ms) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  auto it = g_table.find(std::make_tuple((int)mode, M, N, K));
  if (it == g_table.end()) return false;
  if (cid) *cid = it->second.first;
  if (ms) *ms = it->second.second;
  return true;
}

// ------------------------------------------------------------------- timing
// Median time of `reps` executions of a plan with the given configuration.
gemm_status time_config(int64_t M, int64_t N, int64_t K, gemm_mode mode, int cid, const float* A,
                        const float* B, float* C, int reps, float* median_ms) {
  gemm_plan_t p = nullptr;
  gemm_status st = plan_create_impl(M, N, K, std::max<int64_t>(K, 1), std::max<int64_t>(N, 1),
                                    std::max<int64_t>(N, 1), mode, cid, GEMM_SELECT_DEFAULT, &p);
  if (st != GEMM_OK) return st;
  reps = std::max(1, reps);
  std::vector<cudaEvent_t> ev(2 * reps, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) break;
  if (e == cudaSuccess) {
    for (int w = 0; w < 2 && st == GEMM_OK; ++w) st = plan_execute_impl(p, 1.0f, A, B, 0.0f, C, nullptr);
    for (int r = 0; r < reps && st == GEMM_OK; ++r) {
      cudaEventRecord(ev[2 * r], nullptr);
      st = plan_execute_impl(p, 1.0f, A, B, 0.0f, C, nullptr);
      cudaEventRecord(ev[2 * r + 1], nullptr);
    }
    if (st == GEMM_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) st = cuda_fail(e, "tuning run");
    if (st == GEMM_OK) {
      std::vector<float> t(reps);
      for (int r = 0; r < reps; ++r) cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]);
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

gemm_status make_inputs(int64_t M, int64_t N, int64_t K, uint64_t seed, DeviceInputs* in) {
  cudaError_t e;
  if ((e = cudaMalloc(&in->A, (size_t)std::max<int64_t>(M * K, 1) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&in->B, (size_t)std::max<int64_t>(K * N, 1) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&in->C, (size_t)std::max<int64_t>(M * N, 1) * 4)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "tuning inputs for %lldx%lldx%lld do not fit", (long long)M,
                (long long)N, (long long)K);
  }
  if ((e = fill_uniform_launch(in->A, (size_t)(M * K), seed, nullptr)) != cudaSuccess ||
      (e = fill_uniform_launch(in->B, (size_t)(K * N), seed + 1, nullptr)) != cudaSuccess ||
      (e = fill_uniform_launch(in->C, (size_t)(M * N), seed + 2, nullptr)) != cudaSuccess)
    return cuda_fail(e, "fill tuning inputs");
  return GEMM_OK;
}

}  // namespace

// Time every distinct configuration of one shape; calls `row` for each.
template <class RowFn>
gemm_status tune_shape(int64_t M, int64_t N, int64_t K, gemm_mode mode, int reps, RowFn row,
                       int* best_cid, float* best_ms) {
  DeviceInputs in;
  gemm_status st = make_inputs(M, N, K, 0x5EEDull + (uint64_t)(M * 31 + N * 17 + K), &in);
  if (st != GEMM_OK) return st;
  *best_cid = -1;
  *best_ms = 0.0f;
  for (int cid : distinct_configs(mode, M, N, K)) {
    float ms = 0.0f;
    st = time_config(M, N, K, mode, cid, in.A, in.B, in.C, reps, &ms);
    if (st != GEMM_OK) return st;
    row(cid, ms);
    table_offer(mode, M, N, K, cid, ms);
    if (*best_cid < 0 || ms < *best_ms) *best_cid = cid, *best_ms = ms;
  }
  return GEMM_OK;
}

int select_config(gemm_mode mode, int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                  int64_t ldc, gemm_select sel, int sms) {
  (void)lda, (void)ldb, (void)ldc;
  int cid = -1;
  float ms = 0.0f;
  switch (sel) {
    case GEMM_SELECT_TABLE:
      if (table_lookup(mode, M, N, K, &cid, &ms)) return cid;
      break;
    case GEMM_SELECT_MODEL:
      if (costmodel_pick(mode, M, N, K, &cid, &ms) == GEMM_OK && cid >= 0) return cid;
      break;
    case GEMM_SELECT_EXHAUSTIVE: {
      if (tune_shape(M, N, K, mode, 5, [](int, float) {}, &cid, &ms) == GEMM_OK && cid >= 0) return cid;
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
  FILE* f = nullptr;
  if (out_path && *out_path) {
    f = std::fopen(out_path, "a");
    if (!f) return fail(GEMM_ERR_IO, "cannot open %s for appending", out_path);
    std::fseek(f, 0, SEEK_END);
    if (std::ftell(f) == 0)
      std::fprintf(f, "M,N,K,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused\n");
  }
  gemm_status st = GEMM_OK;
  for (int s = 0; s < G && st == GEMM_OK; ++s) {
    const int64_t M = shapes[3 * s], N = shapes[3 * s + 1], K = shapes[3 * s + 2];
    if ((st = validate_shape(M, N, K, std::max<int64_t>(K, 1), std::max<int64_t>(N, 1),
                             std::max<int64_t>(N, 1))) != GEMM_OK)
      break;
    if (M == 0 || N == 0 || K == 0) continue;
    int best = -1;
    float best_ms = 0;
    st = tune_shape(
        M, N, K, mode, reps,
        [&](int cid, float ms) {
          if (!f) return;
          gemm_config c;
          config_get(cid, &c);
          std::fprintf(f, "%lld,%lld,%lld,%d,%d,%.6f,%d,%d,%d,%d,%d\n", (long long)M, (long long)N,
                       (long long)K, (int)mode, cid, ms, c.block_n, c.split_k, c.kb, c.group_m,
                       c.fused);
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
    long long M, N, K;
    int mode, cid;
    float ms;
    if (std::sscanf(line, "%lld,%lld,%lld,%d,%d,%f", &M, &N, &K, &mode, &cid, &ms) != 6) continue;
    if (cid < 0 || cid >= config_count((gemm_mode)mode)) continue;
    table_offer((gemm_mode)mode, M, N, K, cid, ms);
    ++rows;
  }
  std::fclose(f);
  if (rows == 0) return fail(GEMM_ERR_IO, "no timing rows in %s", path);
  return GEMM_OK;
}

gemm_status gemm_autotune_best(int64_t M, int64_t N, int64_t K, gemm_mode mode, int* config_id,
                               float* ms) {
  clear_error();
  if (!table_lookup(mode, M, N, K, config_id, ms))
    return fail(GEMM_ERR_INVALID_ARG, "shape not in the tuned table");
  return GEMM_OK;
}

}  // extern "C"
