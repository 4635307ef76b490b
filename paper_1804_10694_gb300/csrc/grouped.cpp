// Grouped gemm: G independent problems C_g = alpha_g * A_g * B_g + beta_g * C_g
// of uneven shapes in ONE persistent tensor-core launch (plus one launch for
// all block maxima and one for all hi/lo planes), captured into a CUDA graph
// on the first execution and replayed afterwards.
//
// Host side of the plan: the problem table (tensor maps, plane addresses,
// sizes) is written to device memory once; problems are ordered by
// decreasing K so that the persistent CTAs, which walk the global tile list
// in a fixed stride, take the longest tiles first and the short ones fill the
// tail.  Per-execution values (A, B, C pointers, alpha, beta) live in a
// second small table that is re-uploaded only when it changes, ahead of the
// graph launch on the same stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/gemm.h"
#include "internal.h"
#include "runtime.h"

struct gemm_grouped_plan_s {
  int G = 0;
  gemm_mode mode = GEMM_MODE_BF16X3;
  gb::Prec prec = gb::Prec::BF16;
  int device = 0, sms = 0;
  int bn = 128, kb = 4, group_m = 16;
  std::vector<int64_t> M, N, K, lda, ldb, ldc;   // caller's order
  std::vector<int> order;                        // table slot -> caller index
  void* ws = nullptr;
  size_t ws_bytes = 0;
  gb::GroupedProblem* d_probs = nullptr;
  gb::GroupedPtrs* d_ptrs = nullptr;
  gb::GroupedUnit* d_units = nullptr;
  int* d_split_prefix = nullptr;
  size_t amax_count = 0;          // words of block maxima and counters (the unit counter follows)
  unsigned* d_amax = nullptr;
  size_t amax_bytes = 0;
  int num_units = 0, split_total = 0;
  std::vector<gb::GroupedPtrs> h_ptrs, uploaded;
  bool have_uploaded = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* err = nullptr;
};

namespace gb {

namespace {

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

gemm_status launch_all(gemm_grouped_plan_t p, cudaStream_t s) {
  cudaError_t e;
  if (p->mode == GEMM_MODE_F32_SIMT) {
    // reference form: one plain FP32 launch per problem (graph-captured too)
    std::vector<GroupedPtrs> h(p->h_ptrs);
    for (int slot = 0; slot < p->G; ++slot) {
      const int i = p->order[slot];
      const GroupedPtrs& q = h[slot];
      if (p->M[i] == 0 || p->N[i] == 0) continue;
      if (p->K[i] == 0 || q.alpha == 0.0f)
        e = scale_c_launch(p->M[i], p->N[i], q.beta, q.C, p->ldc[i], s);
      else
        e = simt_gemm_launch(p->M[i], p->N[i], p->K[i], q.alpha, q.A, p->lda[i], q.B, p->ldb[i],
                             q.beta, q.C, p->ldc[i], s);
      if (e != cudaSuccess) return cuda_fail(e, "grouped SIMT launch");
    }
    return GEMM_OK;
  }
  if (p->num_units == 0) return GEMM_OK;
  // (the block maxima, counters and unit counter are zero: the previous
  // execution's gemm launch cleared them)
  if ((e = grouped_pack_launch(p->prec, p->d_probs, p->d_ptrs, p->d_split_prefix, p->split_total, p->G,
                               p->sms, s)) != cudaSuccess)
    return cuda_fail(e, "grouped pack launch");
  GroupedArgs a{};
  a.probs = p->d_probs;
  a.ptrs = p->d_ptrs;
  a.units = p->d_units;
  a.G = p->G;
  a.num_units = p->num_units;
  a.kb = p->kb;
  a.group_m = p->group_m;
  a.err = p->err;
  a.unit_ctr = reinterpret_cast<int*>(p->d_amax + p->amax_count);
  a.state = p->d_amax;
  a.state_words = (int)(p->amax_count + 1);
  const int grid = std::min(p->num_units, p->sms);
  if ((e = tc_grouped_launch(p->bn, p->prec, grid, a, s)) != cudaSuccess)
    return cuda_fail(e, "grouped tensor-core launch");
  return GEMM_OK;
}

gemm_status upload_ptrs(gemm_grouped_plan_t p, const float* alpha, const float* const* A,
                        const float* const* B, const float* beta, float* const* C, cudaStream_t s) {
  if (!alpha || !beta || !A || !B || !C) return fail(GEMM_ERR_INVALID_ARG, "null argument array");
  for (int slot = 0; slot < p->G; ++slot) {
    const int i = p->order[slot];
    GroupedPtrs& q = p->h_ptrs[slot];
    q.A = A[i];
    q.B = B[i];
    q.C = C[i];
    q.alpha = alpha[i];
    q.beta = beta[i];
    if (p->M[i] > 0 && p->N[i] > 0) {
      if (!C[i]) return fail(GEMM_ERR_INVALID_ARG, "null C for problem %d", i);
      if (p->K[i] > 0 && alpha[i] != 0.0f && (!A[i] || !B[i]))
        return fail(GEMM_ERR_INVALID_ARG, "null A or B for problem %d", i);
    }
  }
  if (p->mode == GEMM_MODE_F32_SIMT) return GEMM_OK;   // pointers are kernel arguments
  if (p->have_uploaded &&
      std::memcmp(p->uploaded.data(), p->h_ptrs.data(), p->G * sizeof(GroupedPtrs)) == 0)
    return GEMM_OK;
  // pageable source: the copy is staged before the call returns, so h_ptrs may change afterwards
  cudaError_t e = cudaMemcpyAsync(p->d_ptrs, p->h_ptrs.data(), p->G * sizeof(GroupedPtrs),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "upload of the pointer table");
  p->uploaded = p->h_ptrs;
  p->have_uploaded = true;
  return GEMM_OK;
}

void destroy_graph(gemm_grouped_plan_t p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

}  // namespace

// Grouped configuration for a set of shapes under a selection policy.
void grouped_default_config(const std::vector<int64_t>& N, int* bn, int* kb) {
  // output columns computed per useful column: pick the tile width that wastes less
  double waste64 = 0, waste128 = 0, total = 0;
  for (int64_t n : N) {
    total += (double)n;
    waste64 += (double)((n + 63) / 64 * 64 - n);
    waste128 += (double)((n + 127) / 128 * 128 - n);
  }
  *bn = (waste128 - waste64) > 0.25 * total ? 64 : 128;
  *kb = 4;
}

gemm_status grouped_create_impl(int G, const int64_t* M, const int64_t* N, const int64_t* K,
                                const int64_t* lda, const int64_t* ldb, const int64_t* ldc,
                                gemm_mode mode, int bn_override, int kb_override,
                                gemm_grouped_plan_t* out) {
  if (!out) return fail(GEMM_ERR_INVALID_ARG, "null plan output pointer");
  *out = nullptr;
  if (G < 0) return fail(GEMM_ERR_INVALID_ARG, "negative problem count");
  if (G > 0 && (!M || !N || !K || !lda || !ldb || !ldc))
    return fail(GEMM_ERR_INVALID_ARG, "null shape array");
  for (int i = 0; i < G; ++i) {
    gemm_status st = validate_shape(M[i], N[i], K[i], lda[i], ldb[i], ldc[i]);
    if (st != GEMM_OK) {
      const std::string msg = gemm_last_error();
      return fail(st, "problem %d: %s", i, msg.c_str());
    }
  }
  if (mode == GEMM_MODE_AUTO) mode = GEMM_MODE_BF16X3;
  if (mode != GEMM_MODE_F32_SIMT && !mode_is_split(mode))
    return fail(GEMM_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int major = 0, minor = 0, sms = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (mode != GEMM_MODE_F32_SIMT && !(major == 10 && minor == 3))
    return fail(GEMM_ERR_UNSUPPORTED_DEVICE, "tensor-core modes need compute capability 10.3");

  std::unique_ptr<gemm_grouped_plan_s, void (*)(gemm_grouped_plan_t)> p(new gemm_grouped_plan_s(),
                                                                         grouped_destroy_impl);
  p->G = G;
  p->mode = mode;
  p->prec = prec_of_mode(mode);
  p->device = dev;
  p->sms = sms;
  p->M.assign(M, M + G), p->N.assign(N, N + G), p->K.assign(K, K + G);
  p->lda.assign(lda, lda + G), p->ldb.assign(ldb, ldb + G), p->ldc.assign(ldc, ldc + G);
  p->order.resize(G);
  std::iota(p->order.begin(), p->order.end(), 0);
  // longest k-loop first (stable: equal K keep the caller's order)
  std::stable_sort(p->order.begin(), p->order.end(),
                   [&](int a, int b) { return p->K[a] > p->K[b]; });
  p->h_ptrs.assign(G, GroupedPtrs{});
  gemm_status st = device_err_word(&p->err);
  if (st != GEMM_OK) return st;
  e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  if (mode == GEMM_MODE_F32_SIMT || G == 0) {
    *out = p.release();
    return GEMM_OK;
  }

  grouped_default_config(p->N, &p->bn, &p->kb);
  if (bn_override > 0) p->bn = bn_override;
  if (kb_override > 0) p->kb = kb_override;
  if (p->bn != 64 && p->bn != 128) return fail(GEMM_ERR_INVALID_ARG, "grouped tile width must be 64 or 128");
  p->kb = std::max(1, std::min(p->kb, 8));

  // layout of the workspace: per problem A planes | B planes, then block
  // maxima, then the device tables
  const Prec pr = p->prec;
  const int es = prec_elem_bytes(pr);
  std::vector<GroupedProblem> hp(G);
  std::vector<size_t> offA(G), offB(G);
  std::vector<int> tile_prefix(G + 1, 0), spl_prefix(G + 1, 0);
  size_t off = 0, amax_count = 0;
  std::vector<size_t> amax_off(G);
  for (int slot = 0; slot < G; ++slot) {
    const int i = p->order[slot];
    const int64_t Ki = std::max<int64_t>(p->K[i], 1);
    const int64_t pitch = packed_k_pitch(pr, Ki);
    GroupedProblem& g = hp[slot];
    std::memset(&g, 0, sizeof g);
    g.M = (int)p->M[i], g.N = (int)p->N[i], g.K = (int)p->K[i];
    g.pitch = pitch, g.lda = p->lda[i], g.ldb = p->ldb[i], g.ldc = p->ldc[i];
    g.chunks = (int)((p->K[i] + prec_chunk_elems(pr) - 1) / prec_chunk_elems(pr));
    const bool empty = p->M[i] == 0 || p->N[i] == 0;
    g.tiles_m = empty ? 0 : (int)((p->M[i] + 127) / 128);
    g.tiles_n = empty ? 0 : (int)((p->N[i] + p->bn - 1) / p->bn);
    offA[slot] = off;
    off = round256(off + (size_t)prec_planes(pr) * std::max<int64_t>(p->M[i], 1) * pitch * es);
    offB[slot] = off;
    off = round256(off + (size_t)prec_planes(pr) * std::max<int64_t>(p->N[i], 1) * pitch * es);
    // per problem: maxima of A's and B's blocks, then one pack counter per block
    amax_off[slot] = amax_count;
    amax_count += 2 * ((size_t)(p->M[i] + kScaleBlock - 1) / kScaleBlock +
                       (size_t)(p->N[i] + kScaleBlock - 1) / kScaleBlock);
    tile_prefix[slot + 1] = tile_prefix[slot] + g.tiles_m * g.tiles_n;
    const bool pack = !empty && p->K[i] > 0;
    spl_prefix[slot + 1] = spl_prefix[slot] + (pack ? pack_first_items(p->M[i], p->N[i], pitch) : 0);
  }
  // per-execution state: block maxima and pack counters of every problem,
  // then the launch's unit counter (its dynamic tile order), then the gemm
  // launch's done counter; zeroed once here and, after every execution, by
  // the last CTA of the gemm launch
  const size_t off_amax = off;
  p->amax_bytes = (amax_count + 2) * sizeof(unsigned);
  p->amax_count = amax_count;
  off = round256(off + p->amax_bytes);
  const size_t off_probs = off;
  off = round256(off + (size_t)G * sizeof(GroupedProblem));
  const size_t off_ptrs = off;
  off = round256(off + (size_t)G * sizeof(GroupedPtrs));
  const size_t off_units = off;
  off = round256(off + (size_t)std::max(tile_prefix[G], 1) * sizeof(GroupedUnit));
  const size_t off_pref = off;
  off = round256(off + (size_t)(G + 1) * sizeof(int));
  p->ws_bytes = off;
  if ((e = cudaMalloc(&p->ws, p->ws_bytes)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "cudaMalloc(%zu bytes) for the grouped workspace", p->ws_bytes);
  }
  char* w = static_cast<char*>(p->ws);
  p->d_amax = reinterpret_cast<unsigned*>(w + off_amax);
  p->d_probs = reinterpret_cast<GroupedProblem*>(w + off_probs);
  p->d_ptrs = reinterpret_cast<GroupedPtrs*>(w + off_ptrs);
  p->d_units = reinterpret_cast<GroupedUnit*>(w + off_units);
  p->d_split_prefix = reinterpret_cast<int*>(w + off_pref);
  if ((e = cudaMemset(p->d_amax, 0, p->amax_bytes)) != cudaSuccess) return cuda_fail(e, "cudaMemset(plan state)");
  for (int slot = 0; slot < G; ++slot) {
    const int i = p->order[slot];
    GroupedProblem& g = hp[slot];
    g.planesA = w + offA[slot];
    g.planesB = w + offB[slot];
    const int64_t nbA = (p->M[i] + kScaleBlock - 1) / kScaleBlock, nbB = (p->N[i] + kScaleBlock - 1) / kScaleBlock;
    g.amaxA = p->d_amax + amax_off[slot];
    g.amaxB = g.amaxA + nbA;
    g.cntA = g.amaxB + nbB;
    g.cntB = g.cntA + nbA;
    const int64_t Ki = std::max<int64_t>(p->K[i], 1);
    if ((st = encode_planes_map(&g.tmA, pr, g.planesA, std::max<int64_t>(p->M[i], 1), Ki, g.pitch, 128,
                                128)) != GEMM_OK)
      return st;
    if ((st = encode_planes_map(&g.tmB, pr, g.planesB, std::max<int64_t>(p->N[i], 1), Ki, g.pitch,
                                p->bn, 128)) != GEMM_OK)
      return st;
  }
  if ((e = tc_prepare(p->bn, pr)) != cudaSuccess) return cuda_fail(e, "kernel attribute");
  p->num_units = tile_prefix[G];
  p->split_total = spl_prefix[G];
  if ((e = cudaMemcpy(p->d_probs, hp.data(), (size_t)G * sizeof(GroupedProblem), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload of the problem table");
  // unit table: each problem's tiles in grouped raster order (groups of
  // group_m row tiles, columns inside a group, rows fastest)
  std::vector<GroupedUnit> units;
  units.reserve(p->num_units);
  for (int slot = 0; slot < G; ++slot) {
    const GroupedProblem& g = hp[slot];
    const int gm = std::max(1, std::min(p->group_m, g.tiles_m));
    for (int t = 0; t < g.tiles_m * g.tiles_n; ++t) {
      const int group_tiles = gm * g.tiles_n;
      const int first_m = (t / group_tiles) * gm;
      const int rows = std::min(g.tiles_m - first_m, gm);
      const int r = t % group_tiles;
      units.push_back(GroupedUnit{slot, first_m + r % rows, r / rows, g.chunks});
    }
  }
  if (!units.empty() &&
      (e = cudaMemcpy(p->d_units, units.data(), units.size() * sizeof(GroupedUnit), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload of the unit table");
  if ((e = cudaMemcpy(p->d_split_prefix, spl_prefix.data(), spl_prefix.size() * sizeof(int),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload of the prefix table");
  *out = p.release();
  return GEMM_OK;
}

gemm_status grouped_execute_impl(gemm_grouped_plan_t p, const float* alpha, const float* const* A,
                                 const float* const* B, const float* beta, float* const* C,
                                 cudaStream_t s, bool use_graph) {
  if (!p) return fail(GEMM_ERR_INVALID_ARG, "null plan");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(GEMM_ERR_INVALID_ARG, "plan belongs to device %d", p->device);
  if (p->G == 0) return GEMM_OK;
  gemm_status st = upload_ptrs(p, alpha, A, B, beta, C, s);
  if (st != GEMM_OK) return st;
  if (!use_graph) return launch_all(p, s);
  if (p->mode == GEMM_MODE_F32_SIMT) {
    // the per-problem launches carry the pointers: recapture when they change
    destroy_graph(p);
  }
  if (!p->exec) {
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    st = launch_all(p, p->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->cap_stream, &g);
    if (st != GEMM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    p->graph = g;
    if ((e = cudaGraphInstantiate(&p->exec, g, 0)) != cudaSuccess) {
      destroy_graph(p);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  cudaError_t e = cudaGraphLaunch(p->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return GEMM_OK;
}

void grouped_destroy_impl(gemm_grouped_plan_t p) {
  if (!p) return;
  destroy_graph(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->ws) cudaFree(p->ws);
  delete p;
}

}  // namespace gb

using namespace gb;

extern "C" {

gemm_status gemm_grouped_plan_create(int G, const int64_t* M, const int64_t* N, const int64_t* K,
                                     const int64_t* lda, const int64_t* ldb, const int64_t* ldc,
                                     gemm_mode mode, gemm_select sel, gemm_grouped_plan_t* out) {
  clear_error();
  if (sel == GEMM_SELECT_EXHAUSTIVE && mode != GEMM_MODE_F32_SIMT)
    return grouped_tune_and_create(G, M, N, K, lda, ldb, ldc, mode, out);
  return grouped_create_impl(G, M, N, K, lda, ldb, ldc, mode, 0, 0, out);
}

gemm_status gemm_grouped_plan_create_config(int G, const int64_t* M, const int64_t* N,
                                            const int64_t* K, const int64_t* lda,
                                            const int64_t* ldb, const int64_t* ldc, gemm_mode mode,
                                            int block_n, int kb, gemm_grouped_plan_t* out) {
  clear_error();
  if (block_n != 64 && block_n != 128) return fail(GEMM_ERR_INVALID_ARG, "block_n must be 64 or 128");
  if (kb < 1 || kb > 8) return fail(GEMM_ERR_INVALID_ARG, "kb must be in 1..8");
  return grouped_create_impl(G, M, N, K, lda, ldb, ldc, mode, block_n, kb, out);
}

gemm_status gemm_grouped_execute(gemm_grouped_plan_t plan, const float* alpha, const float* const* A,
                                 const float* const* B, const float* beta, float* const* C,
                                 gemm_stream_t stream) {
  clear_error();
  return grouped_execute_impl(plan, alpha, A, B, beta, C, reinterpret_cast<cudaStream_t>(stream), true);
}

gemm_status gemm_grouped_execute_eager(gemm_grouped_plan_t plan, const float* alpha,
                                       const float* const* A, const float* const* B,
                                       const float* beta, float* const* C, gemm_stream_t stream) {
  clear_error();
  return grouped_execute_impl(plan, alpha, A, B, beta, C, reinterpret_cast<cudaStream_t>(stream), false);
}

gemm_status gemm_grouped_plan_info(gemm_grouped_plan_t plan, int* block_n, int* kb, int* tiles,
                                   size_t* workspace_bytes) {
  clear_error();
  if (!plan) return fail(GEMM_ERR_INVALID_ARG, "null plan");
  if (block_n) *block_n = plan->bn;
  if (kb) *kb = plan->kb;
  if (tiles) *tiles = plan->num_units;
  if (workspace_bytes) *workspace_bytes = plan->ws_bytes;
  return GEMM_OK;
}

gemm_status gemm_grouped_plan_destroy(gemm_grouped_plan_t plan) {
  clear_error();
  grouped_destroy_impl(plan);
  return GEMM_OK;
}

}  // extern "C"
