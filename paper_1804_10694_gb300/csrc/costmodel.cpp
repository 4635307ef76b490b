// Learned tile-choice cost model.  The paper picks tile sizes and unroll
// factors by autotuning (Section VI-A); here a small MLP, trained on the
// autotuner's own timings, predicts log execution time from shape and
// configuration features, so that a configuration can be chosen (argmin over
// the candidates) without timing them.  Exhaustive tuning stays available as
// the fallback and as the reference that the model's regret is measured
// against.
//
// Training runs on the GPU with the library's kernels: forward and per-sample
// backward kernels (mlp.cu), weight gradients as dZ^T H products by the
// library's plain FP32 gemm kernel, and an Adam update kernel.  Full-batch
// Adam with a cosine-decayed learning rate minimises the mean squared error
// of normalised log time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gemm.h"
#include "mlp.h"
#include "runtime.h"
#include "tuning.h"

namespace gb {

// ------------------------------------------------------------------ features
void costmodel_features(gemm_mode mode, int64_t M, int64_t N, int64_t K, const gemm_config& c,
                        int sms, float* out) {
  const Prec p = prec_of_mode(mode);
  const EffConfig e = effective_config(c, p, M, N, K);
  const int ck = prec_chunk_elems(p);
  const double chunks = (double)((K + ck - 1) / ck);
  // units run on sms / cluster processors (SMs, or pairs of SMs)
  const double procs = (double)(sms / e.cluster);
  const double units = (double)e.tiles * e.split_k;
  const double waves = units / procs;
  const double rem = units - std::floor(waves) * procs;
  const double fill = rem == 0.0 ? 1.0 : rem / procs;
  const double tile_h = 128.0 * e.cluster;
  const double tiles_m = std::ceil((double)M / tile_h), tiles_n = (double)((N + e.bn - 1) / e.bn);
  const double padded = (tiles_m * tile_h) * (tiles_n * e.bn) * (chunks * ck) /
                            ((double)M * (double)N * (double)K) - 1.0;
  const double ai = 2.0 * M * N * K / (4.0 * ((double)M * K + (double)K * N + 2.0 * M * N));
  out[0] = (float)std::log2((double)M);
  out[1] = (float)std::log2((double)N);
  out[2] = (float)std::log2((double)K);
  out[3] = (float)(e.bn / 128.0);
  out[4] = (float)std::log2((double)e.split_k);
  out[5] = (float)(e.kb / 8.0);
  out[6] = (float)std::log2((double)e.group_m);
  out[7] = (float)std::log2((double)e.tiles);
  out[8] = (float)std::log2(1.0 + waves);
  out[9] = (float)fill;
  out[10] = (float)padded;
  out[11] = (float)std::log2(ai);
  out[12] = (float)std::log2((double)e.chunks_per_split);
  out[13] = mode == GEMM_MODE_TF32X3 ? 1.0f : 0.0f;
  out[14] = c.fused ? 1.0f : 0.0f;
  out[15] = mode == GEMM_MODE_BF16X6 ? 1.0f : 0.0f;   // six products per k-step, three planes
  out[16] = e.cluster == 2 ? 1.0f : 0.0f;              // a 256-row tile on a pair of SMs
}

namespace {

// An ensemble of `members` networks trained from different initial weights
// on the same data (theta holds their parameters one after another); the
// prediction is the mean of their outputs, which evens out the run-to-run
// spread of a single network's choices.
struct Model {
  bool loaded = false;
  int members = 0;
  std::vector<float> mean, stdv, theta;
  float ymean = 0.0f, ystd = 1.0f;
};
constexpr int kMembers = 5;
std::mutex g_model_mu;
Model g_model;

struct DevBuf {
  float* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(float)); }
};

int sm_count() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Device workspace of one forward + backward pass over n samples.
struct Pass {
  int n = 0;
  DevBuf X, t, y, Z1, Z2, H1, H2, dZ1T, dZ2T, dy, ones, theta, grad, loss, part;
  gemm_status alloc(int n_) {
    n = n_;
    const int P = mlp_param_count();
    const size_t nh = (size_t)n * kHidden;
    if (X.alloc((size_t)n * kFeatures) || t.alloc(n) || y.alloc(n) || Z1.alloc(nh) || Z2.alloc(nh) ||
        H1.alloc(nh) || H2.alloc(nh) || dZ1T.alloc(nh) || dZ2T.alloc(nh) || dy.alloc(n) ||
        ones.alloc(n) || theta.alloc(P) || grad.alloc(P) || loss.alloc(1) ||
        part.alloc((size_t)batch_outer_parts(n) * kHidden * kHidden)) {
      cudaGetLastError();
      return fail(GEMM_ERR_ALLOC, "cost-model buffers for %d samples", n);
    }
    cudaError_t e = fill_value_launch(ones.p, n, 1.0f, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "fill");
    return GEMM_OK;
  }
};

// Loss (optional) and gradient of the MSE loss at pass.theta, on the GPU.
gemm_status loss_and_grad(Pass& ps, bool want_loss, cudaStream_t s) {
  const int n = ps.n, F = kFeatures, Hd = kHidden;
  cudaError_t e;
  if ((e = mlp_forward_launch(ps.X.p, n, ps.theta.p, ps.y.p, ps.Z1.p, ps.Z2.p, s)) != cudaSuccess)
    return cuda_fail(e, "mlp forward");
  if (want_loss && (e = mse_launch(ps.y.p, ps.t.p, n, ps.loss.p, s)) != cudaSuccess)
    return cuda_fail(e, "mse");
  if ((e = mlp_backward_sample_launch(ps.t.p, n, ps.theta.p, ps.y.p, ps.Z1.p, ps.Z2.p, ps.dZ1T.p,
                                      ps.dZ2T.p, ps.H1.p, ps.H2.p, ps.dy.p, s)) != cudaSuccess)
    return cuda_fail(e, "mlp backward");
  float* g = ps.grad.p;
  float* gW1 = g;
  float* gb1 = gW1 + Hd * F;
  float* gW2 = gb1 + Hd;
  float* gb2 = gW2 + Hd * Hd;
  float* gw3 = gb2 + Hd;
  float* gb3 = gw3 + Hd;
  // weight gradients: products over the batch (the partials of one product
  // are summed before the next one overwrites the scratch: same stream)
  float* pt = ps.part.p;
  if ((e = batch_outer_launch(ps.dZ1T.p, n, ps.X.p, F, Hd, F, n, pt, gW1, s)) ||
      (e = batch_outer_launch(ps.dZ1T.p, n, ps.ones.p, 1, Hd, 1, n, pt, gb1, s)) ||
      (e = batch_outer_launch(ps.dZ2T.p, n, ps.H1.p, Hd, Hd, Hd, n, pt, gW2, s)) ||
      (e = batch_outer_launch(ps.dZ2T.p, n, ps.ones.p, 1, Hd, 1, n, pt, gb2, s)) ||
      (e = batch_outer_launch(ps.dy.p, n, ps.H2.p, Hd, 1, Hd, n, pt, gw3, s)) ||
      (e = batch_outer_launch(ps.dy.p, n, ps.ones.p, 1, 1, 1, n, pt, gb3, s)))
    return cuda_fail(e, "gradient products");
  return GEMM_OK;
}

uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// He-uniform weights, zero biases, from a counter-based generator.
std::vector<float> init_params(uint64_t seed) {
  const int F = kFeatures, Hd = kHidden;
  std::vector<float> th(mlp_param_count(), 0.0f);
  auto uni = [&](uint64_t i, double bound) {
    const double u = (double)(splitmix64(seed * 0x9E3779B97F4A7C15ull + i) >> 11) / 9007199254740992.0;
    return (float)((2.0 * u - 1.0) * bound);
  };
  uint64_t k = 0;
  for (int i = 0; i < Hd * F; ++i) th[i] = uni(k++, std::sqrt(6.0 / F));
  float* W2 = th.data() + Hd * F + Hd;
  for (int i = 0; i < Hd * Hd; ++i) W2[i] = uni(k++, std::sqrt(6.0 / Hd));
  float* w3 = W2 + Hd * Hd + Hd;
  for (int i = 0; i < Hd; ++i) w3[i] = uni(k++, std::sqrt(6.0 / Hd));
  return th;
}

gemm_status save_model(const Model& m, const char* path) {
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(GEMM_ERR_IO, "cannot write %s", path);
  const int P = mlp_param_count();
  std::fprintf(f, "gb300-gemm-costmodel 2\nfeatures %d hidden %d params %d members %d\n", kFeatures,
               kHidden, P, m.members);
  std::fprintf(f, "mean");
  for (float v : m.mean) std::fprintf(f, " %.9g", v);
  std::fprintf(f, "\nstd");
  for (float v : m.stdv) std::fprintf(f, " %.9g", v);
  std::fprintf(f, "\ntarget %.9g %.9g", m.ymean, m.ystd);
  for (int k = 0; k < m.members; ++k) {
    std::fprintf(f, "\ntheta");
    for (int i = 0; i < P; ++i) std::fprintf(f, " %.9g", m.theta[(size_t)k * P + i]);
  }
  std::fprintf(f, "\n");
  const bool ok = std::ferror(f) == 0;
  std::fclose(f);
  return ok ? GEMM_OK : fail(GEMM_ERR_IO, "write error on %s", path);
}

gemm_status load_model(const char* path, Model* m) {
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(GEMM_ERR_IO, "cannot open %s", path);
  char tag[64];
  int ver = 0, F = 0, Hd = 0, P = 0;
  auto bad = [&](const char* what) {
    std::fclose(f);
    return fail(GEMM_ERR_IO, "%s: malformed cost-model file (%s)", path, what);
  };
  // version 1: one network; version 2: "members K" networks
  if (std::fscanf(f, "%63s %d", tag, &ver) != 2 || std::strcmp(tag, "gb300-gemm-costmodel") ||
      (ver != 1 && ver != 2))
    return bad("header");
  if (std::fscanf(f, " features %d hidden %d params %d", &F, &Hd, &P) != 3 || F != kFeatures ||
      Hd != kHidden || P != mlp_param_count())
    return bad("dimensions");
  int K = 1;
  if (ver == 2 && (std::fscanf(f, " members %d", &K) != 1 || K < 1 || K > 64)) return bad("members");
  m->members = K;
  m->mean.resize(F), m->stdv.resize(F), m->theta.resize((size_t)K * P);
  if (std::fscanf(f, " %63s", tag) != 1 || std::strcmp(tag, "mean")) return bad("mean");
  for (auto& v : m->mean)
    if (std::fscanf(f, "%f", &v) != 1) return bad("mean values");
  if (std::fscanf(f, " %63s", tag) != 1 || std::strcmp(tag, "std")) return bad("std");
  for (auto& v : m->stdv)
    if (std::fscanf(f, "%f", &v) != 1 || !(v > 0.0f)) return bad("std values");
  if (std::fscanf(f, " target %f %f", &m->ymean, &m->ystd) != 2 || !(m->ystd > 0.0f)) return bad("target");
  for (int k = 0; k < K; ++k) {
    if (std::fscanf(f, " %63s", tag) != 1 || std::strcmp(tag, "theta")) return bad("theta");
    for (int i = 0; i < P; ++i) {
      float& v = m->theta[(size_t)k * P + i];
      if (std::fscanf(f, "%f", &v) != 1 || !std::isfinite(v)) return bad("theta values");
    }
  }
  std::fclose(f);
  m->loaded = true;
  return GEMM_OK;
}

struct Row {
  int64_t M, N, K;
  int mode, cid;
  float ms;
};

gemm_status read_timings(const char* path, std::vector<Row>* rows) {
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(GEMM_ERR_IO, "cannot open %s", path);
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    TimingRow t;
    if (!parse_timing_row(line, &t)) continue;
    Row r;
    r.M = t.sh.M, r.N = t.sh.N, r.K = t.sh.K, r.mode = t.mode, r.cid = t.cid, r.ms = t.ms;
    if (r.M <= 0 || r.N <= 0 || r.K <= 0 || !(r.ms > 0.0f)) continue;
    if (r.cid < 0 || r.cid >= config_count((gemm_mode)r.mode)) continue;
    rows->push_back(r);
  }
  std::fclose(f);
  if (rows->empty()) return fail(GEMM_ERR_IO, "no timing rows in %s", path);
  return GEMM_OK;
}

}  // namespace

gemm_status costmodel_pick(gemm_mode mode, int64_t M, int64_t N, int64_t K, int* cid, float* ms) {
  Model m;
  {
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!g_model.loaded) return fail(GEMM_ERR_INVALID_ARG, "no cost model loaded");
    m = g_model;
  }
  const std::vector<int> ids = distinct_configs(mode, M, N, K);
  const int n = (int)ids.size();
  if (n == 0) return fail(GEMM_ERR_INVALID_ARG, "no candidate configuration");
  const int sms = sm_count();
  std::vector<float> X((size_t)n * kFeatures);
  gemm_config c;
  for (int i = 0; i < n; ++i) {
    config_get(ids[i], &c);
    costmodel_features(mode, M, N, K, c, sms, &X[(size_t)i * kFeatures]);
    for (int f = 0; f < kFeatures; ++f)
      X[(size_t)i * kFeatures + f] = (X[(size_t)i * kFeatures + f] - m.mean[f]) / m.stdv[f];
  }
  const int P = mlp_param_count();
  DevBuf dX, dth, dy;
  if (dX.alloc(X.size()) || dth.alloc(m.theta.size()) || dy.alloc((size_t)n * m.members)) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "cost-model prediction buffers");
  }
  cudaError_t e;
  if ((e = cudaMemcpy(dX.p, X.data(), X.size() * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(dth.p, m.theta.data(), m.theta.size() * 4, cudaMemcpyHostToDevice)))
    return cuda_fail(e, "cost-model upload");
  for (int k = 0; k < m.members; ++k)
    if ((e = mlp_forward_launch(dX.p, n, dth.p + (size_t)k * P, dy.p + (size_t)k * n, nullptr, nullptr,
                                nullptr)) != cudaSuccess)
      return cuda_fail(e, "cost-model forward");
  std::vector<float> ys((size_t)n * m.members), y(n, 0.0f);
  if ((e = cudaMemcpy(ys.data(), dy.p, ys.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cost-model prediction copy");
  for (int k = 0; k < m.members; ++k)
    for (int i = 0; i < n; ++i) y[i] += ys[(size_t)k * n + i] / m.members;
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (y[i] < y[best]) best = i;
  *cid = ids[best];
  *ms = std::exp(y[best] * m.ystd + m.ymean);
  return GEMM_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

int gemm_costmodel_feature_count(void) { return kFeatures; }

gemm_status gemm_costmodel_features(int64_t M, int64_t N, int64_t K, gemm_mode mode, int config_id,
                                    int sms, float* out) {
  clear_error();
  gemm_config c;
  if (!out || M <= 0 || N <= 0 || K <= 0 || sms <= 0) return fail(GEMM_ERR_INVALID_ARG, "bad arguments");
  if (config_count(mode) == 0 || !config_get(config_id, &c))
    return fail(GEMM_ERR_INVALID_ARG, "bad mode or configuration id");
  costmodel_features(mode, M, N, K, c, sms, out);
  return GEMM_OK;
}

gemm_status gemm_mlp_loss_grad(int n, const float* theta, const float* X, const float* t, float* loss,
                               float* grad) {
  clear_error();
  if (n <= 0 || !theta || !X || !t || !grad) return fail(GEMM_ERR_INVALID_ARG, "bad arguments");
  Pass ps;
  gemm_status st = ps.alloc(n);
  if (st != GEMM_OK) return st;
  const int P = mlp_param_count();
  cudaError_t e;
  if ((e = cudaMemcpy(ps.X.p, X, (size_t)n * kFeatures * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(ps.t.p, t, (size_t)n * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(ps.theta.p, theta, (size_t)P * 4, cudaMemcpyHostToDevice)))
    return cuda_fail(e, "upload");
  if ((st = loss_and_grad(ps, true, nullptr)) != GEMM_OK) return st;
  if ((e = cudaMemcpy(grad, ps.grad.p, (size_t)P * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "download gradient");
  if (loss && (e = cudaMemcpy(loss, ps.loss.p, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "download loss");
  return GEMM_OK;
}

gemm_status gemm_mlp_adam_step(int P, float* theta, const float* grad, float* m, float* v, int step,
                               float lr, float beta1, float beta2, float eps) {
  clear_error();
  if (P <= 0 || !theta || !grad || !m || !v || step < 1) return fail(GEMM_ERR_INVALID_ARG, "bad arguments");
  DevBuf a, b, c, d;
  if (a.alloc(P) || b.alloc(P) || c.alloc(P) || d.alloc(P)) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "adam buffers");
  }
  cudaError_t e;
  if ((e = cudaMemcpy(a.p, theta, P * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b.p, grad, P * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(c.p, m, P * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(d.p, v, P * 4, cudaMemcpyHostToDevice)) ||
      (e = adam_launch(a.p, b.p, c.p, d.p, P, step, lr, beta1, beta2, eps, nullptr)) ||
      (e = cudaMemcpy(theta, a.p, P * 4, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(m, c.p, P * 4, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(v, d.p, P * 4, cudaMemcpyDeviceToHost)))
    return cuda_fail(e, "adam step");
  return GEMM_OK;
}

gemm_status gemm_costmodel_train(const char* timings_path, int epochs, uint64_t seed,
                                 const char* out_model, float* final_loss) {
  clear_error();
  if (!timings_path || epochs < 1) return fail(GEMM_ERR_INVALID_ARG, "bad arguments");
  std::vector<Row> rows;
  gemm_status st = read_timings(timings_path, &rows);
  if (st != GEMM_OK) return st;
  const int n = (int)rows.size();
  const int sms = sm_count();
  std::vector<float> X((size_t)n * kFeatures), t(n);
  gemm_config c;
  for (int i = 0; i < n; ++i) {
    config_get(rows[i].cid, &c);
    costmodel_features((gemm_mode)rows[i].mode, rows[i].M, rows[i].N, rows[i].K, c, sms,
                       &X[(size_t)i * kFeatures]);
    t[i] = std::log(rows[i].ms);
  }
  Model m;
  m.mean.assign(kFeatures, 0.0f), m.stdv.assign(kFeatures, 1.0f);
  for (int f = 0; f < kFeatures; ++f) {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) s += X[(size_t)i * kFeatures + f];
    const double mu = s / n;
    for (int i = 0; i < n; ++i) {
      const double d = X[(size_t)i * kFeatures + f] - mu;
      s2 += d * d;
    }
    const double sd = std::sqrt(s2 / n);
    m.mean[f] = (float)mu;
    m.stdv[f] = sd > 1e-6 ? (float)sd : 1.0f;
    for (int i = 0; i < n; ++i)
      X[(size_t)i * kFeatures + f] = (float)((X[(size_t)i * kFeatures + f] - mu) / m.stdv[f]);
  }
  {
    double s = 0, s2 = 0;
    for (float v : t) s += v;
    const double mu = s / n;
    for (float v : t) s2 += (v - mu) * (v - mu);
    const double sd = std::sqrt(s2 / n);
    m.ymean = (float)mu;
    m.ystd = sd > 1e-6 ? (float)sd : 1.0f;
    for (float& v : t) v = (float)((v - mu) / m.ystd);
  }
  Pass ps;
  if ((st = ps.alloc(n)) != GEMM_OK) return st;
  const int P = mlp_param_count();
  DevBuf mom, var;
  if (mom.alloc(P) || var.alloc(P)) {
    cudaGetLastError();
    return fail(GEMM_ERR_ALLOC, "adam state");
  }
  cudaError_t e;
  if ((e = cudaMemcpy(ps.X.p, X.data(), X.size() * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(ps.t.p, t.data(), t.size() * 4, cudaMemcpyHostToDevice)))
    return cuda_fail(e, "upload training data");
  m.members = kMembers;
  m.theta.assign((size_t)kMembers * P, 0.0f);
  float loss_sum = 0.0f;
  for (int k = 0; k < kMembers; ++k) {
    // member k: its own initial weights, the same data and schedule
    const std::vector<float> th0 = init_params(splitmix64(seed + 0x632BE59BD9B4E019ull * (uint64_t)k));
    if ((e = cudaMemcpy(ps.theta.p, th0.data(), P * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(mom.p, 0, P * 4)) || (e = cudaMemset(var.p, 0, P * 4)))
      return cuda_fail(e, "upload initial weights");
    const float lr0 = 3e-3f;
    for (int step = 1; step <= epochs; ++step) {
      if ((st = loss_and_grad(ps, false, nullptr)) != GEMM_OK) return st;
      const double frac = (double)(step - 1) / epochs;
      const float lr = (float)(lr0 * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.14159265358979 * frac))));
      if ((e = adam_launch(ps.theta.p, ps.grad.p, mom.p, var.p, P, step, lr, 0.9f, 0.999f, 1e-8f, nullptr)))
        return cuda_fail(e, "adam");
    }
    if ((st = loss_and_grad(ps, true, nullptr)) != GEMM_OK) return st;
    float loss = 0;
    if ((e = cudaMemcpy(&loss, ps.loss.p, 4, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(m.theta.data() + (size_t)k * P, ps.theta.p, P * 4, cudaMemcpyDeviceToHost)))
      return cuda_fail(e, "download model");
    loss_sum += loss;
  }
  if (final_loss) *final_loss = loss_sum / kMembers;   // mean training loss of the members
  m.loaded = true;
  if (out_model && *out_model && (st = save_model(m, out_model)) != GEMM_OK) return st;
  std::lock_guard<std::mutex> lk(g_model_mu);
  g_model = m;
  return GEMM_OK;
}

gemm_status gemm_costmodel_load(const char* path) {
  clear_error();
  if (!path) return fail(GEMM_ERR_INVALID_ARG, "null path");
  Model m;
  gemm_status st = load_model(path, &m);
  if (st != GEMM_OK) return st;
  std::lock_guard<std::mutex> lk(g_model_mu);
  g_model = m;
  return GEMM_OK;
}

gemm_status gemm_costmodel_predict(int64_t M, int64_t N, int64_t K, gemm_mode mode, int* config_id,
                                   float* pred_ms) {
  clear_error();
  if (!config_id || M <= 0 || N <= 0 || K <= 0) return fail(GEMM_ERR_INVALID_ARG, "bad arguments");
  if (mode == GEMM_MODE_AUTO) mode = GEMM_MODE_BF16X3;
  if (config_count(mode) == 0) return fail(GEMM_ERR_INVALID_ARG, "mode has no configurations");
  float ms = 0;
  gemm_status st = costmodel_pick(mode, M, N, K, config_id, &ms);
  if (st == GEMM_OK && pred_ms) *pred_ms = ms;
  return st;
}

}  // extern "C"
