// costmodel.cpp - the learned launch-configuration cost model (host side).
//
// No counterpart in the paper, which names auto-tuning as future work (§8).
// The model maps 4 features of (stencil, grid side, dtype, tile) to the
// natural log of the sweep time in microseconds.  It is trained on the GPU by
// the kernels of mlp.cu (full-batch Adam, mean squared error) on timings the
// exhaustive autotuner produced, and it picks a tile by the argmin of its
// predictions.  It defers to the exhaustive autotuner when the shape lies
// outside the side range it was trained on, or when its two best
// predictions are closer than a margin.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../kernels/mlp.h"
#include "jacc_internal.h"

namespace jacc {

struct CostModel {
  float* d_p = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  unsigned* d_step = nullptr;
  float* d_partial = nullptr;
  float* d_losspart = nullptr;
  int cap_parts = 0;
  // pick buffers
  float* d_feat = nullptr;
  float* d_pred = nullptr;
  int* d_valid = nullptr;
  int* d_pick = nullptr;
  float* d_gap = nullptr;
  double side_lo = 0.0, side_hi = 1e300, margin = 0.0;
};

static bool g_mlp_ready = false;

static jacc_status ensure_setup() {
  if (g_mlp_ready) return ok();
  jacc_status st = cuda_check(mlp_setup(), "cudaFuncSetAttribute(MLP shared memory)");
  if (!st) g_mlp_ready = true;
  return st;
}

static jacc_status ensure_parts(CostModel& m, int n) {
  const int np = mlp_nparts(n);
  if (np <= m.cap_parts) return ok();
  if (m.d_partial) cudaFree(m.d_partial);
  if (m.d_losspart) cudaFree(m.d_losspart);
  m.d_partial = nullptr;
  m.d_losspart = nullptr;
  m.cap_parts = 0;
  jacc_status st =
      cuda_check(cudaMalloc(reinterpret_cast<void**>(&m.d_partial), sizeof(float) * JACC_MLP_NPARAM * (size_t)np),
                 "cudaMalloc(gradient partials)");
  if (!st) st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&m.d_losspart), sizeof(float) * (size_t)np), "cudaMalloc");
  if (!st) m.cap_parts = np;
  return st;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) on a counter: the same
// published generator the test-suite's inputs use, implemented here on its own.
static uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Kaiming-uniform initialisation for ReLU layers (He et al., ICCV 2015):
// W ~ U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)), biases 0.
static void kaiming_init(uint64_t seed, float* p) {
  const uint64_t key = mix64(mix64(seed));
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  const int fan[4] = {4, 64, 64, 64};
  const int off[4] = {0, 320, 4480, 8640};
  const int cnt[4] = {256, 4096, 4096, 64};
  std::memset(p, 0, sizeof(float) * JACC_MLP_NPARAM);
  uint64_t i = 0;
  for (int l = 0; l < 4; ++l) {
    const double b = std::sqrt(6.0 / fan[l]);
    for (int j = 0; j < cnt[l]; ++j) {
      const uint64_t bits = mix64(key + (++i) * G);
      const double u = static_cast<double>(bits >> 11) * 0x1p-53;
      p[off[l] + j] = static_cast<float>((2.0 * u - 1.0) * b);
    }
  }
}

}  // namespace jacc

using namespace jacc;

extern "C" jacc_status jacc_costmodel_features(int32_t stencil, double side, int32_t dtype, int32_t tile, float* out4) {
  if (!out4 || !(side > 0.0) || tile < 0 || tile >= JACC_NUM_TILES) return fail(JACC_ERR_INVALID_ARG, "bad feature args");
  out4[0] = static_cast<float>(stencil / 27.0);
  out4[1] = static_cast<float>(std::log2(side) / 10.0);
  out4[2] = static_cast<float>(dtype / 64.0);
  out4[3] = static_cast<float>(tile / 23.0);
  return ok();
}

extern "C" jacc_status jacc_costmodel_create(const float* init_params, uint64_t seed, jacc_costmodel* out) {
  if (!out) return fail(JACC_ERR_INVALID_ARG, "NULL output");
  jacc_status st = ensure_setup();
  if (st) return st;
  std::unique_ptr<CostModel> m(new CostModel());
  const size_t pb = sizeof(float) * JACC_MLP_NPARAM;
  char* blk = nullptr;
  st = cuda_check(cudaMalloc(&blk, 3 * pb + 256), "cudaMalloc(cost model)");
  if (st) return st;
  m->d_p = reinterpret_cast<float*>(blk);
  m->d_m = reinterpret_cast<float*>(blk + pb);
  m->d_v = reinterpret_cast<float*>(blk + 2 * pb);
  m->d_step = reinterpret_cast<unsigned*>(blk + 3 * pb);
  std::vector<float> p(JACC_MLP_NPARAM);
  if (init_params) std::memcpy(p.data(), init_params, pb);
  else kaiming_init(seed, p.data());
  st = cuda_check(cudaMemcpy(m->d_p, p.data(), pb, cudaMemcpyHostToDevice), "cudaMemcpy(params)");
  if (!st) st = cuda_check(cudaMemset(blk + pb, 0, 2 * pb + 256), "cudaMemset(Adam state)");
  if (st) {
    cudaFree(blk);
    return st;
  }
  *out = reinterpret_cast<jacc_costmodel>(m.release());
  return ok();
}

extern "C" jacc_status jacc_costmodel_set_params(jacc_costmodel h, const float* host_params) {
  if (!h || !host_params) return fail(JACC_ERR_INVALID_ARG, "NULL model or params");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  const size_t pb = sizeof(float) * JACC_MLP_NPARAM;
  jacc_status st = cuda_check(cudaMemcpy(m.d_p, host_params, pb, cudaMemcpyHostToDevice), "cudaMemcpy(params)");
  if (!st) st = cuda_check(cudaMemset(m.d_m, 0, 2 * pb + 256), "cudaMemset(Adam state)");
  return st;
}

extern "C" jacc_status jacc_costmodel_get_params(jacc_costmodel h, float* host_params) {
  if (!h || !host_params) return fail(JACC_ERR_INVALID_ARG, "NULL model or params");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  return cuda_check(cudaMemcpy(host_params, m.d_p, sizeof(float) * JACC_MLP_NPARAM, cudaMemcpyDeviceToHost),
                    "cudaMemcpy(params)");
}

extern "C" jacc_status jacc_costmodel_loss_grad(jacc_costmodel h, const float* x_dev, const float* y_dev, int32_t n,
                                                float* grad_dev, float* loss_dev, uintptr_t stream) {
  if (!h || !x_dev || !y_dev || n < 1 || !grad_dev) return fail(JACC_ERR_INVALID_ARG, "bad loss_grad arguments");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  jacc_status st = ensure_parts(m, n);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  st = cuda_check(mlp_fwd_bwd(m.d_p, x_dev, y_dev, n, m.d_partial, m.d_losspart, nullptr, s), "MLP forward/backward");
  if (st) return st;
  return cuda_check(mlp_adam(m.d_p, m.d_m, m.d_v, m.d_partial, mlp_nparts(n), m.d_losspart, n, loss_dev, nullptr, 0.f,
                             0.f, 0.f, 0.f, grad_dev, s),
                    "MLP gradient reduction");
}

extern "C" jacc_status jacc_costmodel_train(jacc_costmodel h, const float* x_dev, const float* y_dev, int32_t n,
                                            int32_t epochs, float lr, uintptr_t stream, float* loss_dev) {
  if (!h || !x_dev || !y_dev || n < 1 || epochs < 1 || !(lr > 0.f)) return fail(JACC_ERR_INVALID_ARG, "bad train args");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  jacc_status st = ensure_parts(m, n);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int np = mlp_nparts(n);
  auto step = [&](cudaStream_t q, float* lossp) -> jacc_status {
    jacc_status e = cuda_check(mlp_fwd_bwd(m.d_p, x_dev, y_dev, n, m.d_partial, m.d_losspart, m.d_step, q), "MLP fwd/bwd");
    if (e) return e;
    return cuda_check(mlp_adam(m.d_p, m.d_m, m.d_v, m.d_partial, np, m.d_losspart, n, lossp, m.d_step, lr, 0.9f,
                               0.999f, 1e-8f, nullptr, q),
                      "MLP Adam step");
  };
  // Capture a block of steps as one graph and replay it.
  const int K = epochs < 64 ? epochs : 64;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!st) st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  if (!st) {
    jacc_status est = ok();
    for (int k = 0; k < K && !est; ++k) est = step(cap, k == K - 1 ? loss_dev : nullptr);
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    st = est ? est : cuda_check(ce, "cudaStreamEndCapture");
    if (!st) st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
  }
  int done = 0;
  while (!st && done + K <= epochs) {
    st = cuda_check(cudaGraphLaunch(exec, s), "cudaGraphLaunch(train)");
    done += K;
  }
  while (!st && done < epochs) {
    st = step(s, done == epochs - 1 ? loss_dev : nullptr);
    ++done;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  return st;
}

extern "C" jacc_status jacc_costmodel_predict(jacc_costmodel h, const float* x_dev, int32_t n, float* y_dev,
                                              uintptr_t stream) {
  if (!h || !x_dev || !y_dev || n < 1) return fail(JACC_ERR_INVALID_ARG, "bad predict arguments");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  return cuda_check(mlp_forward(m.d_p, x_dev, n, y_dev, reinterpret_cast<cudaStream_t>(stream)), "MLP forward");
}

extern "C" jacc_status jacc_costmodel_pick(jacc_costmodel h, const float* feats_dev, const int32_t* valid_dev, int32_t nq,
                                           float* pred_dev, int32_t* pick_dev, float* gap_dev, uintptr_t stream) {
  if (!h || !feats_dev || !valid_dev || nq < 1 || !pred_dev || !pick_dev || !gap_dev)
    return fail(JACC_ERR_INVALID_ARG, "bad pick arguments");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  jacc_status st = cuda_check(mlp_forward(m.d_p, feats_dev, nq * JACC_NUM_TILES, pred_dev, s), "MLP forward");
  if (st) return st;
  return cuda_check(mlp_pick(pred_dev, valid_dev, nq, JACC_NUM_TILES, pick_dev, gap_dev, s), "MLP pick");
}

extern "C" jacc_status jacc_costmodel_set_range(jacc_costmodel h, double side_lo, double side_hi, double margin) {
  if (!h || !(side_lo > 0.0) || !(side_hi >= side_lo) || !(margin >= 0.0)) return fail(JACC_ERR_INVALID_ARG, "bad range");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  m.side_lo = side_lo;
  m.side_hi = side_hi;
  m.margin = margin;
  return ok();
}

extern "C" jacc_status jacc_costmodel_choose(jacc_costmodel h, const jacc_kernel_desc* desc, void* u0, void* u1,
                                             uintptr_t stream, int32_t* tile, int32_t* used_fallback) {
  if (!h || !desc || !tile || !used_fallback) return fail(JACC_ERR_INVALID_ARG, "bad choose arguments");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double vol = static_cast<double>(desc->nx) * desc->ny * desc->nz;
  const double side = desc->stencil == JACC_STENCIL_5PT ? std::sqrt(vol) : std::cbrt(vol);
  float feats[JACC_NUM_TILES * 4];
  int valid[JACC_NUM_TILES];
  for (int t = 0; t < JACC_NUM_TILES; ++t) {
    jacc_costmodel_features(desc->stencil, side, desc->dtype, t, feats + 4 * t);
    valid[t] = tile_valid(*desc, t) ? 1 : 0;
  }
  jacc_status st = ok();
  if (!m.d_feat) {
    char* blk = nullptr;
    st = cuda_check(cudaMalloc(&blk, 1024 + sizeof(feats) + 3 * sizeof(float) * JACC_NUM_TILES), "cudaMalloc(pick)");
    if (st) return st;
    m.d_feat = reinterpret_cast<float*>(blk);
    m.d_pred = reinterpret_cast<float*>(blk + sizeof(feats));
    m.d_valid = reinterpret_cast<int*>(blk + sizeof(feats) + sizeof(float) * JACC_NUM_TILES);
    m.d_pick = reinterpret_cast<int*>(blk + sizeof(feats) + 2 * sizeof(float) * JACC_NUM_TILES);
    m.d_gap = reinterpret_cast<float*>(blk + sizeof(feats) + 2 * sizeof(float) * JACC_NUM_TILES + 256);
  }
  st = cuda_check(cudaMemcpyAsync(m.d_feat, feats, sizeof(feats), cudaMemcpyHostToDevice, s), "upload features");
  if (!st) st = cuda_check(cudaMemcpyAsync(m.d_valid, valid, sizeof(valid), cudaMemcpyHostToDevice, s), "upload valid");
  if (!st) st = jacc_costmodel_pick(h, m.d_feat, m.d_valid, 1, m.d_pred, m.d_pick, m.d_gap, stream);
  int pick = -1;
  float gap = 0.f;
  if (!st) st = cuda_check(cudaMemcpyAsync(&pick, m.d_pick, sizeof(int), cudaMemcpyDeviceToHost, s), "read pick");
  if (!st) st = cuda_check(cudaMemcpyAsync(&gap, m.d_gap, sizeof(float), cudaMemcpyDeviceToHost, s), "read gap");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (st) return st;
  const bool outside = side < m.side_lo || side > m.side_hi;
  if (pick < 0 || outside || gap < m.margin) {
    if (!u0 || !u1) return fail(JACC_ERR_INVALID_ARG, "fallback to the exhaustive autotuner needs u0 and u1");
    jacc_tune_result r;
    st = jacc_autotune(desc, u0, u1, 2, 3, stream, &r);
    if (st) return st;
    *tile = r.best_tile;
    *used_fallback = 1;
    return ok();
  }
  *tile = pick;
  *used_fallback = 0;
  remember_tile(*desc, pick);
  return ok();
}

extern "C" jacc_status jacc_costmodel_choose_topk(jacc_costmodel h, const jacc_kernel_desc* desc, void* u0, void* u1,
                                                  uintptr_t stream, int32_t k, int32_t* tile) {
  if (!h || !desc || !tile || !u0 || !u1 || k < 1) return fail(JACC_ERR_INVALID_ARG, "bad choose_topk arguments");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double vol = static_cast<double>(desc->nx) * desc->ny * desc->nz;
  const double side = desc->stencil == JACC_STENCIL_5PT ? std::sqrt(vol) : std::cbrt(vol);
  float feats[JACC_NUM_TILES * 4];
  int valid[JACC_NUM_TILES];
  for (int t = 0; t < JACC_NUM_TILES; ++t) {
    jacc_costmodel_features(desc->stencil, side, desc->dtype, t, feats + 4 * t);
    valid[t] = tile_valid(*desc, t) ? 1 : 0;
  }
  float pred[JACC_NUM_TILES];
  jacc_status st = ok();
  float* d_feat = nullptr;
  st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&d_feat), sizeof(feats) + sizeof(pred)), "cudaMalloc(topk)");
  if (st) return st;
  float* d_pred = d_feat + JACC_NUM_TILES * 4;
  st = cuda_check(cudaMemcpyAsync(d_feat, feats, sizeof(feats), cudaMemcpyHostToDevice, s), "upload features");
  if (!st) st = jacc_costmodel_predict(h, d_feat, JACC_NUM_TILES, d_pred, stream);
  if (!st) st = cuda_check(cudaMemcpyAsync(pred, d_pred, sizeof(pred), cudaMemcpyDeviceToHost, s), "read predictions");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  cudaFree(d_feat);
  if (st) return st;
  // the k valid tiles with the lowest predicted time (ties to the lower id)
  std::vector<int32_t> order;
  for (int t = 0; t < JACC_NUM_TILES; ++t)
    if (valid[t]) order.push_back(t);
  if (order.empty()) return fail(JACC_ERR_UNSUPPORTED, "no tile configuration fits this shape");
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return pred[a] < pred[b]; });
  if (static_cast<int32_t>(order.size()) > k) order.resize(static_cast<size_t>(k));
  jacc_tune_result r;
  st = jacc_autotune_tiles(desc, u0, u1, 2, 3, stream, order.data(), static_cast<int32_t>(order.size()), &r);
  if (st) return st;
  *tile = r.best_tile;
  return ok();
}

// ---------------------------------------------------------------- pipeline from autotuner tables

namespace jacc {

static bool table_ok(const jacc_tune_table& q) {
  return (q.stencil == 5 || q.stencil == 7 || q.stencil == 27) && (q.dtype == 32 || q.dtype == 64) && q.side > 0.0;
}

// Predictions for every (query, tile) of the tables: pred[q * 24 + t].
static jacc_status predict_tables(jacc_costmodel h, int32_t nq, const jacc_tune_table* tables, cudaStream_t s,
                                  std::vector<float>& pred) {
  const size_t rows = static_cast<size_t>(nq) * JACC_NUM_TILES;
  std::vector<float> feats(rows * 4);
  for (int32_t q = 0; q < nq; ++q)
    for (int t = 0; t < JACC_NUM_TILES; ++t)
      jacc_costmodel_features(tables[q].stencil, tables[q].side, tables[q].dtype, t, &feats[(q * JACC_NUM_TILES + t) * 4]);
  float* d = nullptr;
  jacc_status st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&d), sizeof(float) * rows * 5), "cudaMalloc(eval)");
  if (st) return st;
  pred.resize(rows);
  st = cuda_check(cudaMemcpyAsync(d, feats.data(), sizeof(float) * rows * 4, cudaMemcpyHostToDevice, s), "upload");
  if (!st) st = jacc_costmodel_predict(h, d, static_cast<int32_t>(rows), d + rows * 4, reinterpret_cast<uintptr_t>(s));
  if (!st)
    st = cuda_check(cudaMemcpyAsync(pred.data(), d + rows * 4, sizeof(float) * rows, cudaMemcpyDeviceToHost, s), "read");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  cudaFree(d);
  return st;
}

// Valid tiles of one query ordered by prediction (ties to the lower tile).
static std::vector<int> ranked(const jacc_tune_table& q, const float* pred) {
  std::vector<int> order;
  for (int t = 0; t < JACC_NUM_TILES; ++t)
    if (q.valid[t]) order.push_back(t);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pred[a] < pred[b]; });
  return order;
}

static double best_ms(const jacc_tune_table& q) {
  double b = 1e300;
  for (int t = 0; t < JACC_NUM_TILES; ++t)
    if (q.valid[t] && q.ms[t] < b) b = q.ms[t];
  return b;
}

}  // namespace jacc

extern "C" jacc_status jacc_costmodel_fit_tables(jacc_costmodel h, int32_t nq, const jacc_tune_table* tables,
                                                 int32_t epochs, float lr, uintptr_t stream, double* final_mse) {
  if (!h || nq < 1 || !tables || epochs < 1 || !(lr > 0.f)) return fail(JACC_ERR_INVALID_ARG, "bad fit_tables arguments");
  std::vector<float> X, Y;
  for (int32_t q = 0; q < nq; ++q) {
    const jacc_tune_table& T = tables[q];
    if (!table_ok(T)) return fail(JACC_ERR_INVALID_ARG, "bad table row " + std::to_string(q));
    double sum = 0.0;
    int n = 0;
    for (int t = 0; t < JACC_NUM_TILES; ++t)
      if (T.valid[t]) {
        if (!(T.ms[t] > 0.0) || !std::isfinite(T.ms[t]))
          return fail(JACC_ERR_INVALID_ARG, "a valid tile needs a finite positive time");
        sum += std::log(T.ms[t] * 1e3);
        ++n;
      }
    if (n == 0) continue;
    const double mean = sum / n;
    for (int t = 0; t < JACC_NUM_TILES; ++t)
      if (T.valid[t]) {
        float f[4];
        jacc_costmodel_features(T.stencil, T.side, T.dtype, t, f);
        X.insert(X.end(), f, f + 4);
        Y.push_back(static_cast<float>(std::log(T.ms[t] * 1e3) - mean));
      }
  }
  if (Y.empty()) return fail(JACC_ERR_INVALID_ARG, "no valid (query, tile) pair to train on");
  const size_t n = Y.size();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* d = nullptr;
  jacc_status st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&d), sizeof(float) * (5 * n + 1)), "cudaMalloc(fit)");
  if (st) return st;
  st = cuda_check(cudaMemcpyAsync(d, X.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice, s), "upload features");
  if (!st) st = cuda_check(cudaMemcpyAsync(d + 4 * n, Y.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s), "upload targets");
  if (!st) st = jacc_costmodel_train(h, d, d + 4 * n, static_cast<int32_t>(n), epochs, lr, stream, d + 5 * n);
  float loss = 0.f;
  if (!st) st = cuda_check(cudaMemcpyAsync(&loss, d + 5 * n, sizeof(float), cudaMemcpyDeviceToHost, s), "read loss");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  cudaFree(d);
  if (!st && final_mse) *final_mse = loss;
  return st;
}

extern "C" jacc_status jacc_costmodel_evaluate(jacc_costmodel h, int32_t nq, const jacc_tune_table* tables, double margin,
                                               int32_t topk, uintptr_t stream, jacc_costmodel_eval* out) {
  if (!h || nq < 1 || !tables || !out || topk < 1 || !(margin >= 0.0))
    return fail(JACC_ERR_INVALID_ARG, "bad evaluate arguments");
  for (int32_t q = 0; q < nq; ++q)
    if (!table_ok(tables[q])) return fail(JACC_ERR_INVALID_ARG, "bad table row " + std::to_string(q));
  std::vector<float> pred;
  jacc_status st = predict_tables(h, nq, tables, reinterpret_cast<cudaStream_t>(stream), pred);
  if (st) return st;
  for (int32_t q = 0; q < nq; ++q) {
    const jacc_tune_table& T = tables[q];
    const std::vector<int> order = ranked(T, &pred[static_cast<size_t>(q) * JACC_NUM_TILES]);
    jacc_costmodel_eval& e = out[q];
    if (order.empty()) {
      e = jacc_costmodel_eval{-1, 1, 0.0, 0.0, 0.0, 0.0};
      continue;
    }
    const float* pq = &pred[static_cast<size_t>(q) * JACC_NUM_TILES];
    const double best = best_ms(T);
    e.pick = order[0];
    e.gap = order.size() > 1 ? static_cast<double>(pq[order[1]]) - static_cast<double>(pq[order[0]]) : 1e300;
    e.fallback = e.gap < margin ? 1 : 0;
    e.regret = T.ms[e.pick] / best - 1.0;
    const size_t k = std::min<size_t>(static_cast<size_t>(topk), order.size());
    double fastest = 1e300, cost = 0.0;
    for (size_t i = 0; i < k; ++i) {
      fastest = std::min(fastest, T.ms[order[i]]);
      cost += T.ms[order[i]];
    }
    e.regret_topk = fastest / best - 1.0;
    e.search_ms_topk = cost;
  }
  return ok();
}

extern "C" jacc_status jacc_costmodel_fixed_tile(int32_t nq, const jacc_tune_table* tables, int32_t* tile) {
  if (nq < 1 || !tables || !tile) return fail(JACC_ERR_INVALID_ARG, "bad fixed_tile arguments");
  int best = -1;
  double best_mean = 1e300;
  for (int t = 0; t < JACC_NUM_TILES; ++t) {
    double sum = 0.0;
    bool everywhere = true;
    for (int32_t q = 0; q < nq && everywhere; ++q) {
      if (!tables[q].valid[t] || !(tables[q].ms[t] > 0.0)) everywhere = false;
      else sum += std::log(tables[q].ms[t]);
    }
    if (everywhere && sum / nq < best_mean) {
      best_mean = sum / nq;
      best = t;
    }
  }
  if (best < 0) return fail(JACC_ERR_UNSUPPORTED, "no tile is valid for every query");
  *tile = best;
  return ok();
}

extern "C" jacc_status jacc_costmodel_regret(int32_t nq, const jacc_tune_table* tables, const int32_t* picks,
                                             double* regret) {
  if (nq < 1 || !tables || !picks || !regret) return fail(JACC_ERR_INVALID_ARG, "bad regret arguments");
  for (int32_t q = 0; q < nq; ++q) {
    const int32_t p = picks[q];
    if (p < 0 || p >= JACC_NUM_TILES || !tables[q].valid[p])
      return fail(JACC_ERR_INVALID_ARG, "pick " + std::to_string(p) + " is not a valid tile of query " + std::to_string(q));
    regret[q] = tables[q].ms[p] / best_ms(tables[q]) - 1.0;
  }
  return ok();
}

extern "C" jacc_status jacc_costmodel_margin(jacc_costmodel h, int32_t nq, const jacc_tune_table* tables, double fraction,
                                             uintptr_t stream, double* margin) {
  if (!h || nq < 1 || !tables || !margin || !(fraction >= 0.0 && fraction <= 1.0))
    return fail(JACC_ERR_INVALID_ARG, "bad margin arguments");
  std::vector<jacc_costmodel_eval> ev(static_cast<size_t>(nq));
  jacc_status st = jacc_costmodel_evaluate(h, nq, tables, 0.0, 1, stream, ev.data());
  if (st) return st;
  std::vector<double> gaps;
  for (const auto& e : ev)
    if (e.pick >= 0) gaps.push_back(e.gap);
  std::sort(gaps.begin(), gaps.end());
  // the largest g with #{gap < g} < fraction * nq: the gap of rank floor(fraction * nq)
  const size_t r = static_cast<size_t>(std::floor(fraction * static_cast<double>(gaps.size())));
  *margin = (r == 0 || gaps.empty()) ? 0.0 : gaps[std::min(r, gaps.size()) - 1];
  return ok();
}

extern "C" jacc_status jacc_costmodel_save(jacc_costmodel h, const char* path) {
  if (!h || !path) return fail(JACC_ERR_INVALID_ARG, "NULL model or path");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  std::vector<float> p(JACC_MLP_NPARAM);
  jacc_status st = jacc_costmodel_get_params(h, p.data());
  if (st) return st;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(JACC_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const char magic[8] = {'J', 'A', 'C', 'C', 'M', 'L', 'P', '1'};
  const double range[3] = {m.side_lo, m.side_hi, m.margin};
  bool okw = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(range, sizeof(double), 3, f) == 3 &&
             std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
  okw = (std::fclose(f) == 0) && okw;
  return okw ? ok() : fail(JACC_ERR_INVALID_ARG, std::string("short write to ") + path);
}

extern "C" jacc_status jacc_costmodel_load(jacc_costmodel h, const char* path) {
  if (!h || !path) return fail(JACC_ERR_INVALID_ARG, "NULL model or path");
  CostModel& m = *reinterpret_cast<CostModel*>(h);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(JACC_ERR_INVALID_ARG, std::string("cannot open ") + path);
  char magic[8];
  double range[3];
  std::vector<float> p(JACC_MLP_NPARAM);
  bool okr = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "JACCMLP1", 8) == 0 &&
             std::fread(range, sizeof(double), 3, f) == 3 && std::fread(p.data(), sizeof(float), p.size(), f) == p.size();
  std::fclose(f);
  if (!okr) return fail(JACC_ERR_INVALID_ARG, std::string("not a cost-model file: ") + path);
  m.side_lo = range[0];
  m.side_hi = range[1];
  m.margin = range[2];
  return jacc_costmodel_set_params(h, p.data());
}

extern "C" jacc_status jacc_costmodel_release(jacc_costmodel h) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL model");
  CostModel* m = reinterpret_cast<CostModel*>(h);
  if (m->d_p) cudaFree(m->d_p);
  if (m->d_partial) cudaFree(m->d_partial);
  if (m->d_losspart) cudaFree(m->d_losspart);
  if (m->d_feat) cudaFree(m->d_feat);
  delete m;
  return ok();
}
