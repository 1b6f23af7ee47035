// autotune.cpp - exhaustive autotuner over the 24 tile configurations.
//
// Auto-tuning is named as future work in the paper (§8); OptACC's grid
// search over OpenACC parallelism is the related prior art it cites (§7).
// For one descriptor the tuner specialises each valid tile, runs a
// graph-captured sweep sequence once to warm up, times `reps` further runs
// with CUDA events on the caller's stream and keeps the median per sweep.
// The fastest tile is remembered per shape, so that later jacc_specialize
// calls with tile_id = -1 use it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "jacc_internal.h"

namespace jacc {

static std::map<std::string, int>& tune_cache() {
  static std::map<std::string, int> c;
  return c;
}

std::string shape_key(const jacc_kernel_desc& d) {
  jacc_kernel_desc c = d;
  c.tile_id = -1;
  c.flags = 0;
  c.reserved = 0;
  if (c.tblock == 0) c.tblock = 1;
  return std::string(reinterpret_cast<const char*>(&c), sizeof(c));
}

int tuned_tile(const jacc_kernel_desc& d) {
  std::lock_guard<std::mutex> lock(global_mutex());
  auto it = tune_cache().find(shape_key(d));
  return it == tune_cache().end() ? -1 : it->second;
}

void remember_tile(const jacc_kernel_desc& d, int tile) {
  std::lock_guard<std::mutex> lock(global_mutex());
  tune_cache()[shape_key(d)] = tile;
}

}  // namespace jacc

using namespace jacc;

// Times the tiles with want[t] set (each valid one), fills `out`, remembers
// the fastest for the shape.
static jacc_status autotune_subset(const jacc_kernel_desc* desc, void* u0, void* u1, int32_t sweeps_per_rep,
                                   int32_t reps, uintptr_t stream, const bool* want, jacc_tune_result* out) {
  if (!desc || !out || sweeps_per_rep < 1 || reps < 1) return fail(JACC_ERR_INVALID_ARG, "bad autotune arguments");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  jacc_status st = cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
  if (st) return st;
  st = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  if (st) {
    cudaEventDestroy(e0);
    return st;
  }
  out->best_tile = -1;
  out->best_ms = std::numeric_limits<double>::infinity();
  for (int t = 0; t < JACC_NUM_TILES && !st; ++t) {
    out->ms[t] = std::numeric_limits<double>::infinity();
    out->valid[t] = 0;
    jacc_kernel_desc d = *desc;
    d.tile_id = t;
    d.flags &= ~JACC_SPEC_JIT;
    if (!want[t] || !tile_valid(d, t)) continue;
    jacc_kernel k = nullptr;
    st = jacc_specialize(&d, &k);
    if (st) break;
    std::vector<double> times;
    int32_t fb = 0;
    for (int r = 0; r <= reps && !st; ++r) {
      st = cuda_check(cudaEventRecord(e0, s), "cudaEventRecord");
      if (!st) st = jacc_sweep(k, u0, u1, sweeps_per_rep, nullptr, JACC_SWEEP_GRAPH, stream, &fb);
      if (!st) st = cuda_check(cudaEventRecord(e1, s), "cudaEventRecord");
      if (!st) st = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (!st && r > 0) times.push_back(static_cast<double>(ms) / sweeps_per_rep);  // run 0 warms up
    }
    jacc_release(k);
    if (st) break;
    std::sort(times.begin(), times.end());
    out->ms[t] = times[times.size() / 2];
    out->valid[t] = 1;
    if (out->ms[t] < out->best_ms) {
      out->best_ms = out->ms[t];
      out->best_tile = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if (out->best_tile < 0) return fail(JACC_ERR_UNSUPPORTED, "no tile configuration fits this shape");
  std::lock_guard<std::mutex> lock(global_mutex());
  tune_cache()[shape_key(*desc)] = out->best_tile;
  return ok();
}

extern "C" jacc_status jacc_autotune(const jacc_kernel_desc* desc, void* u0, void* u1, int32_t sweeps_per_rep,
                                     int32_t reps, uintptr_t stream, jacc_tune_result* out) {
  bool all[JACC_NUM_TILES];
  std::fill(all, all + JACC_NUM_TILES, true);
  return autotune_subset(desc, u0, u1, sweeps_per_rep, reps, stream, all, out);
}

extern "C" jacc_status jacc_autotune_tiles(const jacc_kernel_desc* desc, void* u0, void* u1, int32_t sweeps_per_rep,
                                           int32_t reps, uintptr_t stream, const int32_t* tiles, int32_t ntiles,
                                           jacc_tune_result* out) {
  if (!tiles || ntiles < 1) return fail(JACC_ERR_INVALID_ARG, "no tiles to time");
  bool want[JACC_NUM_TILES];
  std::fill(want, want + JACC_NUM_TILES, false);
  for (int32_t i = 0; i < ntiles; ++i) {
    if (tiles[i] < 0 || tiles[i] >= JACC_NUM_TILES) return fail(JACC_ERR_INVALID_ARG, "tile id out of range");
    want[tiles[i]] = true;
  }
  return autotune_subset(desc, u0, u1, sweeps_per_rep, reps, stream, want, out);
}

extern "C" jacc_status jacc_autotune_forget(void) {
  std::lock_guard<std::mutex> lock(global_mutex());
  tune_cache().clear();
  return ok();
}
