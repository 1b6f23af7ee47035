// batch.cpp - plans, tuning and graph-captured runs of the batched persistent launch.
//
// A plan holds the device tables of one batch (grids, the schedule's item
// table, per-grid counters and fixed-point scale words) in one allocation.
// The schedule has three knobs: points per item (band height), persistent
// CTAs per SM, and the item order; jacc_batch_tune times every candidate on
// the caller's buffers and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../kernels/batched.h"
#include "jacc_internal.h"

namespace jacc {

struct Batch {
  std::vector<jacc_grid> grids;
  jacc_batch_config cfg{};
  int sms = 0;
  int max_ctas_per_sm = 0;
  int nctas = 0;
  int total_items = 0;
  std::vector<int> nitems;  // items per grid under the current schedule
  i64 max_n = 0;
  // device block: [ticket u64][status i32][pad][done u32 x ngrids] [maxwords] [grids] [items]
  char* block = nullptr;
  size_t counters_bytes = 0;
  unsigned long long* d_ticket = nullptr;
  int* d_status = nullptr;
  unsigned* d_done = nullptr;
  u64* d_maxwords = nullptr;
  JBGrid* d_grids = nullptr;
  JBItem* d_items = nullptr;
  std::map<std::pair<int32_t, const double*>, SweepGraph> graphs;
};

static void drop_graphs(Batch& b) {
  for (auto& g : b.graphs) {
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (g.second.graph) cudaGraphDestroy(g.second.graph);
  }
  b.graphs.clear();
}

static int jacc_config_default(jacc_batch_config* c) {
  c->item_points = 16384;
  c->ctas_per_sm = 0;
  c->order = 0;
  c->timeout_ms = 2000;
  c->test_stall_ticket = -1;
  return 0;
}

// Builds the host tables for cfg and uploads them (synchronously).
static jacc_status plan(Batch& b, const jacc_batch_config& in) {
  jacc_batch_config c = in;
  if (c.item_points <= 0) c.item_points = 16384;
  if (c.timeout_ms <= 0) c.timeout_ms = 2000;
  if (c.order != 0 && c.order != 1) return fail(JACC_ERR_INVALID_ARG, "batch order must be 0 or 1");
  if (c.ctas_per_sm < 0) return fail(JACC_ERR_INVALID_ARG, "ctas_per_sm < 0");
  const int ng = static_cast<int>(b.grids.size());
  std::vector<JBGrid> hg(ng);
  for (int g = 0; g < ng; ++g) {
    const jacc_grid& G = b.grids[g];
    JBGrid& d = hg[g];
    d.u[0] = static_cast<double*>(G.u0);
    d.u[1] = static_cast<double*>(G.u1);
    d.nx = G.nx;
    d.ny = G.ny;
    d.rows = std::max<i64>(1, std::min<i64>(G.ny, c.item_points / G.nx));
    d.nitems = static_cast<int>((G.ny + d.rows - 1) / d.rows);
    d.vec = (G.nx % 2 == 0) ? 2 : 1;
  }
  // item order
  std::vector<int> byarea(ng);
  std::iota(byarea.begin(), byarea.end(), 0);
  std::stable_sort(byarea.begin(), byarea.end(),
                   [&](int a, int z) { return hg[a].nx * hg[a].ny > hg[z].nx * hg[z].ny; });
  std::vector<JBItem> items;
  if (c.order == 0) {
    for (int g : byarea)
      for (int i = 0; i < hg[g].nitems; ++i) items.push_back({g, i});
  } else {
    int maxi = 0;
    for (int g = 0; g < ng; ++g) maxi = std::max(maxi, hg[g].nitems);
    for (int i = 0; i < maxi; ++i)
      for (int g : byarea)
        if (i < hg[g].nitems) items.push_back({g, i});
  }
  if (items.size() > (1u << 30)) return fail(JACC_ERR_UNSUPPORTED, "too many items");
  const int per_sm = c.ctas_per_sm == 0 ? b.max_ctas_per_sm : std::min(c.ctas_per_sm, b.max_ctas_per_sm);
  if (per_sm < 1) return fail(JACC_ERR_UNSUPPORTED, "the batched kernel does not fit on an SM");

  const size_t n_items = items.size();
  const size_t cb = 16 + sizeof(unsigned) * static_cast<size_t>(ng);
  const size_t counters_bytes = (cb + 255) / 256 * 256;
  const size_t mw_bytes = (sizeof(u64) * ng + 255) / 256 * 256;
  const size_t g_bytes = (sizeof(JBGrid) * ng + 255) / 256 * 256;
  const size_t it_bytes = sizeof(JBItem) * n_items;
  char* blk = nullptr;
  jacc_status st = cuda_check(cudaMalloc(&blk, counters_bytes + mw_bytes + g_bytes + it_bytes), "cudaMalloc(batch)");
  if (st) return st;
  st = cuda_check(cudaMemcpy(blk + counters_bytes + mw_bytes, hg.data(), sizeof(JBGrid) * ng, cudaMemcpyHostToDevice),
                  "cudaMemcpy(batch grids)");
  if (!st)
    st = cuda_check(cudaMemcpy(blk + counters_bytes + mw_bytes + g_bytes, items.data(), it_bytes, cudaMemcpyHostToDevice),
                    "cudaMemcpy(batch items)");
  if (st) {
    cudaFree(blk);
    return st;
  }
  drop_graphs(b);
  if (b.block) cudaFree(b.block);
  b.block = blk;
  b.counters_bytes = counters_bytes;
  b.d_ticket = reinterpret_cast<unsigned long long*>(blk);
  b.d_status = reinterpret_cast<int*>(blk + 8);
  b.d_done = reinterpret_cast<unsigned*>(blk + 16);
  b.d_maxwords = reinterpret_cast<u64*>(blk + counters_bytes);
  b.d_grids = reinterpret_cast<JBGrid*>(blk + counters_bytes + mw_bytes);
  b.d_items = reinterpret_cast<JBItem*>(blk + counters_bytes + mw_bytes + g_bytes);
  b.total_items = static_cast<int>(n_items);
  b.nitems.resize(ng);
  for (int g = 0; g < ng; ++g) b.nitems[g] = hg[g].nitems;
  b.nctas = per_sm * b.sms;
  b.cfg = c;
  b.cfg.ctas_per_sm = per_sm;
  return ok();
}

static jacc_status enqueue(Batch& b, int32_t nsweeps, double* resid, cudaStream_t s) {
  const int ng = static_cast<int>(b.grids.size());
  jacc_status st = cuda_check(cudaMemsetAsync(b.block, 0, b.counters_bytes, s), "memset batch counters");
  if (st) return st;
  if (resid) {
    st = cuda_check(cudaMemsetAsync(resid, 0, sizeof(double) * static_cast<size_t>(ng) * nsweeps, s), "memset resid");
    if (st) return st;
  }
  st = cuda_check(launch_maxabs_batched(b.d_grids, ng, b.max_n, b.d_maxwords, s), "batched max-abs pre-pass");
  if (st) return st;
  JBatchParams bp{};
  bp.grids = b.d_grids;
  bp.items = b.d_items;
  bp.ngrids = ng;
  bp.total_items = b.total_items;
  bp.nsweeps = nsweeps;
  bp.maxwords = b.d_maxwords;
  bp.done = b.d_done;
  bp.ticket = b.d_ticket;
  bp.status = b.d_status;
  bp.resid = resid;
  bp.timeout_ns = static_cast<u64>(b.cfg.timeout_ms) * 1000000ull;
  bp.stall_ticket = b.cfg.test_stall_ticket;
  return cuda_check(launch_batched(bp, b.nctas, s), "batched persistent launch");
}

}  // namespace jacc

using namespace jacc;

extern "C" jacc_status jacc_batch_create(int32_t ngrids, const jacc_grid* grids, const jacc_batch_config* cfg,
                                         jacc_batch* out) {
  if (ngrids < 1 || !grids || !out) return fail(JACC_ERR_INVALID_ARG, "need ngrids >= 1, grids and out");
  for (int g = 0; g < ngrids; ++g) {
    const jacc_grid& G = grids[g];
    if (G.nx < 3 || G.ny < 3) return fail(JACC_ERR_INVALID_ARG, "grid extents must be >= 3");
    if (G.nx > (1ll << 31) || G.ny > (1ll << 31)) return fail(JACC_ERR_UNSUPPORTED, "grid extent above 2^31");
    if (!G.u0 || !G.u1) return fail(JACC_ERR_INVALID_ARG, "NULL grid field");
    if ((reinterpret_cast<uintptr_t>(G.u0) % 16) || (reinterpret_cast<uintptr_t>(G.u1) % 16))
      return fail(JACC_ERR_INVALID_ARG, "grid fields must be 16-byte aligned");
    const uintptr_t bytes = static_cast<uintptr_t>(G.nx * G.ny) * 8;
    const uintptr_t a = reinterpret_cast<uintptr_t>(G.u0), z = reinterpret_cast<uintptr_t>(G.u1);
    if (a < z + bytes && z < a + bytes) return fail(JACC_ERR_INVALID_ARG, "grid fields u0 and u1 overlap");
  }
  std::unique_ptr<Batch> b(new Batch());
  b->grids.assign(grids, grids + ngrids);
  for (const auto& G : b->grids) b->max_n = std::max<i64>(b->max_n, G.nx * G.ny);
  int dev = 0;
  jacc_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (!st) st = cuda_check(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  int coop = 0;
  if (!st) st = cuda_check(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "cooperative attr");
  if (st) return st;
  if (!coop) return fail(JACC_ERR_UNSUPPORTED, "device lacks cooperative launch");
  st = cuda_check(batched_occupancy(&b->max_ctas_per_sm), "occupancy of the batched kernel");
  if (st) return st;
  jacc_batch_config c;
  jacc_config_default(&c);
  if (cfg) c = *cfg;
  st = plan(*b, c);
  if (st) return st;
  *out = reinterpret_cast<jacc_batch>(b.release());
  return ok();
}

extern "C" jacc_status jacc_batch_configure(jacc_batch h, const jacc_batch_config* cfg) {
  if (!h || !cfg) return fail(JACC_ERR_INVALID_ARG, "NULL batch or config");
  std::lock_guard<std::mutex> lock(global_mutex());
  return plan(*reinterpret_cast<Batch*>(h), *cfg);
}

extern "C" jacc_status jacc_batch_get_config(jacc_batch h, jacc_batch_config* out) {
  if (!h || !out) return fail(JACC_ERR_INVALID_ARG, "NULL batch or output");
  *out = reinterpret_cast<Batch*>(h)->cfg;
  return ok();
}

extern "C" jacc_status jacc_batch_sweep(jacc_batch h, int32_t nsweeps, double* resid_dev, uint32_t flags,
                                        uintptr_t stream, int32_t* final_buf) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL batch");
  if (nsweeps < 1) return fail(JACC_ERR_INVALID_ARG, "nsweeps must be >= 1");
  if (flags & ~JACC_SWEEP_GRAPH) return fail(JACC_ERR_INVALID_ARG, "unknown sweep flags");
  Batch& b = *reinterpret_cast<Batch*>(h);
  for (int n : b.nitems)
    if (static_cast<double>(nsweeps) * static_cast<double>(n) > 2.0e9)
      return fail(JACC_ERR_UNSUPPORTED, "nsweeps x items of a grid exceeds the 32-bit completion counter");
  if (static_cast<double>(nsweeps) * static_cast<double>(b.total_items) > 4.0e18)
    return fail(JACC_ERR_UNSUPPORTED, "ticket count overflows");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (final_buf) *final_buf = nsweeps % 2;
  if (!(flags & JACC_SWEEP_GRAPH)) return enqueue(b, nsweeps, resid_dev, s);
  std::lock_guard<std::mutex> lock(global_mutex());
  const auto key = std::make_pair(nsweeps, static_cast<const double*>(resid_dev));
  auto it = b.graphs.find(key);
  if (it == b.graphs.end()) {
    SweepGraph g;
    cudaStream_t cap = nullptr;
    jacc_status st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (!st) {
      jacc_status est = enqueue(b, nsweeps, resid_dev, cap);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(cap, &graph);
      st = est ? est : cuda_check(ce, "cudaStreamEndCapture");
      g.graph = graph;
      if (!st) st = cuda_check(cudaGraphInstantiate(&g.exec, g.graph, 0), "cudaGraphInstantiate");
    }
    if (cap) cudaStreamDestroy(cap);
    if (st) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      return st;
    }
    it = b.graphs.emplace(key, g).first;
  }
  return cuda_check(cudaGraphLaunch(it->second.exec, s), "cudaGraphLaunch(batch)");
}

extern "C" jacc_status jacc_batch_status(jacc_batch h, uintptr_t stream) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL batch");
  Batch& b = *reinterpret_cast<Batch*>(h);
  jacc_status st = cuda_check(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "cudaStreamSynchronize");
  if (st) return st;
  int v = 0;
  st = cuda_check(cudaMemcpy(&v, b.d_status, sizeof(int), cudaMemcpyDeviceToHost), "read batch status");
  if (st) return st;
  if (v == JACC_ERR_TIMEOUT) return fail(JACC_ERR_TIMEOUT, "a batched-sweep wait exceeded its time limit");
  if (v != 0) return fail(JACC_ERR_CUDA, "unexpected batch status " + std::to_string(v));
  return ok();
}

extern "C" jacc_status jacc_batch_tune(jacc_batch h, int32_t probe_sweeps, uintptr_t stream, jacc_batch_config* best,
                                       double* best_ms) {
  if (!h || probe_sweeps < 1) return fail(JACC_ERR_INVALID_ARG, "NULL batch or probe_sweeps < 1");
  Batch& b = *reinterpret_cast<Batch*>(h);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const jacc_batch_config base = b.cfg;
  std::vector<int> per_sm = {1, 2, b.max_ctas_per_sm};
  std::sort(per_sm.begin(), per_sm.end());
  per_sm.erase(std::unique(per_sm.begin(), per_sm.end()), per_sm.end());
  cudaEvent_t e0, e1;
  jacc_status st = cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
  if (st) return st;
  st = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  if (st) {
    cudaEventDestroy(e0);
    return st;
  }
  double best_t = 1e300;
  jacc_batch_config best_c = base;
  for (int pts : {4096, 8192, 16384, 32768, 65536}) {
    for (int p : per_sm) {
      if (p > b.max_ctas_per_sm || p < 1) continue;
      for (int order : {0, 1}) {
        jacc_batch_config c = base;
        c.item_points = pts;
        c.ctas_per_sm = p;
        c.order = order;
        c.test_stall_ticket = -1;
        {
          std::lock_guard<std::mutex> lock(global_mutex());
          st = plan(b, c);
        }
        if (st) break;
        double t = 1e300;
        for (int rep = 0; rep < 3 && !st; ++rep) {
          st = cuda_check(cudaEventRecord(e0, s), "cudaEventRecord");
          if (!st) st = enqueue(b, probe_sweeps, nullptr, s);
          if (!st) st = cuda_check(cudaEventRecord(e1, s), "cudaEventRecord");
          if (!st) st = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
          float ms = 0;
          if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
          if (!st && rep > 0) t = std::min(t, static_cast<double>(ms));  // rep 0 warms up
        }
        if (!st) st = jacc_batch_status(h, stream);
        if (st) break;
        if (t < best_t) {
          best_t = t;
          best_c = b.cfg;
        }
      }
      if (st) break;
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lock(global_mutex());
    st = plan(b, best_c);
  }
  if (st) return st;
  if (best) *best = b.cfg;
  if (best_ms) *best_ms = best_t;
  return ok();
}

extern "C" jacc_status jacc_batch_release(jacc_batch h) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL batch");
  Batch* b = reinterpret_cast<Batch*>(h);
  {
    std::lock_guard<std::mutex> lock(global_mutex());
    drop_graphs(*b);
  }
  if (b->block) cudaFree(b->block);
  delete b;
  return ok();
}
