// batch.cpp - plans, tuning and graph-captured runs of the batched persistent launch.
//
// A plan cuts every grid into items (tiles of rows x cols points), packs the
// grids into groups whose two fields fit an L2 budget together, and lays out
// the item table group by group; it holds the device tables (counters,
// per-grid scale words, grids, items, groups) in one allocation.  Knobs:
// points per item (or a tile per grid), persistent CTAs per SM, item order
// within a group, the L2 budget per group, and the load path (rows staged in
// shared memory by bulk copies, or marched through registers).  jacc_batch_tune
// picks the global knobs by timing the whole batch, then a tile size per
// group (so per grid) by timing each group alone.
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
  std::vector<jacc_batch_tile> tile_override;  // rows/cols per grid; 0 = from item_points
  jacc_batch_config cfg{};
  int sms = 0;
  int max_ctas_per_sm[2] = {0, 0};  // [march]: staged, registers
  size_t l2_bytes = 0;
  int nctas = 0;
  int total_items = 0;
  std::vector<JBGrid> hgrids;   // the plan's grid table (host copy)
  std::vector<int> group_of;    // per grid
  std::vector<JBGroup> hgroups;
  i64 max_n = 0;
  // device block: [ticket u64][status i32][pad][done u32 x items] [maxwords] [grids] [items] [groups]
  char* block = nullptr;
  size_t counters_bytes = 0;
  unsigned long long* d_ticket = nullptr;
  int* d_status = nullptr;
  unsigned* d_done = nullptr;
  u64* d_maxwords = nullptr;
  JBGrid* d_grids = nullptr;
  JBItem* d_items = nullptr;
  JBGroup* d_groups = nullptr;
  std::map<std::pair<int32_t, const double*>, SweepGraph> graphs;
};

static void drop_graphs(Batch& b) {
  for (auto& g : b.graphs) {
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (g.second.graph) cudaGraphDestroy(g.second.graph);
  }
  b.graphs.clear();
}

static void config_defaults(jacc_batch_config* c) {
  c->item_points = 8192;
  c->ctas_per_sm = 0;
  c->order = 0;
  c->timeout_ms = 2000;
  c->test_stall_ticket = -1;
  c->group_bytes = 0;
  c->march = 0;
  c->test_stall_row = 0;
}

static bool valid_cols(int c) { return c == 64 || c == 128 || c == 256 || c == 512; }

// The tile of one grid: an override, or item_points spread over the fewest
// 64-column strips that cover the row, at most 2 (128 columns, one strip of
// the bulk-copy march's four-column lanes) for the staged march and 8 for
// the register march; 8 warps per tile.  Tall 128-column items measured
// faster than 512-column ones of the same size on the 64-grid workload
// (368.0 against 320.9 GLUP/s at 64K points).
static void grid_tile(const jacc_grid& G, const jacc_batch_tile& o, int item_points, int march, int* rows,
                      int* cols) {
  int c = o.cols;
  if (c <= 0) {
    const int cap = march == 0 ? 128 : 512;
    c = 64;
    while (c < cap && c < G.nx) c *= 2;
  }
  const int slices = 8 / (c / 64);
  i64 r = o.rows;
  if (r <= 0) r = std::max<i64>(slices, item_points / std::min<i64>(G.nx, c));
  r = std::max<i64>(1, std::min<i64>(r, G.ny));
  *rows = static_cast<int>(r);
  *cols = c;
}

// Builds the tables for cfg and uploads them (synchronous).
static jacc_status plan(Batch& b, const jacc_batch_config& in) {
  jacc_batch_config c = in;
  if (c.item_points <= 0) c.item_points = 8192;
  if (c.timeout_ms <= 0) c.timeout_ms = 2000;
  if (c.order != 0 && c.order != 1) return fail(JACC_ERR_INVALID_ARG, "batch order must be 0 or 1");
  if (c.march != 0 && c.march != 1) return fail(JACC_ERR_INVALID_ARG, "batch march must be 0 or 1");
  if (c.ctas_per_sm < 0) return fail(JACC_ERR_INVALID_ARG, "ctas_per_sm < 0");
  if (c.test_stall_row < 0) return fail(JACC_ERR_INVALID_ARG, "test_stall_row < 0");
  const int ng = static_cast<int>(b.grids.size());
  std::vector<JBGrid> hg(ng);
  int next_item = 0;
  for (int g = 0; g < ng; ++g) {
    const jacc_grid& G = b.grids[g];
    JBGrid& d = hg[g];
    d.u[0] = static_cast<double*>(G.u0);
    d.u[1] = static_cast<double*>(G.u1);
    d.nx = G.nx;
    d.ny = G.ny;
    grid_tile(G, b.tile_override[g], c.item_points, c.march, &d.rows, &d.cols);
    d.nb = static_cast<int>((G.ny + d.rows - 1) / d.rows);
    d.nc = static_cast<int>((G.nx + d.cols - 1) / d.cols);
    d.item_base = next_item;
    d.pad_ = 0;
    if (static_cast<double>(next_item) + static_cast<double>(d.nb) * d.nc > (1u << 30))
      return fail(JACC_ERR_UNSUPPORTED, "too many items");
    next_item += d.nb * d.nc;
  }
  // groups: grids by area, largest first, packed in turn while their fields fit the budget
  const i64 budget = c.group_bytes == 0 ? static_cast<i64>(b.l2_bytes * 2 / 5)
                                        : (c.group_bytes < 0 ? INT64_MAX : c.group_bytes);
  std::vector<int> byarea(ng);
  std::iota(byarea.begin(), byarea.end(), 0);
  std::stable_sort(byarea.begin(), byarea.end(),
                   [&](int a, int z) { return hg[a].nx * hg[a].ny > hg[z].nx * hg[z].ny; });
  std::vector<std::vector<int>> groups;
  i64 used = 0;
  for (int g : byarea) {
    const i64 bytes = 16 * hg[g].nx * hg[g].ny;
    if (groups.empty() || used + bytes > budget) {
      groups.emplace_back();
      used = 0;
    }
    groups.back().push_back(g);
    used += bytes;
  }
  std::vector<JBItem> items;
  std::vector<JBGroup> hq;
  std::vector<int> group_of(ng, 0);
  for (size_t q = 0; q < groups.size(); ++q) {
    JBGroup Q{static_cast<int>(items.size()), 0};
    for (int g : groups[q]) group_of[g] = static_cast<int>(q);
    if (c.order == 0) {
      for (int g : groups[q])
        for (int bb = 0; bb < hg[g].nb; ++bb)
          for (int cc = 0; cc < hg[g].nc; ++cc) items.push_back({g, bb, cc, 0});
    } else {
      int maxi = 0;
      for (int g : groups[q]) maxi = std::max(maxi, hg[g].nb * hg[g].nc);
      for (int i = 0; i < maxi; ++i)
        for (int g : groups[q])
          if (i < hg[g].nb * hg[g].nc) items.push_back({g, i / hg[g].nc, i % hg[g].nc, 0});
    }
    Q.nitems = static_cast<int>(items.size()) - Q.item_begin;
    hq.push_back(Q);
  }
  const int maxc = b.max_ctas_per_sm[c.march];
  const int per_sm = c.ctas_per_sm == 0 ? maxc : std::min(c.ctas_per_sm, maxc);
  if (per_sm < 1) return fail(JACC_ERR_UNSUPPORTED, "the batched kernel does not fit on an SM");

  const size_t n_items = items.size();
  const size_t cb = 16 + sizeof(unsigned) * n_items;
  const size_t counters_bytes = (cb + 255) / 256 * 256;
  const size_t mw_bytes = (sizeof(u64) * ng + 255) / 256 * 256;
  const size_t g_bytes = (sizeof(JBGrid) * ng + 255) / 256 * 256;
  const size_t it_bytes = (sizeof(JBItem) * n_items + 255) / 256 * 256;
  const size_t q_bytes = sizeof(JBGroup) * hq.size();
  char* blk = nullptr;
  jacc_status st = cuda_check(cudaMalloc(&blk, counters_bytes + mw_bytes + g_bytes + it_bytes + q_bytes),
                              "cudaMalloc(batch)");
  if (st) return st;
  char* p_grids = blk + counters_bytes + mw_bytes;
  char* p_items = p_grids + g_bytes;
  char* p_groups = p_items + it_bytes;
  st = cuda_check(cudaMemcpy(p_grids, hg.data(), sizeof(JBGrid) * ng, cudaMemcpyHostToDevice), "cudaMemcpy(grids)");
  if (!st)
    st = cuda_check(cudaMemcpy(p_items, items.data(), sizeof(JBItem) * n_items, cudaMemcpyHostToDevice),
                    "cudaMemcpy(items)");
  if (!st)
    st = cuda_check(cudaMemcpy(p_groups, hq.data(), q_bytes, cudaMemcpyHostToDevice), "cudaMemcpy(groups)");
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
  b.d_grids = reinterpret_cast<JBGrid*>(p_grids);
  b.d_items = reinterpret_cast<JBItem*>(p_items);
  b.d_groups = reinterpret_cast<JBGroup*>(p_groups);
  b.total_items = static_cast<int>(n_items);
  b.hgrids = hg;
  b.hgroups = hq;
  b.group_of = group_of;
  b.nctas = per_sm * b.sms;
  b.cfg = c;
  b.cfg.ctas_per_sm = per_sm;
  return ok();
}

// Enqueues one run of groups [q0, q1) (all groups: 0, ngroups).
static jacc_status enqueue(Batch& b, int32_t nsweeps, double* resid, cudaStream_t s, int q0, int q1) {
  const int ng = static_cast<int>(b.grids.size());
  jacc_status st = cuda_check(cudaMemsetAsync(b.block, 0, b.counters_bytes, s), "memset batch counters");
  if (st) return st;
  if (resid) {
    st = cuda_check(cudaMemsetAsync(resid, 0, sizeof(double) * static_cast<size_t>(ng) * nsweeps, s), "memset resid");
    if (st) return st;
  }
  st = cuda_check(launch_maxabs_batched(b.d_grids, ng, b.max_n, b.d_maxwords, s), "batched max-abs pre-pass");
  if (st) return st;
  long long items = 0;
  for (int q = q0; q < q1; ++q) items += b.hgroups[q].nitems;
  JBatchParams bp{};
  bp.grids = b.d_grids;
  bp.items = b.d_items;
  bp.groups = b.d_groups + q0;
  bp.ngroups = q1 - q0;
  bp.nsweeps = nsweeps;
  bp.total_tickets = items * nsweeps;
  bp.maxwords = b.d_maxwords;
  bp.done = b.d_done;
  bp.ticket = b.d_ticket;
  bp.status = b.d_status;
  bp.staged = b.cfg.march == 0 ? 1 : 0;
  bp.resid = resid;
  bp.timeout_ns = static_cast<u64>(b.cfg.timeout_ms) * 1000000ull;
  bp.stall_ticket = b.cfg.test_stall_ticket;
  bp.stall_row = b.cfg.test_stall_row;
  return cuda_check(launch_batched(bp, b.nctas, s), "batched persistent launch");
}

static jacc_status read_status(Batch& b, cudaStream_t s) {
  jacc_status st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (st) return st;
  int v = 0;
  st = cuda_check(cudaMemcpy(&v, b.d_status, sizeof(int), cudaMemcpyDeviceToHost), "read batch status");
  if (st) return st;
  if (v == JACC_ERR_TIMEOUT) return fail(JACC_ERR_TIMEOUT, "a batched-sweep wait exceeded its time limit");
  if (v != 0) return fail(JACC_ERR_CUDA, "unexpected batch status " + std::to_string(v));
  return ok();
}

// Best of `reps` timed runs (after one warm-up) of groups [q0, q1).
static jacc_status time_run(Batch& b, int32_t sweeps, cudaStream_t s, int q0, int q1, int reps, cudaEvent_t e0,
                            cudaEvent_t e1, double* ms_out) {
  double best = 1e300;
  jacc_status st = ok();
  for (int rep = 0; rep <= reps && !st; ++rep) {
    st = cuda_check(cudaEventRecord(e0, s), "cudaEventRecord");
    if (!st) st = enqueue(b, sweeps, nullptr, s, q0, q1);
    if (!st) st = cuda_check(cudaEventRecord(e1, s), "cudaEventRecord");
    if (!st) st = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0;
    if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (!st && rep > 0) best = std::min(best, static_cast<double>(ms));
  }
  if (!st) st = read_status(b, s);
  *ms_out = best;
  return st;
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
  b->tile_override.assign(ngrids, jacc_batch_tile{0, 0, 0, 0});
  for (const auto& G : b->grids) b->max_n = std::max<i64>(b->max_n, G.nx * G.ny);
  int dev = 0, l2 = 0;
  jacc_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (!st) st = cuda_check(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (!st) st = cuda_check(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev), "L2 size");
  int coop = 0;
  if (!st) st = cuda_check(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "cooperative attr");
  if (st) return st;
  if (!coop) return fail(JACC_ERR_UNSUPPORTED, "device lacks cooperative launch");
  b->l2_bytes = static_cast<size_t>(l2);
  st = cuda_check(batched_occupancy(1, &b->max_ctas_per_sm[0]), "occupancy of the staged batched kernel");
  if (!st) st = cuda_check(batched_occupancy(0, &b->max_ctas_per_sm[1]), "occupancy of the batched kernel");
  if (st) return st;
  jacc_batch_config c;
  config_defaults(&c);
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

extern "C" jacc_status jacc_batch_set_tiles(jacc_batch h, int32_t ngrids, const jacc_batch_tile* tiles) {
  if (!h || !tiles) return fail(JACC_ERR_INVALID_ARG, "NULL batch or tiles");
  Batch& b = *reinterpret_cast<Batch*>(h);
  if (ngrids != static_cast<int32_t>(b.grids.size())) return fail(JACC_ERR_INVALID_ARG, "ngrids differs from the batch");
  for (int g = 0; g < ngrids; ++g) {
    if (tiles[g].rows < 0 || (tiles[g].cols != 0 && !valid_cols(tiles[g].cols)))
      return fail(JACC_ERR_INVALID_ARG, "tile rows must be >= 0 and cols 0, 64, 128, 256 or 512");
  }
  std::lock_guard<std::mutex> lock(global_mutex());
  std::vector<jacc_batch_tile> old = b.tile_override;
  for (int g = 0; g < ngrids; ++g) b.tile_override[g] = jacc_batch_tile{tiles[g].rows, tiles[g].cols, 0, 0};
  jacc_status st = plan(b, b.cfg);
  if (st) b.tile_override = old;
  return st;
}

extern "C" jacc_status jacc_batch_get_tiles(jacc_batch h, int32_t ngrids, jacc_batch_tile* out) {
  if (!h || !out) return fail(JACC_ERR_INVALID_ARG, "NULL batch or output");
  Batch& b = *reinterpret_cast<Batch*>(h);
  if (ngrids != static_cast<int32_t>(b.grids.size())) return fail(JACC_ERR_INVALID_ARG, "ngrids differs from the batch");
  for (int g = 0; g < ngrids; ++g) {
    const JBGrid& G = b.hgrids[g];
    out[g] = jacc_batch_tile{G.rows, G.cols, G.nb * G.nc, b.group_of[g]};
  }
  return ok();
}

extern "C" jacc_status jacc_batch_sweep(jacc_batch h, int32_t nsweeps, double* resid_dev, uint32_t flags,
                                        uintptr_t stream, int32_t* final_buf) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL batch");
  if (nsweeps < 1) return fail(JACC_ERR_INVALID_ARG, "nsweeps must be >= 1");
  if (flags & ~JACC_SWEEP_GRAPH) return fail(JACC_ERR_INVALID_ARG, "unknown sweep flags");
  Batch& b = *reinterpret_cast<Batch*>(h);
  if (nsweeps > (1 << 30)) return fail(JACC_ERR_UNSUPPORTED, "nsweeps exceeds the 32-bit completion counters");
  if (static_cast<double>(nsweeps) * static_cast<double>(b.total_items) > 4.0e18)
    return fail(JACC_ERR_UNSUPPORTED, "ticket count overflows");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nq = static_cast<int>(b.hgroups.size());
  if (final_buf) *final_buf = nsweeps % 2;
  if (!(flags & JACC_SWEEP_GRAPH)) return enqueue(b, nsweeps, resid_dev, s, 0, nq);
  std::lock_guard<std::mutex> lock(global_mutex());
  const auto key = std::make_pair(nsweeps, static_cast<const double*>(resid_dev));
  auto it = b.graphs.find(key);
  if (it == b.graphs.end()) {
    SweepGraph g;
    cudaStream_t cap = nullptr;
    jacc_status st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (!st) {
      jacc_status est = enqueue(b, nsweeps, resid_dev, cap, 0, nq);
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
  return read_status(*reinterpret_cast<Batch*>(h), reinterpret_cast<cudaStream_t>(stream));
}

extern "C" jacc_status jacc_batch_tune(jacc_batch h, int32_t probe_sweeps, uintptr_t stream, jacc_batch_config* best,
                                       double* best_ms) {
  if (!h || probe_sweeps < 1) return fail(JACC_ERR_INVALID_ARG, "NULL batch or probe_sweeps < 1");
  Batch& b = *reinterpret_cast<Batch*>(h);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const jacc_batch_config base = b.cfg;
  const std::vector<jacc_batch_tile> base_tiles = b.tile_override;
  cudaEvent_t e0, e1;
  jacc_status st = cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
  if (st) return st;
  st = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  if (st) {
    cudaEventDestroy(e0);
    return st;
  }
  auto replan = [&](const jacc_batch_config& c) {
    std::lock_guard<std::mutex> lock(global_mutex());
    return plan(b, c);
  };
  // phase 1: global knobs, every grid at the default tile for item_points
  std::fill(b.tile_override.begin(), b.tile_override.end(), jacc_batch_tile{0, 0, 0, 0});
  const i64 budgets[] = {0, static_cast<i64>(b.l2_bytes / 5), static_cast<i64>(b.l2_bytes * 3 / 5), -1};
  double best_t = 1e300;
  jacc_batch_config best_c = base;
  for (int march = 0; march < 2 && !st; ++march) {
    std::vector<int> per_sm = {2, b.max_ctas_per_sm[march]};
    per_sm.erase(std::unique(per_sm.begin(), per_sm.end()), per_sm.end());
    for (int p : per_sm) {
      if (p < 1 || p > b.max_ctas_per_sm[march]) continue;
      for (i64 gb : budgets) {
        for (int pts : {8192, 16384, 32768}) {
          jacc_batch_config c = base;
          c.march = march;
          c.ctas_per_sm = p;
          c.group_bytes = gb;
          c.item_points = pts;
          c.test_stall_ticket = -1;
          c.test_stall_row = 0;
          st = replan(c);
          double t = 1e300;
          if (!st) st = time_run(b, probe_sweeps, s, 0, static_cast<int>(b.hgroups.size()), 2, e0, e1, &t);
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
  }
  // phase 2: a tile size per group (so per grid), each group timed alone
  if (!st) st = replan(best_c);
  const int nq = static_cast<int>(b.hgroups.size());
  for (int q = 0; q < nq && !st; ++q) {
    std::vector<int> members;
    for (int g = 0; g < static_cast<int>(b.grids.size()); ++g)
      if (b.group_of[g] == q) members.push_back(g);
    int best_pts = 0;
    double best_q = 1e300;
    for (int pts : {4096, 8192, 16384, 32768, 65536}) {
      for (int g : members) {
        int rows = 0, cols = 0;
        grid_tile(b.grids[g], jacc_batch_tile{0, 0, 0, 0}, pts, best_c.march, &rows, &cols);
        b.tile_override[g] = jacc_batch_tile{rows, cols, 0, 0};
      }
      st = replan(best_c);
      double t = 1e300;
      if (!st) st = time_run(b, probe_sweeps, s, q, q + 1, 2, e0, e1, &t);
      if (st) break;
      if (t < best_q) {
        best_q = t;
        best_pts = pts;
      }
    }
    for (int g : members) {
      int rows = 0, cols = 0;
      grid_tile(b.grids[g], jacc_batch_tile{0, 0, 0, 0}, best_pts, best_c.march, &rows, &cols);
      b.tile_override[g] = jacc_batch_tile{rows, cols, 0, 0};
    }
  }
  double final_t = 1e300;
  if (!st) st = replan(best_c);
  if (!st) st = time_run(b, probe_sweeps, s, 0, static_cast<int>(b.hgroups.size()), 2, e0, e1, &final_t);
  if (!st && final_t > best_t) {  // the per-group tiles did not help the whole run: back to phase 1's tiles
    std::fill(b.tile_override.begin(), b.tile_override.end(), jacc_batch_tile{0, 0, 0, 0});
    st = replan(best_c);
    final_t = best_t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    b.tile_override = base_tiles;
    replan(base);
    return st;
  }
  if (best) *best = b.cfg;
  if (best_ms) *best_ms = final_t;
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
