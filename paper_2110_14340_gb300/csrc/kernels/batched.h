// batched.h - device tables of the batched persistent launch (host and device).
#pragma once

#include <cuda_runtime.h>

#include "jacc_params.h"

// One grid and its tiling.  Items are tiles of `rows` rows x `cols` columns
// (cols a multiple of 64, at most 512), numbered b * nc + c for band b and
// column tile c; item_base is the grid's first item in the per-item
// completion counters.
struct JBGrid {
  double* u[2];  // ping-pong fields; sweep s reads u[s & 1] and writes u[(s + 1) & 1]
  i64 nx, ny;
  int rows;      // rows per item (band height)
  int cols;      // columns per item: 64 x (warps across)
  int nb, nc;    // bands, column tiles
  int item_base; // index of item (0, 0) in the completion counters
  int pad_;
};

struct JBItem {
  int g;  // grid
  int b;  // band
  int c;  // column tile
  int pad_;
};

// A group: grids whose two fields fit the L2 budget together; all sweeps of
// a group's items are consecutive tickets (sweep-major within the group).
// Groups occupy consecutive ranges of the item table, so a group's first
// ticket is (item_begin - the run's first item_begin) x nsweeps.
struct JBGroup {
  int item_begin;  // first entry in the item table
  int nitems;      // items per sweep
};

struct JBatchParams {
  const JBGrid* grids;
  const JBItem* items;   // per group, one sweep's items in schedule order
  const JBGroup* groups;
  int ngroups;           // groups run by this launch: groups[0 .. ngroups)
  int nsweeps;
  long long total_tickets;
  const u64* maxwords;       // per-grid max|u0| bit patterns (fixed point), or null
  unsigned* done;            // per-item count of finished sweeps
  unsigned long long* ticket;
  int* status;               // 0, or JACC_ERR_TIMEOUT after a wait gave up
  int staged;                // 1: rows staged in shared memory; 0: register march
  int stall_row;             // fault-injection hook: warp 0 of the first ticket's CTA never fetches this staged row (1-based; 0: none)
  double* resid;             // [ngrids][nsweeps] or null
  u64 timeout_ns;
  long long stall_ticket;    // fault-injection hook: this ticket never signals (-1: none)
};

namespace jacc {
cudaError_t batched_occupancy(int staged, int* blocks_per_sm);
cudaError_t launch_batched(const JBatchParams& bp, int nctas, cudaStream_t s);
cudaError_t launch_maxabs_batched(const JBGrid* d_grids, int ngrids, i64 max_n, u64* maxwords, cudaStream_t s);
}  // namespace jacc
