// batched.h - device tables of the batched persistent launch (host and device).
#pragma once

#include <cuda_runtime.h>

#include "jacc_params.h"

struct JBGrid {
  double* u[2];  // ping-pong fields; sweep s reads u[s & 1] and writes u[(s + 1) & 1]
  i64 nx, ny;
  i64 rows;      // rows per item (band height)
  int nitems;    // ceil(ny / rows)
  int vec;       // 2: 16-byte vector loads (even nx); 1: scalar
};

struct JBItem {
  int g;     // grid
  int item;  // band index within the grid
};

struct JBatchParams {
  const JBGrid* grids;
  const JBItem* items;  // one sweep's items in schedule order
  int ngrids;
  int total_items;
  int nsweeps;
  int pad_;
  const u64* maxwords;       // per-grid max|u0| bit patterns (fixed point), or null
  unsigned* done;            // per-grid count of finished items, all sweeps
  unsigned long long* ticket;
  int* status;               // 0, or JACC_ERR_TIMEOUT after a wait gave up
  double* resid;             // [ngrids][nsweeps] or null
  u64 timeout_ns;
  long long stall_ticket;    // fault-injection hook: this ticket never signals (-1: none)
};

namespace jacc {
cudaError_t batched_occupancy(int* blocks_per_sm);
cudaError_t launch_batched(const JBatchParams& bp, int nctas, cudaStream_t s);
cudaError_t launch_maxabs_batched(const JBGrid* d_grids, int ngrids, i64 max_n, u64* maxwords, cudaStream_t s);
}  // namespace jacc
