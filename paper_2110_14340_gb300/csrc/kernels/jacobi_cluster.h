// jacobi_cluster.h - the cluster-resident 5-point FP64 sweep sequence.
#pragma once

#include <cuda_runtime.h>

struct JClusterArgs {
  const double* u;   // input field (FP64, nx * ny, row-major)
  double* res;       // receives the field after nsweeps sweeps (FP64)
  double* oth;       // receives sweep nsweeps-1 in the internal form (nsweeps >= 2)
  double* resid;     // nullable: nsweeps doubles, receives the per-sweep max |v - u|
  long long nx, ny;
  long long rows;    // grid rows per CTA (set by the launcher)
  long long pitch;   // shared-memory row pitch in words (set by the launcher)
  int nsweeps;
  int native;        // 1: native FP64 arithmetic (JACC_ARITH_NATIVE)
};

// 1 and the cluster size (16 or 8) if both fields of an nx x ny grid fit in
// the shared memory of one cluster that the current device can run.
int jacobi_cluster_plan(long long nx, long long ny, int* nc_out);
// One launch of one cluster of nc CTAs running all a.nsweeps sweeps.
cudaError_t launch_jacobi_cluster(JClusterArgs a, int nc, cudaStream_t s);
