// until.cu - the device side of jacc_sweep_until: the loop's exit test and
// the choice of the final converting sweep, run inside the CUDA graph so the
// loop needs no host round trip.
#include <cuda_runtime.h>

#include "../host/jacc_internal.h"

namespace {

// After each sweep: move the sweep's residual from its accumulation slot to
// resid[i], clear the slot for the next sweep, count the sweep, and set the
// loop's conditions: continue while resid > tol and fewer than max sweeps ran.
__global__ void jacc_k_until_check(double* slot, int* counter, double* resid, double tol, int max_sweeps,
                                   cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_odd) {
  const double r = *slot;
  *slot = 0.0;
  const int i = *counter;
  resid[i] = r;
  *counter = i + 1;
  const unsigned more = (r > tol && i + 1 < max_sweeps) ? 1u : 0u;
  cudaGraphSetConditional(h_loop, more);
  cudaGraphSetConditional(h_odd, more);
}

// After the loop: report the sweep count and the result buffer, and pick the
// final sweep that rewrites the result in FP64 from the state before it:
// 0 = the only sweep (u0 -> u1, FP64 in and out), 1 = an even count
// (u1 -> u0), 2 = an odd count of 3 or more (u0 -> u1); 3 = none.
__global__ void jacc_k_until_final(const int* counter, int* status, int recompute, cudaGraphConditionalHandle h_final) {
  const int n = *counter;
  status[0] = n;
  status[1] = n & 1;
  unsigned c = 3u;
  if (recompute) c = (n == 1) ? 0u : ((n & 1) ? 2u : 1u);
  cudaGraphSetConditional(h_final, c);
}

}  // namespace

namespace jacc {

cudaError_t launch_until_check(double* slot, int* counter, double* resid, double tol, int max_sweeps,
                               cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_odd, cudaStream_t s) {
  jacc_k_until_check<<<1, 1, 0, s>>>(slot, counter, resid, tol, max_sweeps, h_loop, h_odd);
  return cudaGetLastError();
}

cudaError_t launch_until_final(const int* counter, int* status, int recompute, cudaGraphConditionalHandle h_final,
                               cudaStream_t s) {
  jacc_k_until_final<<<1, 1, 0, s>>>(counter, status, recompute, h_final);
  return cudaGetLastError();
}

}  // namespace jacc
