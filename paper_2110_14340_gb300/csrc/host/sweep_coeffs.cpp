// sweep_coeffs.cpp - jacc_sweep_coeffs: sweeps of the variable-coefficient
// 19-point stencil, whose twelve coefficient fields are passed per call.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "jacc_internal.h"

namespace jacc {

static jacc_status enqueue_coeffs(const Kernel& k, const JParams& p, void* u0, void* u1, int32_t n, double* resid,
                                  cudaStream_t s) {
  if (resid) {
    jacc_status st = cuda_check(cudaMemsetAsync(resid, 0, sizeof(double) * static_cast<size_t>(n), s), "memset resid");
    if (st) return st;
  }
  for (int32_t i = 0; i < n; ++i) {
    const float* src = static_cast<const float*>((i % 2 == 0) ? u0 : u1);
    float* dst = static_cast<float*>((i % 2 == 0) ? u1 : u0);
    jacc_status st = cuda_check(launch_var19(src, dst, p, resid ? resid + i : nullptr, k.grid, k.block, s),
                                "19-point launch");
    if (st) return st;
  }
  return ok();
}

}  // namespace jacc

using namespace jacc;

extern "C" jacc_status jacc_sweep_coeffs(jacc_kernel h, void* u0, void* u1, int32_t nsweeps,
                                         const void* const* fields, int32_t nfields, double* resid_dev,
                                         uint32_t flags, uintptr_t stream, int32_t* final_buf) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  Kernel& k = *reinterpret_cast<Kernel*>(h);
  if (k.desc.stencil != 19) return fail(JACC_ERR_INVALID_ARG, "jacc_sweep_coeffs: 19-point stencil handles only");
  if (nsweeps < 1) return fail(JACC_ERR_INVALID_ARG, "nsweeps must be >= 1");
  if (flags & ~JACC_SWEEP_GRAPH) return fail(JACC_ERR_INVALID_ARG, "unknown sweep flags");
  if (!fields || nfields != 12) return fail(JACC_ERR_INVALID_ARG, "twelve coefficient fields are required");
  jacc_status st = check_buffers(k, u0, u1);
  if (st) return st;
  const uintptr_t bytes = static_cast<uintptr_t>(k.desc.nx * k.desc.ny * k.desc.nz) * 4;
  const uintptr_t pa = reinterpret_cast<uintptr_t>(u0), pb = reinterpret_cast<uintptr_t>(u1);
  JParams p = k.params;
  for (int f = 0; f < 12; ++f) {
    const uintptr_t pf = reinterpret_cast<uintptr_t>(fields[f]);
    if (!pf || (pf % 16)) return fail(JACC_ERR_INVALID_ARG, "coefficient fields must be non-NULL and 16-byte aligned");
    // read through the non-coherent path while u0/u1 are written: no overlap
    if ((pf < pa + bytes && pa < pf + bytes) || (pf < pb + bytes && pb < pf + bytes))
      return fail(JACC_ERR_INVALID_ARG, "a coefficient field overlaps u0 or u1");
    p.cf[f] = static_cast<const float*>(fields[f]);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (final_buf) *final_buf = nsweeps % 2;
  if (!(flags & JACC_SWEEP_GRAPH)) return enqueue_coeffs(k, p, u0, u1, nsweeps, resid_dev, s);

  // graph cached by every pointer of the call (fields included)
  std::string key(reinterpret_cast<const char*>(&u0), sizeof(void*));
  key.append(reinterpret_cast<const char*>(&u1), sizeof(void*));
  key.append(reinterpret_cast<const char*>(&nsweeps), sizeof(nsweeps));
  key.append(reinterpret_cast<const char*>(&resid_dev), sizeof(void*));
  key.append(reinterpret_cast<const char*>(fields), 12 * sizeof(void*));
  std::lock_guard<std::mutex> lock(global_mutex());
  auto it = k.coeff_graphs.find(key);
  if (it == k.coeff_graphs.end()) {
    SweepGraph g;
    cudaStream_t cap = nullptr;
    st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (!st) {
      jacc_status est = enqueue_coeffs(k, p, u0, u1, nsweeps, resid_dev, cap);
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
    it = k.coeff_graphs.emplace(key, g).first;
  }
  return cuda_check(cudaGraphLaunch(it->second.exec, s), "cudaGraphLaunch");
}
