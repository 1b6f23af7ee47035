// sweep_until.cpp - jacc_sweep_until: sweeps until the residual drops to a
// tolerance, with the loop and its exit test on the device.
//
// One CUDA graph per (kernel, fields, max_sweeps, tol, output arrays), built
// once and replayed:
//   A      the first sweep (u0 -> u1; FP64 fixed point converts on load,
//          after the max-abs pre-pass) and a one-thread check kernel;
//   WHILE  (condition set by the checks) a pair of sweeps u1 -> u0 -> u1,
//          each followed by a check; the second sits in an IF node on the
//          same decision, so the loop can stop after either;
//   F      a one-thread kernel that writes the sweep count and the result
//          buffer and picks the final sweep;
//   SWITCH the final sweep run again from the state before it with FP64
//          output (FP64 fixed-point kernels only), so that the result is the
//          exact stencil value rounded once to FP64, as jacc_sweep leaves it.
// The check kernel moves each sweep's residual from an accumulation slot to
// resid[i] and sets the loop's conditions (cudaGraphSetConditional).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "jacc_internal.h"

namespace jacc {

void free_until_graphs(Kernel& k) {
  for (auto& g : k.until_graphs) {
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (g.second.graph) cudaGraphDestroy(g.second.graph);
    if (g.second.scratch) cudaFree(g.second.scratch);
  }
  k.until_graphs.clear();
}

namespace {

// Captures the work `fn` enqueues on stream s into graph g (empty on entry).
template <class Fn> jacc_status capture_into(cudaGraph_t g, cudaStream_t s, Fn fn) {
  jacc_status st = cuda_check(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                              "cudaStreamBeginCaptureToGraph");
  if (st) return st;
  jacc_status body = fn();
  cudaGraph_t out = nullptr;
  jacc_status end = cuda_check(cudaStreamEndCapture(s, &out), "cudaStreamEndCapture");
  return body ? body : end;
}

// A conditional node of `type` on handle h after `dep` (nullable); returns its body graphs.
jacc_status add_conditional(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, unsigned size, cudaGraphNode_t* node,
                            cudaGraph_t** bodies) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = size;
  jacc_status st = cuda_check(cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &p), "add conditional node");
  if (st) return st;
  *bodies = p.conditional.phGraph_out;
  return ok();
}

jacc_status add_child(cudaGraph_t g, cudaGraphNode_t dep, cudaGraph_t child, cudaGraphNode_t* node) {
  return cuda_check(cudaGraphAddChildGraphNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, child),
                    "add child graph node");
}

}  // namespace

// Builds the graph described at the top of this file into ug (scratch set).
static jacc_status build_until(const Kernel& k, void* u0, void* u1, int32_t max_sweeps, double tol, double* resid,
                               int32_t* status, cudaStream_t s, UntilGraph& ug) {
  const bool fixed = k.desc.dtype == 64 && k.params.fpath != JACC_FP_NONE;
  u64* maxword = ug.scratch;
  double* slot = reinterpret_cast<double*>(ug.scratch + 1);
  int* counter = reinterpret_cast<int*>(ug.scratch + 2);
  double* spare = reinterpret_cast<double*>(ug.scratch + 3);
  const u64* mw = fixed ? maxword : nullptr;
  jacc_status st = cuda_check(cudaGraphCreate(&ug.graph, 0), "cudaGraphCreate");
  if (st) return st;
  cudaGraphConditionalHandle h_loop, h_odd, h_final;
  st = cuda_check(cudaGraphConditionalHandleCreate(&h_loop, ug.graph, 0, 0), "conditional handle");
  if (!st) st = cuda_check(cudaGraphConditionalHandleCreate(&h_odd, ug.graph, 0, 0), "conditional handle");
  if (!st) st = cuda_check(cudaGraphConditionalHandleCreate(&h_final, ug.graph, 3, cudaGraphCondAssignDefault),
                           "conditional handle");
  if (st) return st;
  const void* cu0 = u0;
  const void* cu1 = u1;
  auto sweep = [&](const void* src, void* dst, double* r, int flags) {
    return cuda_check(launch_sweep_kernel(k, src, dst, r, mw, flags, s), "stencil launch");
  };
  auto check = [&]() {
    return cuda_check(launch_until_check(slot, counter, resid, tol, max_sweeps, h_loop, h_odd, s), "check launch");
  };
  // A: zero the slots and the counter, pre-pass, first sweep, check
  cudaGraph_t gA = nullptr;
  st = cuda_check(cudaGraphCreate(&gA, 0), "cudaGraphCreate");
  if (st) return st;
  st = capture_into(gA, s, [&]() -> jacc_status {
    jacc_status e = cuda_check(cudaMemsetAsync(ug.scratch, 0, 4 * sizeof(u64), s), "memset scratch");
    if (!e && fixed)
      e = cuda_check(launch_maxabs(static_cast<const double*>(u0), k.desc.nx * k.desc.ny * k.desc.nz, maxword, s),
                     "max-abs pre-pass");
    if (!e) e = sweep(cu0, u1, slot, kFxIn);
    if (!e) e = check();
    return e;
  });
  cudaGraphNode_t nA = nullptr, nW = nullptr, nF = nullptr, nS = nullptr;
  if (!st) st = add_child(ug.graph, nullptr, gA, &nA);
  cudaGraphDestroy(gA);  // the child node holds a copy
  if (st) return st;
  // WHILE: u1 -> u0, check, IF { u0 -> u1, check }
  cudaGraph_t* wb = nullptr;
  st = add_conditional(ug.graph, nA, h_loop, cudaGraphCondTypeWhile, 1, &nW, &wb);
  if (st) return st;
  cudaGraph_t gE = nullptr;
  st = cuda_check(cudaGraphCreate(&gE, 0), "cudaGraphCreate");
  if (st) return st;
  st = capture_into(gE, s, [&]() -> jacc_status {
    jacc_status e = sweep(cu1, u0, slot, 0);
    return e ? e : check();
  });
  cudaGraphNode_t nE = nullptr, nI = nullptr;
  if (!st) st = add_child(wb[0], nullptr, gE, &nE);
  cudaGraphDestroy(gE);
  if (st) return st;
  cudaGraph_t* ib = nullptr;
  st = add_conditional(wb[0], nE, h_odd, cudaGraphCondTypeIf, 1, &nI, &ib);
  if (st) return st;
  st = capture_into(ib[0], s, [&]() -> jacc_status {
    jacc_status e = sweep(cu0, u1, slot, 0);
    return e ? e : check();
  });
  if (st) return st;
  // F: status and the choice of the final sweep
  cudaGraph_t gF = nullptr;
  st = cuda_check(cudaGraphCreate(&gF, 0), "cudaGraphCreate");
  if (st) return st;
  st = capture_into(gF, s, [&]() -> jacc_status {
    return cuda_check(launch_until_final(counter, status, fixed ? 1 : 0, h_final, s), "final launch");
  });
  if (!st) st = add_child(ug.graph, nW, gF, &nF);
  cudaGraphDestroy(gF);
  if (st) return st;
  // SWITCH: the final sweep again, from the state before it, FP64 out
  cudaGraph_t* sb = nullptr;
  st = add_conditional(ug.graph, nF, h_final, cudaGraphCondTypeSwitch, 3, &nS, &sb);
  if (st) return st;
  st = capture_into(sb[0], s, [&]() { return sweep(cu0, u1, spare, kFxIn | kFxOut); });
  if (!st) st = capture_into(sb[1], s, [&]() { return sweep(cu1, u0, spare, kFxOut); });
  if (!st) st = capture_into(sb[2], s, [&]() { return sweep(cu0, u1, spare, kFxOut); });
  if (st) return st;
  return cuda_check(cudaGraphInstantiate(&ug.exec, ug.graph, 0), "cudaGraphInstantiate");
}

}  // namespace jacc

using namespace jacc;

extern "C" jacc_status jacc_sweep_until(jacc_kernel h, void* u0, void* u1, int32_t max_sweeps, double tol,
                                        double* resid_dev, int32_t* status_dev, uintptr_t stream) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  Kernel& k = *reinterpret_cast<Kernel*>(h);
  if (k.desc.stencil == 19) return fail(JACC_ERR_UNSUPPORTED, "jacc_sweep_until: 5-point and 7-point only");
  if (k.desc.stencil == 27)
    return fail(JACC_ERR_UNSUPPORTED, "jacc_sweep_until: the 27-point reduction is a sum, not a convergence measure");
  if (max_sweeps < 1) return fail(JACC_ERR_INVALID_ARG, "max_sweeps must be >= 1");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(JACC_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (!resid_dev || !status_dev) return fail(JACC_ERR_INVALID_ARG, "resid_dev and status_dev are required");
  if ((reinterpret_cast<uintptr_t>(resid_dev) % 8) || (reinterpret_cast<uintptr_t>(status_dev) % 4))
    return fail(JACC_ERR_INVALID_ARG, "misaligned resid_dev or status_dev");
  jacc_status st = check_buffers(k, u0, u1);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(global_mutex());
  const UntilKey key(u0, u1, max_sweeps, tol, resid_dev, status_dev);
  auto it = k.until_graphs.find(key);
  if (it == k.until_graphs.end()) {
    UntilGraph ug;
    st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&ug.scratch), 256), "cudaMalloc(until scratch)");
    cudaStream_t cap = nullptr;  // captures run on a private stream (the caller's may be the legacy one)
    if (!st) st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = build_until(k, u0, u1, max_sweeps, tol, resid_dev, status_dev, cap, ug);
    if (cap) cudaStreamDestroy(cap);
    if (st) {
      if (ug.exec) cudaGraphExecDestroy(ug.exec);
      if (ug.graph) cudaGraphDestroy(ug.graph);
      if (ug.scratch) cudaFree(ug.scratch);
      return st;
    }
    it = k.until_graphs.emplace(key, ug).first;
  }
  return cuda_check(cudaGraphLaunch(it->second.exec, s), "cudaGraphLaunch");
}
