// sweep_host.cpp - jacc_sweep_host: a sweep sequence from and to host
// buffers in one call: the input field is copied into the caller's device
// buffer u0, the sequence runs as jacc_sweep does, and the result field (and,
// if asked, the residuals) are copied back, all enqueued on one stream.
//
// Three cudaMemcpyAsync calls, one per buffer; the library allocates
// nothing.  With page-locked host buffers the copies are asynchronous, so
// calls on two streams with two sets of device buffers overlap one call's
// copies with the other's sweeps; the optional events let the caller keep
// the sweeps of consecutive calls in order (the sweeps wait for wait_event,
// done_event is recorded after them, before the copy back).
#include <cuda_runtime.h>

#include "jacc_internal.h"

using namespace jacc;

extern "C" jacc_status jacc_sweep_host(jacc_kernel h, const void* u_host, void* result_host, void* u0, void* u1,
                                       int32_t nsweeps, double* resid_dev, double* resid_host, uint32_t flags,
                                       uintptr_t stream, uintptr_t wait_event, uintptr_t done_event,
                                       int32_t* final_buf) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  if (!u_host || !result_host) return fail(JACC_ERR_INVALID_ARG, "NULL host buffer");
  if (resid_host && !resid_dev) return fail(JACC_ERR_INVALID_ARG, "resid_host needs resid_dev");
  const Kernel& k = *reinterpret_cast<Kernel*>(h);
  if (k.desc.stencil == 19) return fail(JACC_ERR_INVALID_ARG, "19-point stencil: use jacc_sweep_coeffs");
  jacc_status st = check_buffers(k, u0, u1);
  if (st) return st;
  if (nsweeps < 1) return fail(JACC_ERR_INVALID_ARG, "nsweeps must be >= 1");
  const size_t bytes = static_cast<size_t>(k.desc.nx * k.desc.ny * k.desc.nz) * k.elem;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  st = cuda_check(cudaMemcpyAsync(u0, u_host, bytes, cudaMemcpyHostToDevice, s), "copy of the input field");
  if (st) return st;
  if (wait_event) {
    st = cuda_check(cudaStreamWaitEvent(s, reinterpret_cast<cudaEvent_t>(wait_event), 0), "wait before the sweeps");
    if (st) return st;
  }
  int32_t fb = 0;
  st = jacc_sweep(h, u0, u1, nsweeps, resid_dev, flags, stream, &fb);
  if (st) return st;
  if (done_event) {
    st = cuda_check(cudaEventRecord(reinterpret_cast<cudaEvent_t>(done_event), s), "record after the sweeps");
    if (st) return st;
  }
  st = cuda_check(cudaMemcpyAsync(result_host, fb ? u1 : u0, bytes, cudaMemcpyDeviceToHost, s), "copy of the result");
  if (st) return st;
  if (resid_host) {
    st = cuda_check(cudaMemcpyAsync(resid_host, resid_dev, sizeof(double) * static_cast<size_t>(nsweeps),
                                    cudaMemcpyDeviceToHost, s),
                    "copy of the residuals");
    if (st) return st;
  }
  if (final_buf) *final_buf = fb;
  return ok();
}
