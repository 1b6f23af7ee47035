// errors.cpp - status handling and the per-thread last-error message.
#include <cuda_runtime.h>

#include <string>

#include "jacc_internal.h"

namespace jacc {

static thread_local std::string g_last_error;

jacc_status fail(jacc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

jacc_status ok() { return JACC_OK; }

jacc_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return JACC_OK;
  return fail(JACC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

std::mutex& global_mutex() {
  static std::mutex m;
  return m;
}

}  // namespace jacc

extern "C" const char* jacc_last_error(void) { return jacc::g_last_error.c_str(); }

extern "C" const char* jacc_version(void) { return "jacc-gb300 1.0 (sm_103a)"; }
