// static_scratch.cu - jacc_launch_static: the one entry point that allocates nothing.
//
// jacc_launch keeps the 8-byte fixed-point scale word of an FP64 sweep in a
// small device buffer that jacc_specialize obtains with cudaMalloc.  Some
// callers cannot allocate device memory at the moment they launch: code that
// runs under a memory pool which must account for every device byte, code
// that must not hit cudaMalloc's implicit device synchronisation on a
// latency-critical path, and code that must not fail on allocation at run
// time.  For them, this variant keeps its scratch in a file-scope static
// device array instead.  The array is loaded with the library, so every GPU
// that loads libjacc.so holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../host/jacc_internal.h"

namespace {

// Capacity of the static scratch array: 32 words = 256 bytes.  A sweep uses
// one word (the bit pattern of max|u|), whatever the grid size.
constexpr int kStaticWords = 32;
constexpr int kWordsPerLaunch = 1;

static __device__ __align__(256) u64 g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
u64* g_addr[kMaxDevices] = {nullptr};

// The host-side name g_static_scratch is not a device address; the address
// valid on the current device comes from cudaGetSymbolAddress, taken once per
// device with that device current.  The cached address belongs to the
// device's primary context: jacc_shutdown forgets it (a context reset makes
// it stale, and jacc_shutdown is required after one anyway).
jacc_status static_scratch_address(u64** out) {
  int dev = 0;
  jacc_status st = jacc::cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st) return st;
  if (dev < 0 || dev >= kMaxDevices) return jacc::fail(JACC_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    st = jacc::cuda_check(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress(static scratch)");
    if (st) return st;
    g_addr[dev] = static_cast<u64*>(p);
  }
  *out = g_addr[dev];
  return jacc::ok();
}

}  // namespace

namespace jacc {
void static_scratch_forget() {
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& a : g_addr) a = nullptr;
}
}  // namespace jacc

extern "C" jacc_status jacc_launch_static(jacc_kernel h, const void* u_in, void* u_out, double* resid_dev,
                                          uintptr_t stream) {
  using jacc::cuda_check;
  using jacc::fail;
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  const jacc::Kernel& k = *reinterpret_cast<jacc::Kernel*>(h);
  if (k.desc.stencil == 19) return fail(JACC_ERR_INVALID_ARG, "19-point stencil: use jacc_sweep_coeffs");
  if (!u_in || !u_out) return fail(JACC_ERR_INVALID_ARG, "NULL field pointer");
  if ((reinterpret_cast<uintptr_t>(u_in) % 16) || (reinterpret_cast<uintptr_t>(u_out) % 16))
    return fail(JACC_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
  const uintptr_t bytes = static_cast<uintptr_t>(k.desc.nx * k.desc.ny * k.desc.nz) * k.elem;
  const uintptr_t pa = reinterpret_cast<uintptr_t>(u_in), pb = reinterpret_cast<uintptr_t>(u_out);
  if (pa < pb + bytes && pb < pa + bytes) return fail(JACC_ERR_INVALID_ARG, "input and output fields overlap");
  const bool fixed = k.desc.dtype == 64 && k.params.fpath != JACC_FP_NONE;
  const int need = fixed ? kWordsPerLaunch : 0;
  if (need > kStaticWords)
    return fail(JACC_ERR_UNSUPPORTED, "launch needs more scratch than the 256-byte static array holds");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const u64* mw = nullptr;
  if (fixed) {
    u64* scratch = nullptr;
    jacc_status st = static_scratch_address(&scratch);
    if (st) return st;
    // launch_maxabs zeroes the word (the array keeps the previous call's value)
    st = cuda_check(jacc::launch_maxabs(static_cast<const double*>(u_in), k.desc.nx * k.desc.ny * k.desc.nz, scratch, s),
                    "max-abs pre-pass");
    if (st) return st;
    mw = scratch;
  }
  if (resid_dev) {
    jacc_status st = cuda_check(cudaMemsetAsync(resid_dev, 0, sizeof(double), s), "cudaMemsetAsync(resid)");
    if (st) return st;
  }
  return cuda_check(jacc::launch_sweep_kernel(k, u_in, u_out, resid_dev, mw, jacc::kFxIn | jacc::kFxOut, s),
                    "stencil launch");
}
