// aux.cu - non-template helper kernels (max-abs pre-pass, NaN fill) and their launchers.
#define JACC_AUX_KERNELS
#include "jacc_device.cuh"

#include <cuda_runtime.h>

namespace jacc {

cudaError_t launch_maxabs(const double* u, long long n, u64* maxword, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(maxword, 0, sizeof(u64), s);
  if (e != cudaSuccess) return e;
  // one resident wave of 256-thread blocks (8 per SM) of the current device
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    nsm = 152;
  long long pairs = n / 2;
  long long blocks = (pairs + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 8ll * nsm) blocks = 8ll * nsm;
  jacc_k_maxabs<<<(unsigned)blocks, 256, 0, s>>>(u, n, maxword);
  return cudaGetLastError();
}

cudaError_t launch_to_fixed(double* u, long long n, const u64* maxword, cudaStream_t s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    nsm = 152;
  long long blocks = (n / 2 + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 8ll * nsm) blocks = 8ll * nsm;
  jacc_k_to_fixed<<<(unsigned)blocks, 256, 0, s>>>(u, n, maxword);
  return cudaGetLastError();
}

// Temporally blocked 27-point FP32 kernels: region 128 x 16, depth 2 and 3, 64-plane chunks.
extern "C" const void* const jacc_tab_tb[2] = {(const void*)jacc_k_box27_tb<16, 2, 64>,
                                               (const void*)jacc_k_box27_tb<16, 3, 64>};

cudaError_t launch_fill_skipped(double* resid, int n, int T, cudaStream_t s) {
  jacc_k_fill_skipped<<<(n + 255) / 256, 256, 0, s>>>(resid, n, T);
  return cudaGetLastError();
}

}  // namespace jacc
