/* A plain C client of the boundary: one heat sequence through the C ABI from
 * and to host memory (jacc_specialize, jacc_sweep_host, jacc_release).
 *   heat_c_client <n> <nsweeps> <input file> <output file>
 * Input: n^3 FP64 values (raw, x fastest).  Output: the n^3 result values
 * followed by the nsweeps residuals (raw FP64).  Exit status 0 on success,
 * else the failing step's message on stderr. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "jacc.h"

static int fail(const char* what, const char* why) {
  fprintf(stderr, "%s: %s\n", what, why);
  return 1;
}

int main(int argc, char** argv) {
  if (argc != 5) return fail("usage", "heat_c_client <n> <nsweeps> <input> <output>");
  const long long n = atoll(argv[1]);
  const int ns = atoi(argv[2]);
  if (n < 3 || ns < 1) return fail("arguments", "n >= 3 and nsweeps >= 1");
  const size_t count = (size_t)(n * n * n), bytes = count * sizeof(double);
  double* in = (double*)malloc(bytes);
  double* out = (double*)malloc(bytes);
  double* res = (double*)malloc(sizeof(double) * (size_t)ns);
  if (!in || !out || !res) return fail("malloc", "out of host memory");
  FILE* f = fopen(argv[3], "rb");
  if (!f || fread(in, sizeof(double), count, f) != count) return fail("read", argv[3]);
  fclose(f);

  jacc_kernel_desc d;
  memset(&d, 0, sizeof(d));
  d.stencil = JACC_STENCIL_7PT;
  d.dtype = JACC_F64;
  d.boundary = JACC_DIRICHLET;
  d.tile_id = -1;
  d.nx = d.ny = d.nz = n;
  d.coeffs[0] = 0.125;
  jacc_kernel k = NULL;
  if (jacc_specialize(&d, &k) != JACC_OK) return fail("jacc_specialize", jacc_last_error());

  void *u0 = NULL, *u1 = NULL, *r = NULL;
  if (cudaMalloc(&u0, bytes) != cudaSuccess || cudaMalloc(&u1, bytes) != cudaSuccess ||
      cudaMalloc(&r, sizeof(double) * (size_t)ns) != cudaSuccess)
    return fail("cudaMalloc", "device allocation failed");
  int32_t fb = -1;
  if (jacc_sweep_host(k, in, out, u0, u1, ns, (double*)r, res, JACC_SWEEP_GRAPH, 0, 0, 0, &fb) != JACC_OK)
    return fail("jacc_sweep_host", jacc_last_error());
  if (cudaStreamSynchronize(0) != cudaSuccess) return fail("cudaStreamSynchronize", "stream error");

  f = fopen(argv[4], "wb");
  if (!f || fwrite(out, sizeof(double), count, f) != count || fwrite(res, sizeof(double), (size_t)ns, f) != (size_t)ns)
    return fail("write", argv[4]);
  fclose(f);
  jacc_release(k);
  cudaFree(u0);
  cudaFree(u1);
  cudaFree(r);
  free(in);
  free(out);
  free(res);
  printf("ok: %lld^3 x %d, result in u%d\n", n, ns, fb);
  return 0;
}
