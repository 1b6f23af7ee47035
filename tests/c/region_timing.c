/* Host timing of jacc_region_analyze from plain C (no Python in the loop):
 * the interior loop nest of the 5-point Jacobi sweep of an n x n grid
 * (loops [1, n-2]^2; reads u[i][j-1], u[i][j+1], u[i-1][j], u[i+1][j],
 * u[i][j]; writes v[i][j]).
 *   region_timing <n> <calls>
 * Prints the write and read hulls of the last call and the mean time per
 * call in microseconds; exit status 0 on success. */
#define _POSIX_C_SOURCE 199309L
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "jacc.h"

static double now_us(void) {
  struct timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return (double)t.tv_sec * 1e6 + (double)t.tv_nsec * 1e-3;
}

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: region_timing <n> <calls>\n");
    return 1;
  }
  const long long n = atoll(argv[1]);
  const int calls = atoi(argv[2]);
  if (n < 3 || calls < 1) {
    fprintf(stderr, "n >= 3 and calls >= 1\n");
    return 1;
  }
  jacc_loop loops[2] = {{1, n - 2, 1}, {1, n - 2, 1}};
  jacc_ref refs[6];
  memset(refs, 0, sizeof(refs));
  const long long offs[5][2] = {{0, -1}, {0, 1}, {-1, 0}, {1, 0}, {0, 0}};
  for (int r = 0; r < 6; ++r) {
    refs[r].array_id = r < 5 ? 0 : 1;
    refs[r].ndim = 2;
    refs[r].is_write = r == 5;
    refs[r].coef[0][0] = 1; /* subscript 0 (row) follows loop 0 */
    refs[r].coef[1][1] = 1; /* subscript 1 (column) follows loop 1 */
    if (r < 5) {
      refs[r].off[0] = offs[r][0];
      refs[r].off[1] = offs[r][1];
    }
  }
  jacc_array arrays[2];
  memset(arrays, 0, sizeof(arrays));
  for (int a = 0; a < 2; ++a) {
    arrays[a].ndim = 2;
    arrays[a].extent[0] = arrays[a].extent[1] = n;
  }
  jacc_region out[2];
  jacc_status st = JACC_OK;
  for (int w = 0; w < 100 && st == JACC_OK; ++w) st = jacc_region_analyze(2, loops, 6, refs, 2, arrays, out);
  const double t0 = now_us();
  for (int c = 0; c < calls && st == JACC_OK; ++c) st = jacc_region_analyze(2, loops, 6, refs, 2, arrays, out);
  const double t1 = now_us();
  if (st != JACC_OK) {
    fprintf(stderr, "jacc_region_analyze: %s\n", jacc_last_error());
    return 1;
  }
  printf("write [%lld,%lld]x[%lld,%lld] linear [%lld,%lld]; read [%lld,%lld]x[%lld,%lld] linear [%lld,%lld]\n",
         (long long)out[1].wlo[0], (long long)out[1].whi[0], (long long)out[1].wlo[1], (long long)out[1].whi[1],
         (long long)out[1].wlin_lo, (long long)out[1].wlin_hi, (long long)out[0].rlo[0], (long long)out[0].rhi[0],
         (long long)out[0].rlo[1], (long long)out[0].rhi[1], (long long)out[0].rlin_lo, (long long)out[0].rlin_hi);
  printf("us_per_call %.4f\n", (t1 - t0) / calls);
  return 0;
}
