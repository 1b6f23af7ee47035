/*
 * CPU oracle for the runtime-specialised affine stencil path (JACC, arXiv
 * 2110.14340).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check
 * and the benchmark's CPU-baseline leg; never by the product path.
 *
 * Each function states the definition it follows.  Nothing here is blocked,
 * fused or reordered beyond what that definition states; the code is meant to
 * be checked against the definitions by eye.  Compiled with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * What pins each part (tests/test_oracle_*.py):
 *   region analysis  - brute-force enumeration of every iteration of random
 *                      tiny nests; hand-derived hulls of the paper's own loop
 *                      examples (Listing 1, Listing 5).
 *   Jacobi 2D        - affine fields are exact fixed points; sine modes decay
 *                      by their closed-form eigenvalue; maximum principle;
 *                      monotone residual.
 *   heat 3D          - discrete sine eigenmode decays by lambda^n; affine
 *                      fields are fixed points; maximum principle.
 *   27-point box     - impulse response equals the class weights; constant
 *                      fields scale by the weight sum; sum scales by W^n;
 *                      plane waves decay by the closed-form symbol.
 *   reductions       - exact (fsum) sums within the pairwise error bound.
 *   MLP              - central finite differences of the loss; closed-form
 *                      first Adam step; exact fit of a representable target.
 *   regret           - hand-computed tables.
 *   threads          - every sweep and sum on 2..n threads is bit-identical
 *                      to the same call on one thread (the threads only split
 *                      the outermost loop, or the top of the sum's recursion).
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Region analysis.                                                           */
/*                                                                            */
/* The runtime tracks, per array, the index range a kernel launch reads and   */
/* the range it writes (data ranges linked to pointers, §3.2.1; per-array     */
/* lower/upper write bounds a_lb/a_ub, §4.1).  When several references        */
/* touch one array their ranges are merged to the widest (§4.1).  Reads and   */
/* writes are kept apart because the paper treats read and written pointers   */
/* differently (§4.1, aliasing rule).                                         */
/*                                                                            */
/* For a rectangular nest, an affine subscript off + sum_k c_k i_k reaches    */
/* its minimum and maximum at loop endpoints chosen independently per loop,   */
/* because the iteration domain is a product of arithmetic progressions.      */
/* The flattened (row-major) element offset is again affine in i, so its      */
/* exact extremes follow from the same rule.                                  */
/*                                                                            */
/* Overflow semantics: ORC_ERR_OVERFLOW when any product coefficient x loop   */
/* endpoint, any stride, any flattened coefficient or offset, or any final    */
/* bound does not fit in int64.  Partial sums are exact (128-bit).            */
/* ------------------------------------------------------------------------- */

typedef __int128 i128;

static int fits64(i128 x) { return x >= (i128)INT64_MIN && x <= (i128)INT64_MAX; }

/* First and last value of one loop; returns the iteration count (0 if empty). */
static i128 loop_span(const orc_loop* L, i128* first, i128* last) {
  i128 lo = L->lo, hi = L->hi, s = L->step;
  i128 cnt;
  if (s > 0) cnt = (hi >= lo) ? (hi - lo) / s + 1 : 0;
  else cnt = (lo >= hi) ? (lo - hi) / (-s) + 1 : 0;
  *first = lo;
  *last = lo + (cnt > 0 ? (cnt - 1) * s : 0);
  return cnt;
}

/* Exact min/max of off + sum_k c[k] * i_k over the nest. */
static int affine_extremes(int32_t nloops, const i128* first, const i128* last, const int64_t* c, i128 off,
                           i128* mn, i128* mx) {
  i128 lo = off, hi = off;
  for (int k = 0; k < nloops; ++k) {
    i128 a = (i128)c[k] * first[k];
    i128 b = (i128)c[k] * last[k];
    if (!fits64(a) || !fits64(b)) return ORC_ERR_OVERFLOW;
    lo += (a < b) ? a : b;
    hi += (a < b) ? b : a;
  }
  if (!fits64(lo) || !fits64(hi)) return ORC_ERR_OVERFLOW;
  *mn = lo;
  *mx = hi;
  return ORC_OK;
}

/* Visit every iteration of an affine-bounded nest, recording each
 * reference's subscripts and flattened offset. */
typedef struct {
  int32_t nloops, nrefs;
  const orc_loop_affine* loops;
  const orc_ref* refs;
  const orc_array* arrays;
  orc_region* out;
  int64_t idx[ORC_MAX_LOOPS];
  int64_t visits;
} enum_state;

static void enum_touch(enum_state* S) {
  for (int r = 0; r < S->nrefs; ++r) {
    const orc_ref* R = &S->refs[r];
    const orc_array* A = &S->arrays[R->array_id];
    orc_region* O = &S->out[R->array_id];
    const int w = R->is_write != 0;
    int64_t* lo = w ? O->wlo : O->rlo;
    int64_t* hi = w ? O->whi : O->rhi;
    int64_t* llo = w ? &O->wlin_lo : &O->rlin_lo;
    int64_t* lhi = w ? &O->wlin_hi : &O->rlin_hi;
    int32_t* has = w ? &O->has_write : &O->has_read;
    int64_t flat = 0;
    for (int d = 0; d < R->ndim; ++d) {
      int64_t e = R->off[d];
      for (int k = 0; k < S->nloops; ++k) e += R->coef[d][k] * S->idx[k];
      if (!*has || e < lo[d]) lo[d] = e;
      if (!*has || e > hi[d]) hi[d] = e;
      flat = flat * (d == 0 ? 1 : A->extent[d]) + e;
    }
    if (!*has || flat < *llo) *llo = flat;
    if (!*has || flat > *lhi) *lhi = flat;
    *has = 1;
  }
}

static void enum_loop(enum_state* S, int k) {
  if (k == S->nloops) {
    ++S->visits;
    enum_touch(S);
    return;
  }
  const orc_loop_affine* L = &S->loops[k];
  int64_t lo = L->lo, hi = L->hi;
  for (int m = 0; m < k; ++m) {
    lo += L->lo_coef[m] * S->idx[m];
    hi += L->hi_coef[m] * S->idx[m];
  }
  for (int64_t i = lo; i <= hi && S->visits < (1 << 22); ++i) {
    S->idx[k] = i;
    enum_loop(S, k + 1);
  }
}

int orc_region_enumerate_affine(int32_t nloops, const orc_loop_affine* loops, int32_t nrefs, const orc_ref* refs,
                                int32_t narrays, const orc_array* arrays, orc_region* out) {
  if (nloops < 0 || nloops > ORC_MAX_LOOPS || nrefs < 0 || narrays < 0) return ORC_ERR_INVALID_ARG;
  for (int a = 0; a < narrays; ++a) memset(&out[a], 0, sizeof(orc_region));
  enum_state S;
  S.nloops = nloops;
  S.nrefs = nrefs;
  S.loops = loops;
  S.refs = refs;
  S.arrays = arrays;
  S.out = out;
  S.visits = 0;
  enum_loop(&S, 0);
  return S.visits >= (1 << 22) ? ORC_ERR_INVALID_ARG : ORC_OK;
}

int orc_region_analyze(int32_t nloops, const orc_loop* loops, int32_t nrefs, const orc_ref* refs,
                       int32_t narrays, const orc_array* arrays, orc_region* out) {
  if (nloops < 0 || nloops > ORC_MAX_LOOPS || nrefs < 0 || narrays < 0) return ORC_ERR_INVALID_ARG;
  if ((nloops > 0 && !loops) || (nrefs > 0 && !refs) || (narrays > 0 && (!arrays || !out)))
    return ORC_ERR_INVALID_ARG;
  for (int k = 0; k < nloops; ++k)
    if (loops[k].step == 0) return ORC_ERR_INVALID_ARG;
  for (int a = 0; a < narrays; ++a) {
    if (arrays[a].ndim < 1 || arrays[a].ndim > ORC_MAX_DIMS) return ORC_ERR_INVALID_ARG;
    for (int d = 0; d < arrays[a].ndim; ++d)
      if (arrays[a].extent[d] < 0) return ORC_ERR_INVALID_ARG;
  }
  for (int r = 0; r < nrefs; ++r) {
    if (refs[r].array_id < 0 || refs[r].array_id >= narrays) return ORC_ERR_INVALID_ARG;
    if (refs[r].ndim != arrays[refs[r].array_id].ndim) return ORC_ERR_INVALID_ARG;
  }

  for (int a = 0; a < narrays; ++a) memset(&out[a], 0, sizeof(orc_region));

  i128 first[ORC_MAX_LOOPS], last[ORC_MAX_LOOPS];
  int empty = 0;
  for (int k = 0; k < nloops; ++k)
    if (loop_span(&loops[k], &first[k], &last[k]) == 0) empty = 1;
  if (empty) return ORC_OK; /* no iteration touches anything */

  for (int r = 0; r < nrefs; ++r) {
    const orc_ref* R = &refs[r];
    const orc_array* A = &arrays[R->array_id];
    orc_region* O = &out[R->array_id];
    const int w = R->is_write != 0;

    /* Per-dimension hull. */
    i128 mn[ORC_MAX_DIMS], mx[ORC_MAX_DIMS];
    for (int d = 0; d < R->ndim; ++d) {
      int st = affine_extremes(nloops, first, last, R->coef[d], R->off[d], &mn[d], &mx[d]);
      if (st) return st;
    }

    /* Flattened row-major offset: stride[nd-1] = 1, stride[d] = stride[d+1] * extent[d+1]. */
    i128 stride[ORC_MAX_DIMS];
    stride[R->ndim - 1] = 1;
    for (int d = R->ndim - 2; d >= 0; --d) {
      stride[d] = stride[d + 1] * (i128)A->extent[d + 1];
      if (!fits64(stride[d])) return ORC_ERR_OVERFLOW;
    }
    int64_t lc[ORC_MAX_LOOPS];
    for (int k = 0; k < nloops; ++k) {
      i128 s = 0;
      for (int d = 0; d < R->ndim; ++d) {
        i128 t = stride[d] * (i128)R->coef[d][k];
        if (!fits64(t)) return ORC_ERR_OVERFLOW;
        s += t;
      }
      if (!fits64(s)) return ORC_ERR_OVERFLOW;
      lc[k] = (int64_t)s;
    }
    i128 loff = 0;
    for (int d = 0; d < R->ndim; ++d) {
      i128 t = stride[d] * (i128)R->off[d];
      if (!fits64(t)) return ORC_ERR_OVERFLOW;
      loff += t;
    }
    if (!fits64(loff)) return ORC_ERR_OVERFLOW;
    i128 lmn, lmx;
    int st = affine_extremes(nloops, first, last, lc, loff, &lmn, &lmx);
    if (st) return st;

    /* Merge to the widest range. */
    int64_t* lo = w ? O->wlo : O->rlo;
    int64_t* hi = w ? O->whi : O->rhi;
    int64_t* llo = w ? &O->wlin_lo : &O->rlin_lo;
    int64_t* lhi = w ? &O->wlin_hi : &O->rlin_hi;
    int32_t* has = w ? &O->has_write : &O->has_read;
    for (int d = 0; d < R->ndim; ++d) {
      if (!*has || (int64_t)mn[d] < lo[d]) lo[d] = (int64_t)mn[d];
      if (!*has || (int64_t)mx[d] > hi[d]) hi[d] = (int64_t)mx[d];
    }
    if (!*has || (int64_t)lmn < *llo) *llo = (int64_t)lmn;
    if (!*has || (int64_t)lmx > *lhi) *lhi = (int64_t)lmx;
    *has = 1;
  }

  int oob = 0;
  for (int a = 0; a < narrays; ++a) {
    const orc_region* O = &out[a];
    for (int d = 0; d < arrays[a].ndim; ++d) {
      int64_t ext = arrays[a].extent[d];
      if (O->has_read && (O->rlo[d] < 0 || O->rhi[d] > ext - 1)) oob = 1;
      if (O->has_write && (O->wlo[d] < 0 || O->whi[d] > ext - 1)) oob = 1;
    }
  }
  return oob ? ORC_ERR_OUT_OF_BOUNDS : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Stencils.  The paper's workloads are memory-bound halo stencils (§5.2,     */
/* Table 1: Himeno's Jacobi sweep, CloverLeaf's 2D halo kernels); these are   */
/* the 5-, 7- and 27-point members of that family, written as plain loops.    */
/* ------------------------------------------------------------------------- */

/* ------------------------------------------------------------------------- */
/* Threads.  A sweep may split its outermost loop (rows in 2D, planes in 3D)  */
/* into contiguous slabs, one per thread.  Each thread runs the loop body of  */
/* the single-thread sweep over its slab, so every output value comes from    */
/* the same statements in the same order, and the residual (a maximum, which  */
/* does not depend on the order it is taken in) is the same bits.  The count  */
/* is a process-wide setting, 1 by default.                                   */
/* ------------------------------------------------------------------------- */

#define ORC_MAX_THREADS 256
static int g_nthreads = 1;

int32_t orc_set_threads(int32_t n) {
  g_nthreads = n < 1 ? 1 : (n > ORC_MAX_THREADS ? ORC_MAX_THREADS : n);
  return g_nthreads;
}

int32_t orc_get_threads(void) { return g_nthreads; }

/* A slab body: the sweep's loop over outer indices [lo, hi); returns the
 * largest |v - u| it saw (0 where the sweep has no residual). */
typedef double (*slab_fn)(const void* args, int64_t lo, int64_t hi);

typedef struct {
  slab_fn fn;
  const void* args;
  int64_t lo, hi;
  double res;
} slab_job;

static void* slab_main(void* p) {
  slab_job* j = (slab_job*)p;
  j->res = j->fn(j->args, j->lo, j->hi);
  return NULL;
}

/* Runs fn over [0, n) in up to g_nthreads contiguous slabs; returns the
 * largest residual.  A thread that cannot be started runs on the caller. */
static double run_slabs(slab_fn fn, const void* args, int64_t n) {
  int64_t T = g_nthreads < n ? g_nthreads : n;
  if (T <= 1) return fn(args, 0, n);
  slab_job job[ORC_MAX_THREADS];
  pthread_t th[ORC_MAX_THREADS];
  int started[ORC_MAX_THREADS];
  for (int64_t t = 0; t < T; ++t) {
    job[t].fn = fn;
    job[t].args = args;
    job[t].lo = n * t / T;
    job[t].hi = n * (t + 1) / T;
    job[t].res = 0.0;
  }
  for (int64_t t = 1; t < T; ++t) started[t] = pthread_create(&th[t], NULL, slab_main, &job[t]) == 0;
  slab_main(&job[0]);
  for (int64_t t = 1; t < T; ++t) {
    if (started[t]) pthread_join(th[t], NULL);
    else slab_main(&job[t]);
  }
  double res = 0.0;
  for (int64_t t = 0; t < T; ++t)
    if (job[t].res > res) res = job[t].res;
  return res;
}

/* v[y][x] = 0.25 * ((u[y-1][x] + u[y+1][x]) + (u[y][x-1] + u[y][x+1])) on the
 * interior; boundary rows and columns are held (copied).  Residual: the
 * largest |v - u| over the interior, i.e. the change made by this sweep. */
typedef struct {
  int64_t nx, ny;
  const double* u;
  double* v;
} jacobi2d_args;

static double jacobi2d_rows(const void* args, int64_t y0, int64_t y1) {
  const jacobi2d_args* A = (const jacobi2d_args*)args;
  const int64_t nx = A->nx, ny = A->ny;
  const double* u = A->u;
  double* v = A->v;
  double res = 0.0;
  for (int64_t y = y0; y < y1; ++y) {
    for (int64_t x = 0; x < nx; ++x) {
      int64_t c = y * nx + x;
      if (y == 0 || y == ny - 1 || x == 0 || x == nx - 1) {
        v[c] = u[c];
        continue;
      }
      double s = (u[c - nx] + u[c + nx]) + (u[c - 1] + u[c + 1]);
      v[c] = 0.25 * s;
      double d = fabs(v[c] - u[c]);
      if (d > res) res = d;
    }
  }
  return res;
}

double orc_jacobi2d_sweep(int64_t nx, int64_t ny, const double* u, double* v) {
  jacobi2d_args A = {nx, ny, u, v};
  return run_slabs(jacobi2d_rows, &A, ny);
}

int orc_jacobi2d_run(int64_t nx, int64_t ny, double* u0, double* u1, int32_t nsweeps, double* resid) {
  double* a = u0;
  double* b = u1;
  for (int32_t k = 0; k < nsweeps; ++k) {
    double r = orc_jacobi2d_sweep(nx, ny, a, b);
    if (resid) resid[k] = r;
    double* t = a;
    a = b;
    b = t;
  }
  return (nsweeps % 2 == 0) ? 0 : 1;
}

/* Explicit heat step: v = u + r * ((((xm + xp) + (ym + yp)) + (zm + zp)) - 6 u)
 * on the interior; Dirichlet boundary values are held.  Residual: largest
 * |v - u| over the interior. */
typedef struct {
  int64_t nx, ny, nz;
  double r;
  const double* u;
  double* v;
} heat3d_args;

static double heat3d_planes(const void* args, int64_t z0, int64_t z1) {
  const heat3d_args* A = (const heat3d_args*)args;
  const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
  const double r = A->r;
  const double* u = A->u;
  double* v = A->v;
  const int64_t sy = nx, sz = nx * ny;
  double res = 0.0;
  for (int64_t z = z0; z < z1; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t c = z * sz + y * sy + x;
        if (z == 0 || z == nz - 1 || y == 0 || y == ny - 1 || x == 0 || x == nx - 1) {
          v[c] = u[c];
          continue;
        }
        double lap = (((u[c - 1] + u[c + 1]) + (u[c - sy] + u[c + sy])) + (u[c - sz] + u[c + sz])) - 6.0 * u[c];
        v[c] = u[c] + r * lap;
        double d = fabs(v[c] - u[c]);
        if (d > res) res = d;
      }
  return res;
}

double orc_heat3d_sweep(int64_t nx, int64_t ny, int64_t nz, double r, const double* u, double* v) {
  heat3d_args A = {nx, ny, nz, r, u, v};
  return run_slabs(heat3d_planes, &A, nz);
}

int orc_heat3d_run(int64_t nx, int64_t ny, int64_t nz, double r, double* u0, double* u1, int32_t nsweeps,
                   double* resid) {
  double* a = u0;
  double* b = u1;
  for (int32_t k = 0; k < nsweeps; ++k) {
    double rr = orc_heat3d_sweep(nx, ny, nz, r, a, b);
    if (resid) resid[k] = rr;
    double* t = a;
    a = b;
    b = t;
  }
  return (nsweeps % 2 == 0) ? 0 : 1;
}

/* Variable-coefficient 19-point Jacobi step (see oracle.h for the formula). */
double orc_var19_sweep(int64_t nx, int64_t ny, int64_t nz, float omega, const float* const* c, const float* p,
                       float* v) {
  const int64_t sy = nx, sz = nx * ny;
  const float *a0 = c[0], *a1 = c[1], *a2 = c[2], *a3 = c[3], *b0 = c[4], *b1 = c[5], *b2 = c[6];
  const float *c0 = c[7], *c1 = c[8], *c2 = c[9], *wrk1 = c[10], *bnd = c[11];
  double gosa = 0.0;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        const int64_t i = z * sz + y * sy + x;
        if (z == 0 || z == nz - 1 || y == 0 || y == ny - 1 || x == 0 || x == nx - 1) {
          v[i] = p[i];
          continue;
        }
        float s0 = a0[i] * p[i + 1] + a1[i] * p[i + sy] + a2[i] * p[i + sz];
        s0 = s0 + b0[i] * (p[i + 1 + sy] - p[i + 1 - sy] - p[i - 1 + sy] + p[i - 1 - sy]);
        s0 = s0 + b1[i] * (p[i + sy + sz] - p[i - sy + sz] - p[i + sy - sz] + p[i - sy - sz]);
        s0 = s0 + b2[i] * (p[i + 1 + sz] - p[i - 1 + sz] - p[i + 1 - sz] + p[i - 1 - sz]);
        s0 = s0 + c0[i] * p[i - 1] + c1[i] * p[i - sy] + c2[i] * p[i - sz] + wrk1[i];
        const float ss = (s0 * a3[i] - p[i]) * bnd[i];
        v[i] = p[i] + omega * ss;
        gosa += (double)ss * (double)ss;
      }
  return gosa;
}

int orc_var19_run(int64_t nx, int64_t ny, int64_t nz, float omega, const float* const* c, float* u0, float* u1,
                  int32_t nsweeps, double* resid) {
  float* a = u0;
  float* b = u1;
  for (int32_t k = 0; k < nsweeps; ++k) {
    const double g = orc_var19_sweep(nx, ny, nz, omega, c, a, b);
    if (resid) resid[k] = g;
    float* t = a;
    a = b;
    b = t;
  }
  return (nsweeps % 2 == 0) ? 0 : 1;
}

/* 27-point periodic stencil in FP32.  Offsets (dx,dy,dz) in {-1,0,1}^3 are
 * classed by how many are non-zero: 0 centre, 1 face (6), 2 edge (12),
 * 3 corner (8).  v = w0*centre + wf*F + we*E + wc*C, where F, E, C are the
 * class sums taken in offset order dz, dy, dx = -1..1.  Indices wrap: the
 * wrapped neighbour index of each axis, (i + d + n) % n, is formed once per
 * index instead of once per neighbour. */
typedef struct {
  int64_t nx, ny, nz;
  const float* w;
  const float* u;
  float* v;
} box27_args;

static double box27_planes(const void* args, int64_t z0, int64_t z1) {
  const box27_args* A = (const box27_args*)args;
  const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
  const float* w = A->w;
  const float* u = A->u;
  float* v = A->v;
  for (int64_t z = z0; z < z1; ++z) {
    int64_t zw[3];
    for (int d = -1; d <= 1; ++d) zw[d + 1] = (z + d + nz) % nz;
    for (int64_t y = 0; y < ny; ++y) {
      int64_t yw[3];
      for (int d = -1; d <= 1; ++d) yw[d + 1] = (y + d + ny) % ny;
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xw[3];
        for (int d = -1; d <= 1; ++d) xw[d + 1] = (x + d + nx) % nx;
        float cls[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int k = (dz != 0) + (dy != 0) + (dx != 0);
              cls[k] = cls[k] + u[(zw[dz + 1] * ny + yw[dy + 1]) * nx + xw[dx + 1]];
            }
        float acc = w[0] * cls[0];
        acc = acc + w[1] * cls[1];
        acc = acc + w[2] * cls[2];
        acc = acc + w[3] * cls[3];
        v[(z * ny + y) * nx + x] = acc;
      }
    }
  }
  return 0.0;
}

void orc_box27_sweep(int64_t nx, int64_t ny, int64_t nz, const float w[4], const float* u, float* v) {
  box27_args A = {nx, ny, nz, w, u, v};
  run_slabs(box27_planes, &A, nz);
}

int orc_box27_run(int64_t nx, int64_t ny, int64_t nz, const float w[4], float* u0, float* u1, int32_t nsweeps,
                  double* sums) {
  float* a = u0;
  float* b = u1;
  for (int32_t k = 0; k < nsweeps; ++k) {
    orc_box27_sweep(nx, ny, nz, w, a, b);
    if (sums) sums[k] = orc_sum_f32(b, nx * ny * nz);
    float* t = a;
    a = b;
    b = t;
  }
  return (nsweeps % 2 == 0) ? 0 : 1;
}

/* The same definition with FP64 storage and arithmetic. */
typedef struct {
  int64_t nx, ny, nz;
  const double* w;
  const double* u;
  double* v;
} box27_f64_args;

static double box27_f64_planes(const void* args, int64_t z0, int64_t z1) {
  const box27_f64_args* A = (const box27_f64_args*)args;
  const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
  const double* w = A->w;
  const double* u = A->u;
  double* v = A->v;
  for (int64_t z = z0; z < z1; ++z) {
    int64_t zw[3];
    for (int d = -1; d <= 1; ++d) zw[d + 1] = (z + d + nz) % nz;
    for (int64_t y = 0; y < ny; ++y) {
      int64_t yw[3];
      for (int d = -1; d <= 1; ++d) yw[d + 1] = (y + d + ny) % ny;
      for (int64_t x = 0; x < nx; ++x) {
        int64_t xw[3];
        for (int d = -1; d <= 1; ++d) xw[d + 1] = (x + d + nx) % nx;
        double cls[4] = {0.0, 0.0, 0.0, 0.0};
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int k = (dz != 0) + (dy != 0) + (dx != 0);
              cls[k] = cls[k] + u[(zw[dz + 1] * ny + yw[dy + 1]) * nx + xw[dx + 1]];
            }
        double acc = w[0] * cls[0];
        acc = acc + w[1] * cls[1];
        acc = acc + w[2] * cls[2];
        acc = acc + w[3] * cls[3];
        v[(z * ny + y) * nx + x] = acc;
      }
    }
  }
  return 0.0;
}

void orc_box27_sweep_f64(int64_t nx, int64_t ny, int64_t nz, const double w[4], const double* u, double* v) {
  box27_f64_args A = {nx, ny, nz, w, u, v};
  run_slabs(box27_f64_planes, &A, nz);
}

int orc_box27_run_f64(int64_t nx, int64_t ny, int64_t nz, const double w[4], double* u0, double* u1, int32_t nsweeps,
                      double* sums) {
  double* a = u0;
  double* b = u1;
  for (int32_t k = 0; k < nsweeps; ++k) {
    orc_box27_sweep_f64(nx, ny, nz, w, a, b);
    if (sums) sums[k] = orc_sum_f64(b, nx * ny * nz);
    double* t = a;
    a = b;
    b = t;
  }
  return (nsweeps % 2 == 0) ? 0 : 1;
}

/* ------------------------------------------------------------------------- */
/* Reductions (FP64 accumulation).  The runtime must synchronise after a      */
/* reduction (§3.2.1); the reduction itself is the plain definition.          */
/* ------------------------------------------------------------------------- */

double orc_maxabs_diff(const double* a, const double* b, int64_t n) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = fabs(a[i] - b[i]);
    if (d > m) m = d;
  }
  return m;
}

/* Pairwise (cascade) summation: error O(log n * eps * sum|a|).  The
 * recursion halves the range (first half n/2 elements) down to runs of at
 * most 8, summed left to right. */
static double sum_f64_seq(const double* a, int64_t n) {
  if (n <= 8) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i];
    return s;
  }
  int64_t h = n / 2;
  return sum_f64_seq(a, h) + sum_f64_seq(a + h, n - h);
}

static double sum_f32_seq(const float* a, int64_t n) {
  if (n <= 8) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += (double)a[i];
    return s;
  }
  int64_t h = n / 2;
  return sum_f32_seq(a, h) + sum_f32_seq(a + h, n - h);
}

/* With threads, the top `depth` levels of the same recursion are unrolled:
 * its subranges at that depth are summed in parallel (each by the recursion
 * above) and their sums combined in the recursion's own pairing, so the
 * result is bit-identical to the single-thread sum. */
typedef struct {
  const void* a;
  int64_t n;
  int f32;
  double s;
} sum_job;

static void* sum_main(void* p) {
  sum_job* j = (sum_job*)p;
  j->s = j->f32 ? sum_f32_seq((const float*)j->a, j->n) : sum_f64_seq((const double*)j->a, j->n);
  return NULL;
}

static void sum_leaves(const char* a, int64_t n, int64_t esz, int f32, int depth, sum_job* leaf, int* nl) {
  if (depth == 0 || n <= 8) {
    leaf[*nl].a = a;
    leaf[*nl].n = n;
    leaf[*nl].f32 = f32;
    leaf[*nl].s = 0.0;
    ++*nl;
    return;
  }
  int64_t h = n / 2;
  sum_leaves(a, h, esz, f32, depth - 1, leaf, nl);
  sum_leaves(a + h * esz, n - h, esz, f32, depth - 1, leaf, nl);
}

static double sum_combine(int64_t n, int depth, const sum_job* leaf, int* i) {
  if (depth == 0 || n <= 8) return leaf[(*i)++].s;
  int64_t h = n / 2;
  double l = sum_combine(h, depth - 1, leaf, i);
  double r = sum_combine(n - h, depth - 1, leaf, i);
  return l + r;
}

static double sum_threaded(const void* a, int64_t n, int64_t esz, int f32) {
  int depth = 0;
  while ((1 << depth) < g_nthreads && depth < 8) ++depth;
  sum_job leaf[ORC_MAX_THREADS];
  pthread_t th[ORC_MAX_THREADS];
  int started[ORC_MAX_THREADS];
  int nl = 0;
  sum_leaves((const char*)a, n, esz, f32, depth, leaf, &nl);
  for (int t = 1; t < nl; ++t) started[t] = pthread_create(&th[t], NULL, sum_main, &leaf[t]) == 0;
  sum_main(&leaf[0]);
  for (int t = 1; t < nl; ++t) {
    if (started[t]) pthread_join(th[t], NULL);
    else sum_main(&leaf[t]);
  }
  int i = 0;
  return sum_combine(n, depth, leaf, &i);
}

double orc_sum_f64(const double* a, int64_t n) {
  if (g_nthreads > 1 && n >= (1 << 16)) return sum_threaded(a, n, sizeof(double), 0);
  return sum_f64_seq(a, n);
}

double orc_sum_f32(const float* a, int64_t n) {
  if (g_nthreads > 1 && n >= (1 << 16)) return sum_threaded(a, n, sizeof(float), 1);
  return sum_f32_seq(a, n);
}

/* ------------------------------------------------------------------------- */
/* MLP cost model (no counterpart in the paper, which names auto-tuning as    */
/* future work, §8).  4 -> 64 -> 64 -> 64 -> 1, ReLU, mean squared error.      */
/* ------------------------------------------------------------------------- */

enum { H = 64, NIN = 4 };
enum {
  OFF_W1 = 0,
  OFF_B1 = OFF_W1 + H * NIN,
  OFF_W2 = OFF_B1 + H,
  OFF_B2 = OFF_W2 + H * H,
  OFF_W3 = OFF_B2 + H,
  OFF_B3 = OFF_W3 + H * H,
  OFF_W4 = OFF_B3 + H,
  OFF_B4 = OFF_W4 + H,
  OFF_END = OFF_B4 + 1
};

typedef struct { double z1[H], h1[H], z2[H], h2[H], z3[H], h3[H], y; } mlp_act;

static double relu(double z) { return z > 0.0 ? z : 0.0; }

static void mlp_fwd1(const double* p, const double* x, mlp_act* a) {
  for (int o = 0; o < H; ++o) {
    double s = p[OFF_B1 + o];
    for (int i = 0; i < NIN; ++i) s += p[OFF_W1 + o * NIN + i] * x[i];
    a->z1[o] = s;
    a->h1[o] = relu(s);
  }
  for (int o = 0; o < H; ++o) {
    double s = p[OFF_B2 + o];
    for (int i = 0; i < H; ++i) s += p[OFF_W2 + o * H + i] * a->h1[i];
    a->z2[o] = s;
    a->h2[o] = relu(s);
  }
  for (int o = 0; o < H; ++o) {
    double s = p[OFF_B3 + o];
    for (int i = 0; i < H; ++i) s += p[OFF_W3 + o * H + i] * a->h2[i];
    a->z3[o] = s;
    a->h3[o] = relu(s);
  }
  double s = p[OFF_B4];
  for (int i = 0; i < H; ++i) s += p[OFF_W4 + i] * a->h3[i];
  a->y = s;
}

void orc_mlp_forward(const double* p, const double* x, int64_t n, double* y) {
  mlp_act a;
  for (int64_t s = 0; s < n; ++s) {
    mlp_fwd1(p, x + s * NIN, &a);
    y[s] = a.y;
  }
}

double orc_mlp_loss_grad(const double* p, const double* x, const double* t, int64_t n, double* g) {
  memset(g, 0, sizeof(double) * OFF_END);
  double loss = 0.0;
  mlp_act a;
  double d3[H], d2[H], d1[H];
  for (int64_t s = 0; s < n; ++s) {
    const double* xs = x + s * NIN;
    mlp_fwd1(p, xs, &a);
    double e = a.y - t[s];
    loss += e * e;
    double dy = 2.0 * e / (double)n; /* d(mean e^2)/dy */
    g[OFF_B4] += dy;
    for (int i = 0; i < H; ++i) g[OFF_W4 + i] += dy * a.h3[i];
    for (int i = 0; i < H; ++i) d3[i] = (a.z3[i] > 0.0) ? dy * p[OFF_W4 + i] : 0.0;
    for (int o = 0; o < H; ++o) {
      g[OFF_B3 + o] += d3[o];
      for (int i = 0; i < H; ++i) g[OFF_W3 + o * H + i] += d3[o] * a.h2[i];
    }
    for (int i = 0; i < H; ++i) {
      double s2 = 0.0;
      for (int o = 0; o < H; ++o) s2 += p[OFF_W3 + o * H + i] * d3[o];
      d2[i] = (a.z2[i] > 0.0) ? s2 : 0.0;
    }
    for (int o = 0; o < H; ++o) {
      g[OFF_B2 + o] += d2[o];
      for (int i = 0; i < H; ++i) g[OFF_W2 + o * H + i] += d2[o] * a.h1[i];
    }
    for (int i = 0; i < H; ++i) {
      double s1 = 0.0;
      for (int o = 0; o < H; ++o) s1 += p[OFF_W2 + o * H + i] * d2[o];
      d1[i] = (a.z1[i] > 0.0) ? s1 : 0.0;
    }
    for (int o = 0; o < H; ++o) {
      g[OFF_B1 + o] += d1[o];
      for (int i = 0; i < NIN; ++i) g[OFF_W1 + o * NIN + i] += d1[o] * xs[i];
    }
  }
  return loss / (double)n;
}

/* Adam (Kingma and Ba, 2015) with bias correction. */
void orc_adam_step(double* p, const double* g, double* m, double* v, int64_t n, int64_t t, double lr,
                   double beta1, double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, (double)t);
  double c2 = 1.0 - pow(beta2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    double mh = m[i] / c1;
    double vh = v[i] / c2;
    p[i] = p[i] - lr * mh / (sqrt(vh) + eps);
  }
}

void orc_regret(const double* times, int32_t nq, int32_t ntile, const int32_t* pick, double* regret) {
  for (int32_t q = 0; q < nq; ++q) {
    const double* row = times + (int64_t)q * ntile;
    double best = row[0];
    for (int32_t j = 1; j < ntile; ++j)
      if (row[j] < best) best = row[j];
    regret[q] = row[pick[q]] / best - 1.0;
  }
}
