/*
 * CPU oracle for the runtime-specialised affine stencil path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * restatement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * product path never calls it.
 *
 * Precision: FP64 for the FP64 stencils, the reductions and the MLP; FP32
 * storage and arithmetic for the 27-point FP32 stencil (the precision that
 * stencil is defined in).  Built with -ffp-contract=off so every product and
 * sum is rounded exactly as written.
 */
#ifndef JACC_ORACLE_H
#define JACC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_DIMS 8
#define ORC_MAX_LOOPS 8

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = -1,
  ORC_ERR_OUT_OF_BOUNDS = -2,
  ORC_ERR_OVERFLOW = -3
};

/* One loop of a rectangular nest: i = lo, lo+step, ... while i <= hi (step > 0)
 * or while i >= hi (step < 0). */
typedef struct { int64_t lo, hi, step; } orc_loop;

/* An affine array reference A[e_0]...[e_{ndim-1}],
 * e_d = off[d] + sum_k coef[d][k] * i_k. */
typedef struct {
  int32_t array_id;
  int32_t ndim;
  int32_t is_write;
  int32_t pad_;
  int64_t coef[ORC_MAX_DIMS][ORC_MAX_LOOPS];
  int64_t off[ORC_MAX_DIMS];
} orc_ref;

typedef struct { int32_t ndim; int32_t pad_; int64_t extent[ORC_MAX_DIMS]; } orc_array;

typedef struct {
  int32_t has_read, has_write;
  int64_t rlo[ORC_MAX_DIMS], rhi[ORC_MAX_DIMS];
  int64_t wlo[ORC_MAX_DIMS], whi[ORC_MAX_DIMS];
  int64_t rlin_lo, rlin_hi, wlin_lo, wlin_hi;
} orc_region;

/* A loop with affine bounds: i_k = lo_k .. hi_k step 1, lo_k = lo + sum_{m<k}
 * lo_coef[m] i_m, hi_k likewise (the layout of jacc_loop_affine). */
typedef struct {
  int64_t lo, hi;
  int64_t lo_coef[ORC_MAX_LOOPS];
  int64_t hi_coef[ORC_MAX_LOOPS];
} orc_loop_affine;

/* Threads for the stencil sweeps and the large sums (default 1).  A sweep
 * splits its outermost loop into contiguous slabs, one per thread, each
 * running the single-thread loop body; a sum unrolls the top levels of its
 * pairwise recursion across threads.  Results are bit-identical to one
 * thread for every count.  The variable-coefficient 19-point sweep, whose
 * residual is a sum taken in loop order, always runs on one thread.
 * Returns the count in effect (clamped to [1, 256]). */
int32_t orc_set_threads(int32_t n);
int32_t orc_get_threads(void);

/* Region of an affine-bounded nest by enumerating every iteration (small
 * nests only: at most 2^22 iterations, else ORC_ERR_INVALID_ARG).  Same
 * output as orc_region_analyze; no bounds check. */
int orc_region_enumerate_affine(int32_t nloops, const orc_loop_affine* loops, int32_t nrefs, const orc_ref* refs,
                                int32_t narrays, const orc_array* arrays, orc_region* out);

int orc_region_analyze(int32_t nloops, const orc_loop* loops, int32_t nrefs, const orc_ref* refs,
                       int32_t narrays, const orc_array* arrays, orc_region* out);

/* 2D 5-point Jacobi, FP64, u/v are [ny][nx] row-major (x fastest).
 * One sweep; returns max over the interior of |v - u|. */
double orc_jacobi2d_sweep(int64_t nx, int64_t ny, const double* u, double* v);
/* nsweeps ping-pong sweeps starting from u0; resid[k] = residual of sweep k.
 * Returns 0 if the final field is in u0, 1 if in u1. */
int orc_jacobi2d_run(int64_t nx, int64_t ny, double* u0, double* u1, int32_t nsweeps, double* resid);

/* 3D 7-point explicit heat step, FP64, [nz][ny][nx], Dirichlet boundary held.
 * Returns max over the interior of |v - u|. */
double orc_heat3d_sweep(int64_t nx, int64_t ny, int64_t nz, double r, const double* u, double* v);
int orc_heat3d_run(int64_t nx, int64_t ny, int64_t nz, double r, double* u0, double* u1, int32_t nsweeps,
                   double* resid);

/* 3D 27-point periodic stencil, FP32 storage and arithmetic; weights by class
 * (centre, face, edge, corner).  One sweep over every point. */
void orc_box27_sweep(int64_t nx, int64_t ny, int64_t nz, const float w[4], const float* u, float* v);
/* The same 27-point stencil in FP64 storage and arithmetic. */
void orc_box27_sweep_f64(int64_t nx, int64_t ny, int64_t nz, const double w[4], const double* u, double* v);
int orc_box27_run_f64(int64_t nx, int64_t ny, int64_t nz, const double w[4], double* u0, double* u1, int32_t nsweeps,
                      double* sums);
/* nsweeps ping-pong sweeps; if sums != NULL, sums[k] = FP64 sum of the field
 * after sweep k (k = 0..nsweeps-1).  Returns the parity of the final buffer. */
int orc_box27_run(int64_t nx, int64_t ny, int64_t nz, const float w[4], float* u0, float* u1, int32_t nsweeps,
                  double* sums);

/* Variable-coefficient 19-point Jacobi step in FP32 (the iteration of the
 * paper's Himeno workload, §5.2; written from the stencil's definition).
 * Fields are [nz][ny][nx] (x fastest); c[0..11] are the coefficient fields
 * a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 wrk1 bnd.  For each interior point, with
 * p(dx,dy,dz) the neighbour at that offset:
 *   s0 = a0 p(+x) + a1 p(+y) + a2 p(+z)
 *      + b0 (p(+x+y) - p(+x-y) - p(-x+y) + p(-x-y))
 *      + b1 (p(+y+z) - p(-y+z) - p(+y-z) + p(-y-z))
 *      + b2 (p(+x+z) - p(-x+z) - p(+x-z) + p(-x-z))
 *      + c0 p(-x) + c1 p(-y) + c2 p(-z) + wrk1
 *   ss = (s0 a3 - p) bnd,   v = p + omega ss
 * evaluated left to right in FP32; boundary points keep p.  Returns the FP64
 * sum of ss^2 (each ss^2 formed in FP64) over the interior. */
double orc_var19_sweep(int64_t nx, int64_t ny, int64_t nz, float omega, const float* const* c, const float* p,
                       float* v);
int orc_var19_run(int64_t nx, int64_t ny, int64_t nz, float omega, const float* const* c, float* u0, float* u1,
                  int32_t nsweeps, double* resid);

/* Reductions (FP64 accumulation). */
double orc_maxabs_diff(const double* a, const double* b, int64_t n);
double orc_sum_f64(const double* a, int64_t n);
double orc_sum_f32(const float* a, int64_t n);

/* MLP cost model 4 -> 64 -> 64 -> 64 -> 1, ReLU hidden layers, FP64.
 * Parameter vector layout: W1[64][4] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4[1]. */
#define ORC_MLP_NPARAM 8705
void orc_mlp_forward(const double* p, const double* x /*[n][4]*/, int64_t n, double* y /*[n]*/);
/* Mean squared error over n samples and its gradient w.r.t. every parameter. */
double orc_mlp_loss_grad(const double* p, const double* x, const double* t, int64_t n, double* grad);
/* One Adam update at step t (1-based). */
void orc_adam_step(double* p, const double* g, double* m, double* v, int64_t n, int64_t t, double lr,
                   double beta1, double beta2, double eps);

/* regret[q] = times[q][pick[q]] / min_j times[q][j] - 1 for a [nq][ntile] table. */
void orc_regret(const double* times, int32_t nq, int32_t ntile, const int32_t* pick, double* regret);

#ifdef __cplusplus
}
#endif
#endif
