/*
 * jacc.h - C ABI of the GB300 runtime-specialised affine stencil library
 * (libjacc.so).
 *
 * The library covers the data-parallel hot path that the JACC OpenACC runtime
 * (Matsumura, Garcia De Gonzalo, Pena, HiPC 2021, arXiv 2110.14340) speeds up:
 * runtime analysis of the array regions an affine loop nest touches, kernels
 * specialised with runtime values and cached, and iterative stencil sweeps
 * with a fused convergence reduction, run as CUDA-graph-captured loops.  Two
 * additions have no counterpart in the paper: batched persistent launches over
 * many uneven grids, and an autotuner plus a small learned cost model that
 * picks tile configurations.
 *
 * Conventions for every entry point:
 *  - Returns a jacc_status; JACC_OK is 0 and every error is negative.  The
 *    library never aborts or exits.  jacc_last_error() gives a message for the
 *    last failing call on the calling thread.
 *  - Device pointers are caller-owned CUDA device memory (for instance torch
 *    tensors); the library never frees them.  Host pointers are read during
 *    the call only, unless stated.
 *  - `stream` is a cudaStream_t passed as uintptr_t (0 = legacy default stream).
 *    Device work is enqueued asynchronously on it unless stated.
 *  - Arrays are row-major with x the fastest axis: a 2D grid is [ny][nx], a 3D
 *    grid [nz][ny][nx].
 */
#ifndef JACC_H
#define JACC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef int32_t jacc_status;
#define JACC_OK 0
#define JACC_ERR_INVALID_ARG (-1)   /* bad pointer, size, enum, aliasing */
#define JACC_ERR_OUT_OF_BOUNDS (-2) /* a touched region leaves the array  */
#define JACC_ERR_OVERFLOW (-3)      /* int64 overflow in index arithmetic */
#define JACC_ERR_CUDA (-4)          /* a CUDA runtime call failed         */
#define JACC_ERR_COMPILE (-5)       /* NVRTC or module load failed        */
#define JACC_ERR_TIMEOUT (-6)       /* a bounded device wait gave up      */
#define JACC_ERR_UNSUPPORTED (-7)   /* valid request the library lacks    */
#define JACC_ERR_NOMEM (-8)         /* host or device allocation failed   */

/* Message for the last non-OK status returned on this thread ("" if none).
 * The pointer stays valid until the next jacc call on the same thread. */
const char* jacc_last_error(void);
/* Library version string, e.g. "jacc-gb300 1.0 (sm_103a)". */
const char* jacc_version(void);

/* ---------------------------------------------------------- region analysis
 * The runtime tracks which index ranges of each array a kernel reads and
 * writes (data ranges linked to pointers, paper §3.2.1; per-array lower/upper
 * write bounds, §4.1).  References to one array are merged to the widest range
 * (§4.1); reads and writes are kept separate (§4.1, aliasing rule).
 *
 * A nest is rectangular: loop k runs i_k = lo, lo+step, ... while i_k <= hi
 * (step > 0) or while i_k >= hi (step < 0); step == 0 is JACC_ERR_INVALID_ARG.
 * nloops == 0 means a single iteration.  A reference's subscript d is the
 * affine form off[d] + sum_k coef[d][k] * i_k.  For every array the result
 * holds the per-dimension index hulls [lo, hi] of the reads and of the writes
 * and the exact min/max of the flattened row-major element offset
 * (stride[ndim-1] = 1, stride[d] = stride[d+1] * extent[d+1]).  Hulls are
 * exact: each bound is attained by some iteration.  An empty nest (some loop
 * with no iteration) touches nothing (has_read = has_write = 0).
 *
 * Errors: JACC_ERR_INVALID_ARG for NULL arrays with a non-zero count, a count
 * outside [0, JACC_MAX_*], ndim outside [1, JACC_MAX_DIMS], a negative extent,
 * an array_id out of range or a reference whose ndim differs from its
 * array's; JACC_ERR_OVERFLOW when a coefficient times a loop endpoint, a
 * stride, a flattened coefficient or offset, or a final bound leaves int64
 * (`out` is then unspecified); JACC_ERR_OUT_OF_BOUNDS when some hull leaves
 * [0, extent-1] (`out` is still fully written).  Pure host code, reentrant,
 * no CUDA call. */
#define JACC_MAX_DIMS 8
#define JACC_MAX_LOOPS 8

typedef struct { int64_t lo, hi, step; } jacc_loop;

typedef struct {
  int32_t array_id;                          /* index into the arrays[] argument */
  int32_t ndim;                              /* must equal arrays[array_id].ndim */
  int32_t is_write;                          /* 0 = read, non-zero = write       */
  int32_t reserved;                          /* set to 0                         */
  int64_t coef[JACC_MAX_DIMS][JACC_MAX_LOOPS]; /* coef[d][k]                     */
  int64_t off[JACC_MAX_DIMS];
} jacc_ref;

typedef struct {
  int32_t ndim;
  int32_t reserved;
  int64_t extent[JACC_MAX_DIMS];
} jacc_array;

typedef struct {
  int32_t has_read, has_write;
  int64_t rlo[JACC_MAX_DIMS], rhi[JACC_MAX_DIMS]; /* read hull per dimension  */
  int64_t wlo[JACC_MAX_DIMS], whi[JACC_MAX_DIMS]; /* write hull per dimension */
  int64_t rlin_lo, rlin_hi, wlin_lo, wlin_hi;     /* flattened offset extremes */
} jacc_region;

jacc_status jacc_region_analyze(int32_t nloops, const jacc_loop* loops, int32_t nrefs, const jacc_ref* refs,
                                int32_t narrays, const jacc_array* arrays, jacc_region* out /* [narrays] */);

/* Triangular (affine-bounded) nests.  Loop k runs i_k = lo_k, lo_k + 1, ...,
 * hi_k with lo_k = lo + sum_{m<k} lo_coef[m] i_m and hi_k likewise, so inner
 * bounds may follow outer indices (j = i .. n-1, k = 0 .. i + j, ...);
 * lo_coef[m] and hi_coef[m] must be 0 for m >= k.  The result is that of
 * jacc_region_analyze (exact hulls and flattened-offset extremes over the
 * iterations that run), computed by eliminating the loops from the innermost
 * out: the extreme of c i_k over [lo_k, hi_k] is c hi_k or c lo_k, an affine
 * form in the outer indices (the paper's analysis covers rectangular ranges,
 * §4.1; this extends it to the nests its future work names).  An empty
 * outermost loop touches nothing.  An inner loop that is empty for some
 * iterations of its outer loops, its extent following one outer index whose
 * own bounds are constant (j = i .. 5 over i = 0 .. 9), first tightens that
 * index's bounds to the iterations in which it runs (exact: the body runs
 * nowhere else); JACC_ERR_UNSUPPORTED if the emptiness couples several
 * indices or an index with affine bounds.  Other errors as for
 * jacc_region_analyze, plus JACC_ERR_OVERFLOW when an eliminated form leaves
 * int64. */
typedef struct {
  int64_t lo, hi;
  int64_t lo_coef[JACC_MAX_LOOPS];
  int64_t hi_coef[JACC_MAX_LOOPS];
} jacc_loop_affine;
jacc_status jacc_region_analyze_affine(int32_t nloops, const jacc_loop_affine* loops, int32_t nrefs,
                                       const jacc_ref* refs, int32_t narrays, const jacc_array* arrays,
                                       jacc_region* out /* [narrays] */);

/* Touched sets as a union of boxes (rectangular nests).  Each reference
 * contributes the box of its per-dimension hull; boxes of the same array and
 * access kind that lie inside another are dropped, duplicates kept once.
 * exact = 1 when the reference's touched set is its whole box: every
 * subscript depends on at most one loop, with coefficient +-1 and a loop step
 * of +-1, and no two dimensions depend on the same loop.  When every box of
 * an array and kind is exact their union is the exact touched set (a 5-point
 * read set is a cross, not its hull).  At most max_boxes are written; *nboxes
 * is the number the union has (JACC_ERR_INVALID_ARG if it exceeds max_boxes,
 * the first max_boxes being written).  Errors otherwise as for
 * jacc_region_analyze. */
typedef struct {
  int32_t array_id;
  int32_t is_write;
  int32_t exact;
  int32_t reserved;
  int64_t lo[JACC_MAX_DIMS], hi[JACC_MAX_DIMS];
} jacc_box;
jacc_status jacc_region_boxes(int32_t nloops, const jacc_loop* loops, int32_t nrefs, const jacc_ref* refs,
                              int32_t narrays, const jacc_array* arrays, jacc_box* boxes, int32_t max_boxes,
                              int32_t* nboxes);
/* jacc_region_boxes for an affine nest (jacc_loop_affine, step 1; inner loops
 * that run empty for some outer iterations first tighten their outer index
 * as in jacc_region_analyze_affine).  Each reference contributes the box of
 * its exact per-dimension extremes over the iterations that run; exact = 1
 * when every subscript follows at most one loop with coefficient +-1, no two
 * subscripts the same loop, and those loops have constant bounds (a
 * reference A[i][j] over the triangle j = 0 .. i is not its box; A[i] is).
 * Errors as for jacc_region_boxes and jacc_region_analyze_affine. */
jacc_status jacc_region_boxes_affine(int32_t nloops, const jacc_loop_affine* loops, int32_t nrefs,
                                     const jacc_ref* refs, int32_t narrays, const jacc_array* arrays, jacc_box* boxes,
                                     int32_t max_boxes, int32_t* nboxes);

/* ---------------------------------------------------------- specialisation
 * A kernel descriptor names one stencil sweep.  jacc_specialize returns a
 * handle to a compiled kernel plus its launch configuration, from a cache
 * keyed on the full descriptor (paper §3.1: code compiled once is reused;
 * §3.2.2: runtime-invariant parameters are substituted by constants and
 * non-aliasing pointers are declared restrict).
 *
 * Stencils (interior points; Dirichlet boundary points are copied unchanged):
 *   JACC_STENCIL_5PT  (2D): v = ((u[y-1][x] + u[y+1][x]) + (u[y][x-1] + u[y][x+1])) / 4
 *   JACC_STENCIL_7PT  (3D): v = u + r * (sum of the 6 face neighbours - 6 u),  r = coeffs[0]
 *   JACC_STENCIL_27PT (3D): v = w0*centre + wf*faces + we*edges + wc*corners,
 *                           (w0, wf, we, wc) = coeffs[0..3]
 *   JACC_STENCIL_19PT (3D, FP32, variable coefficients; swept with
 *                 jacc_sweep_coeffs): the Jacobi step of the paper's Himeno
 *                 workload (§5.2), coeffs[0] = omega, twelve coefficient
 *                 fields a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 wrk1 bnd:
 *       s0 = a0 u(+x) + a1 u(+y) + a2 u(+z)
 *          + b0 (u(+x+y) - u(+x-y) - u(-x+y) + u(-x-y))
 *          + b1 (u(+y+z) - u(-y+z) - u(+y-z) + u(-y-z))
 *          + b2 (u(+x+z) - u(-x+z) - u(+x-z) + u(-x-z))
 *          + c0 u(-x) + c1 u(-y) + c2 u(-z) + wrk1
 *       ss = (s0 a3 - u) bnd,   v = u + omega ss
 *     (u(+x-y) is the neighbour at x+1, y-1, and so on).
 * Fused reduction written per sweep into resid_dev[k] (FP64):
 *   5PT and 7PT : max over interior points of |v - u| (the change made by
 *                 the sweep);
 *   27PT        : the sum of the output field (every materialised sweep);
 *   19PT        : the sum over interior points of ss^2.
 *
 * dtype JACC_F64 stores FP64.  Its arithmetic (arith):
 *   JACC_ARITH_AUTO    exact 64-bit fixed-point integer arithmetic when the
 *                      stencil is a convex combination (5PT always; 7PT with
 *                      0 < r <= 1/6; 27PT with non-negative weights summing to
 *                      at most 1 + 2^-20) and the input is finite; native
 *                      FP64 otherwise.  Results are the exact stencil value
 *                      rounded once to FP64.
 *   JACC_ARITH_NATIVE  FP64 instructions throughout.
 * dtype JACC_F32 stores and computes FP32 (arith is ignored).
 *
 * tile_id selects one of JACC_NUM_TILES tile configurations (see
 * jacc_tile_info), or -1 to let the library choose (the autotuner's cached
 * pick for this shape if one exists, else a default).
 *
 * flags: JACC_SPEC_JIT compiles a variant with the extents and coefficients
 * folded in as constants (NVRTC, sm_103a; cached in memory and, if the
 * environment variable JACC_CACHE_DIR names a directory, on disk); for the
 * 3D tiles with 16-byte columns and the long march it marches 40 planes per
 * CTA (27PT: 32) instead of the table's 64 (jacc_kernel_info reports the
 * grid).
 * Without it the handle uses a precompiled kernel that takes them as
 * arguments.
 * JACC_SPEC_CLUSTER (5PT FP64 only; no counterpart in the paper): jacc_sweep
 * runs the whole sequence in one launch of one thread-block cluster (16 or 8
 * CTAs) that keeps both fields in its distributed shared memory; it suits
 * grids of up to about 10^5 points, whose sweeps are otherwise bound by
 * launch latency.  Fields, residuals and the other buffer are bit-identical
 * to the launch-per-sweep sequence; jacc_launch still runs the tile kernel.
 * JACC_ERR_UNSUPPORTED if the grid does not fit a cluster the device can run.
 *
 * tblock (27PT FP32 only, nx a multiple of 4, T <= 3): temporal-blocking
 * depth T >= 1.  Each launch then performs T sweeps and reads and writes
 * the field once (8/T bytes per point-sweep); jacc_sweep accounts for this.
 * T = 2 runs a staged two-sweep kernel whose fields are bit-identical to two
 * single sweeps of the staged 16-byte-vector tiles; T = 3 a register-based
 * kernel (equal within FP32 rounding).  UNSUPPORTED otherwise.
 *
 * The handle is owned by the library and stays valid until jacc_release or
 * jacc_shutdown.  Identical descriptors share one compiled kernel. */
#define JACC_STENCIL_5PT 5
#define JACC_STENCIL_7PT 7
#define JACC_STENCIL_27PT 27
#define JACC_STENCIL_19PT 19
#define JACC_F32 32
#define JACC_F64 64
#define JACC_DIRICHLET 0
#define JACC_PERIODIC 1
#define JACC_ARITH_AUTO 0
#define JACC_ARITH_NATIVE 1
#define JACC_SPEC_JIT 1u
#define JACC_SPEC_CLUSTER 2u
#define JACC_NUM_TILES 24

typedef struct {
  int32_t stencil;   /* JACC_STENCIL_*                                 */
  int32_t dtype;     /* JACC_F32 or JACC_F64                           */
  int32_t boundary;  /* JACC_DIRICHLET (5PT, 7PT) or JACC_PERIODIC (27PT) */
  int32_t tile_id;   /* 0..JACC_NUM_TILES-1, or -1                     */
  int64_t nx, ny, nz;/* extents; nz = 1 for 5PT; each >= 3             */
  double coeffs[4];  /* see above                                      */
  int32_t arith;     /* JACC_ARITH_*                                   */
  uint32_t flags;    /* JACC_SPEC_*                                    */
  int32_t tblock;    /* 27PT temporal-blocking depth (0 or 1 = none)   */
  int32_t reserved;  /* set to 0                                       */
} jacc_kernel_desc;

typedef struct jacc_kernel_s* jacc_kernel;

typedef struct {
  int32_t tile_id;
  int32_t jit;          /* 1 if constants are folded (NVRTC variant)     */
  int32_t fixed_point;  /* 1 if FP64 arithmetic runs in 64-bit fixed point */
  int32_t tblock;
  int32_t block[3];     /* CUDA block shape                               */
  int32_t grid[3];      /* CUDA grid shape                                */
  double compile_ms;    /* NVRTC + load time of this variant (0 if cached) */
} jacc_kernel_info_t;

jacc_status jacc_specialize(const jacc_kernel_desc* desc, jacc_kernel* out);
jacc_status jacc_kernel_info(jacc_kernel k, jacc_kernel_info_t* out);
jacc_status jacc_release(jacc_kernel k);

/* Device status of a handle's launches (no counterpart in the paper).  The
 * 27PT FP32 kernels with 16-byte columns stage their input planes in shared
 * memory with bulk copies and wait for them on mbarriers; each such wait is
 * bounded (default 2 s).  A wait that runs out writes JACC_ERR_TIMEOUT to the
 * handle's device status word and its CTA returns early, so the output of
 * that launch is incomplete.  jacc_kernel_status synchronises the device,
 * stores the word (JACC_OK or JACC_ERR_TIMEOUT) in *status and clears it.
 * jacc_kernel_set_wait sets the limit of each wait (timeout_ms > 0, or 0 for
 * the default) and a test hook: stall_plane >= 0 makes CTA (0,0,0) of later
 * launches never request that staged plane, so its waits run out
 * (-1 = off).  It applies to the handle (shared by identical descriptors)
 * and drops its cached graphs. */
jacc_status jacc_kernel_status(jacc_kernel k, int32_t* status);
jacc_status jacc_kernel_set_wait(jacc_kernel k, int32_t timeout_ms, int32_t stall_plane);

/* Tile configuration `tile_id`: threads (bx, by) per CTA, elements per thread
 * in x (vec: 1 or a 16-byte vector), and the march length zc (planes per CTA
 * in 3D, rows per thread in 2D).  Host only. */
typedef struct { int32_t bx, by, vec16, zc; } jacc_tile;
jacc_status jacc_tile_info(int32_t tile_id, jacc_tile* out);

/* ------------------------------------------------------------------ launch
 * jacc_launch: one sweep from u_in to u_out (each nx*ny*nz elements of the
 * descriptor's dtype, 16-byte aligned).  u_in and u_out must not overlap
 * (they are restrict in the kernel): overlap is JACC_ERR_INVALID_ARG.
 * resid_dev (nullable) receives the sweep's reduction (one double, device
 * memory).  For 27PT with tblock T > 1 one launch performs T sweeps.
 * Asynchronous on `stream`. */
jacc_status jacc_launch(jacc_kernel k, const void* u_in, void* u_out, double* resid_dev, uintptr_t stream);

/* jacc_sweep: nsweeps ping-pong sweeps u0 -> u1 -> u0 ... (nsweeps >= 1; for
 * 27PT a multiple of tblock).  resid_dev (nullable, device, nsweeps doubles)
 * receives resid_dev[k] for sweep k; for 27PT with temporal blocking only
 * sweeps that end a block are materialised and the others get NaN.
 * flags: JACC_SWEEP_GRAPH captures the whole loop as one CUDA graph, cached
 * by (kernel, u0, u1, nsweeps, resid_dev) and replayed on later calls; the
 * graph is dropped by jacc_release.  Without it the launches are issued one
 * by one.  *final_buf (host) is set to 0 if the last sweep wrote u0, 1 if u1.
 * FP64 kernels on the fixed-point path keep the field in 64-bit fixed point
 * between the sweeps of one call (same 8 bytes per value, in u0/u1): the
 * first sweep reads FP64, the last writes FP64, each intermediate sweep rounds
 * once to the fixed-point grid (2^-F with F >= 57 - e(max|u0|), finer than an
 * FP64 ulp of max|u0|).  For fields of at least 2^22 points and nsweeps >= 2
 * the conversion of u0 runs as its own kernel, in place, before the first
 * sweep (u0 is overwritten by the second sweep in any case); the values are
 * those the first sweep would convert on load.  Dirichlet boundary values pass through the same grid:
 * they come back unchanged when they are multiples of 2^-F (for instance any
 * value within 2^52 ulps of max|u0|) and otherwise within 2^-F.  After the
 * call the result buffer holds FP64; the other buffer holds the internal
 * representation.  Asynchronous on `stream`. */
#define JACC_SWEEP_GRAPH 1u
jacc_status jacc_sweep(jacc_kernel k, void* u0, void* u1, int32_t nsweeps, double* resid_dev, uint32_t flags,
                       uintptr_t stream, int32_t* final_buf);

/* jacc_sweep_host: jacc_sweep from and to host memory in one call (the
 * whole-job path of a caller whose fields live on the host).  Enqueues on
 * `stream`, in order: a copy of the input field u_host (host, nx*ny*nz values
 * of the kernel's dtype) into u0, jacc_sweep(k, u0, u1, nsweeps, resid_dev,
 * flags, stream), a copy of the result field into result_host (host, same
 * size) and, if resid_host is non-NULL, of the nsweeps residuals from
 * resid_dev (then required) into resid_host.  u0, u1 and resid_dev are the
 * caller's device buffers with jacc_sweep's rules; the library allocates
 * nothing here.  Host buffers are caller-owned and must stay valid until the
 * stream reaches the copies; with page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) the copies are asynchronous, so calls on two streams with
 * two sets of device buffers overlap each call's copies with the other's
 * sweeps; pageable memory is correct but copies synchronously.  wait_event
 * and done_event (cudaEvent_t as an integer, each 0 for none): the sweeps
 * wait for wait_event (after the input copy is enqueued), and done_event is
 * recorded after the sweeps (before the copy back), so that consecutive
 * calls on two streams can keep their sweeps in order while their copies
 * overlap (pass the previous call's done_event as wait_event).  *final_buf
 * (host, nullable) as jacc_sweep.  Errors: INVALID_ARG for NULL host buffers,
 * resid_host without resid_dev and every jacc_sweep argument error; CUDA for
 * a failed copy.  The paper's runtime copies data to and from the device
 * around its kernels (§3.2.1, data-region tracking); this is that transfer
 * for one sweep sequence. */
jacc_status jacc_sweep_host(jacc_kernel k, const void* u_host, void* result_host, void* u0, void* u1,
                            int32_t nsweeps, double* resid_dev, double* resid_host, uint32_t flags,
                            uintptr_t stream, uintptr_t wait_event, uintptr_t done_event, int32_t* final_buf);

/* jacc_sweep_coeffs: nsweeps ping-pong sweeps of a JACC_STENCIL_19PT kernel,
 * as jacc_sweep (resid_dev, flags, stream and final_buf alike), with its
 * twelve coefficient fields: fields[0..11] = a0 a1 a2 a3 b0 b1 b2 c0 c1 c2
 * wrk1 bnd, each nx*ny*nz FP32 values in device memory, 16-byte aligned,
 * caller-owned, read-only during the call and not overlapping u0 or u1
 * (nfields must be 12).  Graphs (JACC_SWEEP_GRAPH) are cached by every
 * pointer of the call.  The 19-point kernel has one tile (32 x 4 threads,
 * 16-byte columns, input planes staged by bulk copies, 40-plane march); nx
 * must be a multiple of 4.  jacc_launch and jacc_sweep reject 19PT handles. */
jacc_status jacc_sweep_coeffs(jacc_kernel k, void* u0, void* u1, int32_t nsweeps, const void* const* fields,
                              int32_t nfields, double* resid_dev, uint32_t flags, uintptr_t stream,
                              int32_t* final_buf);

/* jacc_sweep_until (no counterpart in the paper, which runs a fixed iteration
 * count; §5.2 notes that Himeno reduces its error each iteration): sweeps
 * u0 -> u1 -> u0 ... until a sweep's residual is <= tol or max_sweeps sweeps
 * ran, with the loop and its exit test on the device: one CUDA graph (cached
 * per kernel, fields, max_sweeps, tol and output arrays, dropped by
 * jacc_release) whose WHILE conditional node runs the sweeps, each followed by
 * a one-thread kernel that stores the residual and sets the loop condition;
 * the host never waits.  5PT and 7PT only (their residual is max |v - u|);
 * 27PT is JACC_ERR_UNSUPPORTED.  tol finite and >= 0, max_sweeps >= 1.
 *   resid_dev  (device, max_sweeps doubles, required): resid_dev[i] for each
 *              sweep i that ran; later slots are untouched.
 *   status_dev (device, 2 int32, required): [0] sweeps run n, [1] the buffer
 *              holding the result (0: u0, 1: u1), written when the loop ends.
 * Fields, residuals and the other buffer are bit-identical to
 * jacc_sweep(k, u0, u1, n, ...): for FP64 fixed-point kernels the loop keeps
 * the resident form and the last sweep is run once more from the state before
 * it with FP64 output (so the result is the exact stencil value rounded once).
 * Asynchronous on `stream`. */
jacc_status jacc_sweep_until(jacc_kernel k, void* u0, void* u1, int32_t max_sweeps, double tol, double* resid_dev,
                             int32_t* status_dev, uintptr_t stream);

/* ------------------------------------------- region-driven async scheduler
 * The runtime's asynchronous execution (§3.2.1 tracks the data range each
 * kernel touches; §4 runs kernels without host synchronisation; §6.1 uses 16
 * queues): a scheduler owns a pool of nstreams CUDA streams (1..64) and runs
 * each submitted task on one of them after cudaStreamWaitEvent on, for every
 * byte the task touches, the last earlier task that wrote it and, for bytes
 * it writes, the earlier tasks that read them since that write (read after
 * write, write after read, write after write); every other earlier task with
 * overlapping ranges is ordered before one of those, and tasks without a
 * conflict run concurrently.  The ranges are kept in an interval map, so a
 * submission costs O(log n) plus the segments it overlaps.  A task that depends on the last task of a
 * stream continues that stream; others take the next stream round-robin.
 * The pool starts after the work queued on `origin` when it is created;
 * jacc_sched_join makes a stream wait for every task.  Tasks completed on the
 * device are retired and wait for nothing.  Not thread-safe across
 * schedulers sharing fields.
 * JACC_SCHED_DRY_RUN: no CUDA call at all; tasks only record their
 * dependencies and stream (jacc_sched_task_info), for checking the
 * dependency logic on a host.  Task ids count from 0 in submission order. */
#define JACC_SCHED_DRY_RUN 1u
typedef struct jacc_sched_s* jacc_sched;
jacc_status jacc_sched_create(int32_t nstreams, uint32_t flags, uintptr_t origin, jacc_sched* out);
/* A jacc_sweep sequence (graph-launched) as a task: it reads u0 and writes
 * u1 (nsweeps = 1) or reads and writes both, and writes resid_dev. */
jacc_status jacc_sched_sweep(jacc_sched s, jacc_kernel k, void* u0, void* u1, int32_t nsweeps, double* resid_dev,
                             int32_t* task_id);
/* A device-to-device copy of `bytes` bytes as a task (no overlap). */
jacc_status jacc_sched_copy(jacc_sched s, void* dst, const void* src, uint64_t bytes, int32_t* task_id);
/* A task for the caller's own device work, described by its loop nest:
 * jacc_region_analyze(nloops, loops, nrefs, refs, narrays, arrays) gives each
 * array's read and written flattened-offset extremes, mapped to bytes through
 * base[a] (device address of array a's element 0) and elem_bytes[a].  The
 * caller enqueues the work on *stream_out, then calls jacc_sched_nest_end;
 * errors of the analysis are returned unchanged. */
jacc_status jacc_sched_nest_begin(jacc_sched s, int32_t nloops, const jacc_loop* loops, int32_t nrefs,
                                  const jacc_ref* refs, int32_t narrays, const jacc_array* arrays,
                                  const uint64_t* base, const int32_t* elem_bytes, int32_t* task_id,
                                  uintptr_t* stream_out);
/* The same for an affine (triangular) nest: its ranges come from
 * jacc_region_analyze_affine, exact over the iterations that run, so a nest
 * such as j = 0 .. i touches (and waits for) no more than its triangle. */
jacc_status jacc_sched_nest_begin_affine(jacc_sched s, int32_t nloops, const jacc_loop_affine* loops, int32_t nrefs,
                                         const jacc_ref* refs, int32_t narrays, const jacc_array* arrays,
                                         const uint64_t* base, const int32_t* elem_bytes, int32_t* task_id,
                                         uintptr_t* stream_out);
jacc_status jacc_sched_nest_end(jacc_sched s, int32_t task_id);
/* The tasks task_id waited for (first max_deps of *ndeps, in id order) and
 * the index of its pool stream.  In live mode such a task that had already
 * completed on the device when task_id was submitted is not listed (it needed
 * no wait); dry-run mode lists all of them. */
jacc_status jacc_sched_task_info(jacc_sched s, int32_t task_id, int32_t* deps, int32_t max_deps, int32_t* ndeps,
                                 int32_t* stream_index);
jacc_status jacc_sched_join(jacc_sched s, uintptr_t stream);
/* Resource count for long runs: first retires every task that has completed
 * on the device and is neither its stream's last task nor an open nest, then
 * reports in *live_events how many tasks still hold a completion event (at
 * most the stream count plus the open nests plus the tasks still running)
 * and, if ntasks is not NULL, how many tasks were submitted.  Dry-run
 * schedulers hold no events (0). */
jacc_status jacc_sched_live_events(jacc_sched s, int64_t* live_events, int64_t* ntasks);
/* Waits for the pool's streams, then frees the scheduler. */
jacc_status jacc_sched_release(jacc_sched s);

/* ---------------------------------------------------------- autotuner
 * Exhaustive search over the JACC_NUM_TILES tile configurations for one
 * descriptor (the paper names auto-tuning as future work, §8, and cites
 * OptACC's grid search over OpenACC parallelism, §7).  Each valid tile is
 * specialised and runs a graph-captured sequence of `sweeps_per_rep` sweeps
 * on the caller's fields u0/u1 (their contents change) once to warm up and
 * `reps` more times, timed with CUDA events on `stream`; out->ms[t] is the
 * median time per sweep (infinity and valid[t] = 0 for tiles that do not fit
 * the shape).  The fastest tile is remembered for the shape, so that
 * jacc_specialize with tile_id = -1 uses it.  Synchronises `stream`. */
typedef struct {
  double ms[JACC_NUM_TILES];    /* median milliseconds per sweep              */
  int32_t valid[JACC_NUM_TILES];
  int32_t best_tile;
  int32_t reserved;
  double best_ms;
} jacc_tune_result;

jacc_status jacc_autotune(const jacc_kernel_desc* desc, void* u0, void* u1, int32_t sweeps_per_rep, int32_t reps,
                          uintptr_t stream, jacc_tune_result* out);
/* jacc_autotune restricted to the ntiles tile ids in `tiles` (host array,
 * each in [0, JACC_NUM_TILES)): only those are timed (out->valid[t] = 1 for
 * the timed tiles that fit the shape, 0 for all others), and the fastest of
 * them is remembered for the shape.  INVALID_ARG for an empty list or an id
 * out of range, UNSUPPORTED if none of them fits. */
jacc_status jacc_autotune_tiles(const jacc_kernel_desc* desc, void* u0, void* u1, int32_t sweeps_per_rep,
                                int32_t reps, uintptr_t stream, const int32_t* tiles, int32_t ntiles,
                                jacc_tune_result* out);
/* Forget every remembered autotuner pick. */
jacc_status jacc_autotune_forget(void);

/* ---------------------------------------------------------- learned cost model
 * An MLP 4 -> 64 -> 64 -> 64 -> 1 (ReLU, FP32, 8705 parameters, layout
 * W1[64][4] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4) that maps
 * the features of (stencil, side, dtype, tile) to the natural log of the sweep
 * time in microseconds.  No counterpart in the paper.  Features
 * (jacc_costmodel_features): [points / 27, log2(side) / 10, dtype bits / 64,
 * tile / 23], side = the grid side (square root of the area for 2D, cube
 * root of the volume for 3D).
 *
 * create      : parameters from `init_params` (host, 8705 floats) or, if
 *               NULL, Kaiming-uniform from `seed`; Adam state zeroed.
 * loss_grad   : mean squared error over n samples (x_dev [n][4], y_dev [n],
 *               device FP32) into *loss_dev and its gradient into grad_dev
 *               (8705 floats); no update.
 * train       : `epochs` full-batch Adam steps (beta1 0.9, beta2 0.999,
 *               eps 1e-8, bias-corrected) with learning rate lr, run as CUDA
 *               graphs on `stream`; *loss_dev (nullable) = loss before the
 *               last step.
 * predict     : y_dev[i] = network(x_dev[i]).
 * pick        : nq queries of JACC_NUM_TILES feature rows each (feats_dev
 *               [nq][24][4], valid_dev [nq][24]); pred_dev [nq][24] receives
 *               the predictions, pick_dev[q] the valid argmin (ties to the
 *               lowest tile, -1 if none) and gap_dev[q] the second-best
 *               minus the best prediction.
 * set_range   : the side range the model was trained on and the decision
 *               margin (in log-microseconds).
 * choose      : the model's tile for `desc`; falls back to jacc_autotune on
 *               u0/u1 (needed then) when the side lies outside the range or
 *               the top-2 gap is below the margin.  *used_fallback tells
 *               which.  The chosen tile is remembered for the shape.
 * choose_topk : the model as a filter: the k valid tiles with the lowest
 *               predicted time for `desc` are timed on u0/u1 (required; their
 *               contents change) by jacc_autotune_tiles and the fastest is
 *               returned and remembered for the shape.  k >= the number of
 *               valid tiles is the exhaustive search.
 * save / load : parameters and range in a small binary file ("JACCMLP1"). */
typedef struct jacc_costmodel_s* jacc_costmodel;

jacc_status jacc_costmodel_features(int32_t stencil, double side, int32_t dtype, int32_t tile, float* out4);
jacc_status jacc_costmodel_create(const float* init_params, uint64_t seed, jacc_costmodel* out);
jacc_status jacc_costmodel_set_params(jacc_costmodel m, const float* host_params);
jacc_status jacc_costmodel_get_params(jacc_costmodel m, float* host_params);
jacc_status jacc_costmodel_loss_grad(jacc_costmodel m, const float* x_dev, const float* y_dev, int32_t n, float* grad_dev,
                                     float* loss_dev, uintptr_t stream);
jacc_status jacc_costmodel_train(jacc_costmodel m, const float* x_dev, const float* y_dev, int32_t n, int32_t epochs,
                                 float lr, uintptr_t stream, float* loss_dev);
jacc_status jacc_costmodel_predict(jacc_costmodel m, const float* x_dev, int32_t n, float* y_dev, uintptr_t stream);
jacc_status jacc_costmodel_pick(jacc_costmodel m, const float* feats_dev, const int32_t* valid_dev, int32_t nq,
                                float* pred_dev, int32_t* pick_dev, float* gap_dev, uintptr_t stream);
jacc_status jacc_costmodel_set_range(jacc_costmodel m, double side_lo, double side_hi, double margin);
jacc_status jacc_costmodel_choose(jacc_costmodel m, const jacc_kernel_desc* desc, void* u0, void* u1, uintptr_t stream,
                                  int32_t* tile, int32_t* used_fallback);
jacc_status jacc_costmodel_choose_topk(jacc_costmodel m, const jacc_kernel_desc* desc, void* u0, void* u1,
                                       uintptr_t stream, int32_t k, int32_t* tile);
/* ---- the model's data pipeline, from raw autotuner tables (host memory).
 * One jacc_tune_table row is one query (stencil, dtype, side) with the
 * per-tile times jacc_autotune reported for it (ms, valid as in
 * jacc_tune_result).
 * fit_tables  : training set = every valid (query, tile): features as
 *               jacc_costmodel_features, target = ln(1000 ms) minus the mean
 *               of that over the query's valid tiles (the argmin over tiles
 *               does not depend on a per-query constant, and centring keeps
 *               the loss on the differences between tiles); then `epochs`
 *               full-batch Adam steps at lr (jacc_costmodel_train).
 *               *final_mse (nullable) = the loss before the last step.
 *               Synchronous; allocates the training arrays on the device.
 * evaluate    : per query: the model's pick (valid argmin of its
 *               predictions, ties to the lowest tile; -1 if no tile is
 *               valid), the top-2 predicted gap, regret = ms[pick] / min
 *               over valid tiles of ms - 1, fallback = (gap < margin), and
 *               for the model used as a filter (k = topk best-ranked valid
 *               tiles timed, the fastest kept) its regret and the summed ms
 *               of those k tiles.  Synchronous.
 * fixed_tile  : the method without the model: the one tile valid for every
 *               query with the lowest mean ln(ms) over the tables (host
 *               only; UNSUPPORTED if no tile is valid everywhere).
 * margin      : the decision margin at which the model falls back on at
 *               most `fraction` of these queries: the largest gap g such
 *               that fewer than fraction x nq queries have gap < g (0 for
 *               fraction 0). */
typedef struct {
  int32_t stencil;               /* 5, 7 or 27                                */
  int32_t dtype;                 /* 32 or 64                                  */
  double side;                   /* grid side (> 0)                           */
  double ms[JACC_NUM_TILES];     /* time per sweep of each tile               */
  int32_t valid[JACC_NUM_TILES]; /* 1 where the tile fits and was timed       */
} jacc_tune_table;

typedef struct {
  int32_t pick;          /* the model's tile, or -1                          */
  int32_t fallback;      /* 1 if gap < margin                                */
  double gap;            /* second-best minus best prediction (ln us)        */
  double regret;         /* ms[pick] / best ms - 1                           */
  double regret_topk;    /* regret of the fastest of the top-k ranked tiles  */
  double search_ms_topk; /* sum of ms over those k tiles                      */
} jacc_costmodel_eval;

jacc_status jacc_costmodel_fit_tables(jacc_costmodel m, int32_t nq, const jacc_tune_table* tables, int32_t epochs,
                                      float lr, uintptr_t stream, double* final_mse);
jacc_status jacc_costmodel_evaluate(jacc_costmodel m, int32_t nq, const jacc_tune_table* tables, double margin,
                                    int32_t topk, uintptr_t stream, jacc_costmodel_eval* out);
jacc_status jacc_costmodel_fixed_tile(int32_t nq, const jacc_tune_table* tables, int32_t* tile);
/* regret[q] = ms[picks[q]] / min over valid tiles of ms - 1 (host only);
 * INVALID_ARG if a pick is out of range or not valid for its query. */
jacc_status jacc_costmodel_regret(int32_t nq, const jacc_tune_table* tables, const int32_t* picks, double* regret);
jacc_status jacc_costmodel_margin(jacc_costmodel m, int32_t nq, const jacc_tune_table* tables, double fraction,
                                  uintptr_t stream, double* margin);
jacc_status jacc_costmodel_save(jacc_costmodel m, const char* path);
jacc_status jacc_costmodel_load(jacc_costmodel m, const char* path);
jacc_status jacc_costmodel_release(jacc_costmodel m);

/* ---------------------------------------------------------- batched sweeps
 * Many independent 2D 5-point Jacobi grids (FP64, Dirichlet boundary held)
 * swept together in one persistent, cooperative launch.  No counterpart in
 * the paper, which overlaps independent kernels on OpenACC queues (§6.1).
 * Every sweep of every grid runs inside that launch.  Each grid is cut into
 * items (tiles of rows x cols points, cols = 64 x the tile's warps across);
 * grids are packed into groups whose two fields fit an L2 budget together;
 * work is a sequence of tickets (sweep, item), group after group and
 * sweep-major within a group, so a group's fields stay in L2 across its
 * sweeps.  An item waits, bounded by a time limit, only until the items
 * whose rows or columns it reads (the tiles above, below, left and right,
 * and itself) have finished the previous sweep.  Arithmetic is the 5-point
 * stencil's (exact fixed point for finite inputs, see jacc_specialize);
 * every schedule gives the same bits.
 *
 * Schedule (jacc_batch_config): target points per item (tile columns: the
 * fewest 64-column strips that cover a row, at most 2 for the staged march
 * and 8 for the register march; rows = max(warps per strip, item_points /
 * columns)), persistent CTAs per SM (0 = as many as
 * fit), item order within a group (0: grid by grid, largest grid first;
 * 1: round-robin over the group's grids), the L2 budget per group in bytes
 * of both fields (0 = 40 % of the device's L2; -1 = one group), and the
 * load path (march 0: each warp stages its rows in shared memory, one bulk
 * copy per row completed on the row slot's mbarrier, 8 rows in flight, or
 * 16-byte cp.async copies for grids on the native FP64 path; 1: rows
 * marched through registers).  timeout_ms bounds every device wait (0 =
 * 2000 ms).  test_stall_ticket and test_stall_row are fault-injection hooks
 * for tests: that ticket never reports completion, so the waits behind it
 * time out (-1 = off); the first compute warp of the CTA that runs the
 * first ticket never fetches the test_stall_row-th row it stages in the
 * bulk-copy march (counted from that item), so its wait for
 * that row times out (0 = off).  Either way the launch ends early with
 * JACC_ERR_TIMEOUT in the status that jacc_batch_status reports, and the
 * fields hold partial results.  jacc_batch_set_tiles overrides
 * the tile of each grid (rows, cols; 0 = from item_points) and
 * jacc_batch_get_tiles reports every grid's tile, item count and group.
 * jacc_batch_tune times, for probe_sweeps sweeps on the batch's own buffers
 * (their contents change), every combination of load path x CTAs per SM in
 * {2, max} x L2 budget in {20 %, 40 %, 60 % of L2, one group} x item size in
 * {8K, 16K, 32K} points, keeps the fastest, then times each group alone at
 * item sizes {4K .. 64K} and gives that group's grids their best tile (kept
 * only if the whole batch then runs faster); returns the schedule and its
 * time.  */
typedef struct {
  int64_t nx, ny; /* extents, each in [3, 2^31]                                   */
  void* u0;       /* device FP64 field [ny][nx], 16-byte aligned: sweep 0 input    */
  void* u1;       /* device FP64 field, same shape, must not overlap u0            */
} jacc_grid;

typedef struct {
  int32_t item_points;       /* target points per item; 0 = 8192                  */
  int32_t ctas_per_sm;       /* persistent CTAs per SM; 0 = as many as fit        */
  int32_t order;             /* 0 grid by grid, 1 round-robin (within a group)    */
  int32_t timeout_ms;        /* bound on each device wait; 0 = 2000               */
  int64_t test_stall_ticket; /* fault injection for tests; -1 = off               */
  int64_t group_bytes;       /* L2 budget per group; 0 = 40 % of L2, -1 = one     */
  int32_t march;             /* 0 staged in shared memory, 1 registers            */
  int32_t test_stall_row;    /* fault injection for tests; 0 = off                */
} jacc_batch_config;

typedef struct {
  int32_t rows;   /* rows per item (set: 0 = from item_points)                     */
  int32_t cols;   /* columns per item: 64, 128, 256 or 512 (set: 0 = from nx)      */
  int32_t nitems; /* items of the grid (get only)                                  */
  int32_t group;  /* the grid's group (get only)                                   */
} jacc_batch_tile;

typedef struct jacc_batch_s* jacc_batch;

/* Copies the grid descriptors and uploads the device tables (synchronous).
 * cfg may be NULL for the defaults.  The fields stay caller-owned. */
jacc_status jacc_batch_create(int32_t ngrids, const jacc_grid* grids, const jacc_batch_config* cfg, jacc_batch* out);
/* Replace the schedule (synchronous; drops cached graphs). */
jacc_status jacc_batch_configure(jacc_batch b, const jacc_batch_config* cfg);
jacc_status jacc_batch_get_config(jacc_batch b, jacc_batch_config* out);
/* Per-grid tiles (arrays of ngrids entries, host memory); set replans
 * synchronously and drops cached graphs. */
jacc_status jacc_batch_set_tiles(jacc_batch b, int32_t ngrids, const jacc_batch_tile* tiles);
jacc_status jacc_batch_get_tiles(jacc_batch b, int32_t ngrids, jacc_batch_tile* out);
/* nsweeps ping-pong sweeps of every grid.  resid_dev (nullable, device,
 * ngrids * nsweeps doubles, row g = grid g) receives each grid's per-sweep
 * max |v - u| over its interior.  flags: JACC_SWEEP_GRAPH captures the
 * sequence once per (nsweeps, resid_dev) and replays it.  *final_buf = 0 if
 * every grid's result is in u0, 1 if in u1.  Asynchronous on `stream`. */
jacc_status jacc_batch_sweep(jacc_batch b, int32_t nsweeps, double* resid_dev, uint32_t flags, uintptr_t stream,
                             int32_t* final_buf);
/* Synchronises `stream` and reports the last run: JACC_OK, or
 * JACC_ERR_TIMEOUT if a device wait gave up (the fields are then partial). */
jacc_status jacc_batch_status(jacc_batch b, uintptr_t stream);
jacc_status jacc_batch_tune(jacc_batch b, int32_t probe_sweeps, uintptr_t stream, jacc_batch_config* best,
                            double* best_ms);
jacc_status jacc_batch_release(jacc_batch b);

/* jacc_launch_static: jacc_launch without any device allocation.
 * The paper has no counterpart; this exists for callers that cannot allocate
 * device memory when they launch (a memory pool that must own every device
 * byte, a latency-critical path that must not hit cudaMalloc's implicit
 * synchronisation, code that must not fail on allocation).  Arguments,
 * results and errors are those of jacc_launch.  Instead of the handle's
 * cudaMalloc'd word, the FP64 fixed-point scale word lives in a file-scope
 * static device array of 256 bytes (32 words; a launch uses one, whatever the
 * grid size), which every GPU that loads the library holds until exit.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept per device for the
 * device's primary context; jacc_shutdown forgets it (call jacc_shutdown
 * after a cudaDeviceReset).  Every call shares the array and the call
 * clears the word it uses; calls that overlap on the GPU (other streams, or
 * other threads) race on it.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  The handle itself comes from jacc_specialize, which
 * may allocate: create it during set-up. */
jacc_status jacc_launch_static(jacc_kernel k, const void* u_in, void* u_out, double* resid_dev, uintptr_t stream);

/* Release every cached kernel, graph and library allocation, and forget the
 * per-device address of jacc_launch_static's array.  Handles become invalid.
 * Safe to call more than once. */
jacc_status jacc_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* JACC_H */
