// jacc_device.cuh - device code of the runtime-specialised stencil path.
//
// No system headers: the same text (plus jacc_params.h) is compiled by nvcc
// into the precompiled "generic" kernels, where extents and coefficients
// arrive as kernel arguments, and by NVRTC into constant-folded variants,
// where a struct with static constexpr members replaces the argument struct
// (the paper's kernel specialisation, §3.2.2: runtime-invariant parameters
// become constants).
//
// Stencils (the paper's workloads are memory-bound halo stencils, §5.2 and
// Table 1; these are the 5-, 7- and 27-point members of that family):
//   5-point Jacobi (2D)  v = (N + S + W + E) / 4
//   7-point heat   (3D)  v = u + r (sum of 6 faces - 6 u)
//   27-point box   (3D)  v = w0 c + wf (6 faces) + we (12 edges) + wc (8 corners), periodic
// Dirichlet boundary points are copied unchanged.
//
// FP64 arithmetic.  On GB300 the FP64 pipe and every conversion to or from a
// 64-bit type issue at about 2 lanes/clock/SM, against ~100-128 for INT32
// and FP32, so an FP64 stencil done in FP64 instructions is ALU-bound far
// below the HBM roof.  For convex stencils the values never leave
// [-M, M], M = max|u| of the sweep input (maximum principle), so each sweep
// runs in exact 64-bit fixed point: value = q * 2^-F with F = 57 - e(M)
// (|q| < 2^57, six bits of headroom).  Conversions FP64 <-> fixed are done
// with integer instructions; sums and power-of-two scalings are exact, so the
// only rounding is the final, correctly rounded conversion of the exact
// stencil value to FP64.  Non-dyadic coefficients use exact 128-bit products.
// Non-convex coefficients, or a non-finite or tiny input, use the native FP64
// path (chosen per launch by a uniform branch).
#pragma once

#include "jacc_params.h"

#define JD __device__ __forceinline__

// ---------------------------------------------------------------- fixed point

// Fraction bits for the sweep from the bit pattern of max|u| (non-negative
// double).  Returns -1 when the fixed path cannot be used (Inf/NaN input, or a
// maximum below 2^-959 so that the format would leave the normal range).
JD int fx_frac_bits(u64 maxbits) {
  if (maxbits == 0ull) return 57;
  int eb = (int)(maxbits >> 52);
  if (eb >= 0x7ff || eb < 64) return -1;
  return 1079 - eb;  // M < 2^(eb-1022)  =>  |q| < 2^57
}

// x * 2^F truncated toward zero; |x| <= M guarantees the shift is <= 4.
JD i64 fx_from(double x, int F) {
  u64 b = (u64)__double_as_longlong(x);
  int eb = (int)((b >> 52) & 0x7ffull);
  u64 m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  int sh = eb - 1075 + F;
  u64 r = (sh >= 0) ? (m << sh) : ((sh > -64) ? (m >> (-sh)) : 0ull);
  r = (eb == 0) ? 0ull : r;
  return (b >> 63) ? -(i64)r : (i64)r;
}

// q * 2^-E rounded to nearest even.  A carry out of the 53-bit mantissa
// propagates into the exponent field by construction.
JD double fx_to(i64 q, int E) {
  u64 s = (u64)q >> 63;
  u64 a = s ? (u64)(-q) : (u64)q;
  int lz = __clzll((i64)a);
  u64 n = a << (lz & 63);
  u64 mant = n >> 11;
  u64 rem = n & 0x7ffull;
  mant += (u64)((rem > 0x400ull) | ((rem == 0x400ull) & (mant & 1ull)));
  i64 eb = 63 - lz - E + 1023;
  u64 bits = (s << 63) | (((u64)(eb - 1) << 52) + mant);
  return a ? __longlong_as_double((i64)bits) : 0.0;
}

// Unsigned magnitude version (for residual maxima).
JD double fx_to_u(u64 a, int E) { return fx_to((i64)a, E); }

// 128-bit two's complement value.
struct s128 { u64 lo; u64 hi; };

JD s128 mul_s64_u64(i64 a, u64 b) {
  s128 r;
  r.lo = (u64)a * b;
  r.hi = __umul64hi((u64)a, b) - ((a < 0) ? b : 0ull);
  return r;
}
JD s128 add128(s128 x, s128 y) {
  s128 r;
  r.lo = x.lo + y.lo;
  r.hi = x.hi + y.hi + (u64)(r.lo < x.lo);
  return r;
}
JD s128 from_s64_shl(i64 a, int k) {  // a * 2^k, 0 <= k < 64
  s128 r;
  r.lo = (u64)a << k;
  r.hi = (k == 0) ? (u64)(a >> 63) : (u64)(a >> (64 - k));
  return r;
}
// (x.hi:x.lo) * 2^-E rounded to nearest even.
JD double fx128_to(s128 x, int E) {
  u64 s = x.hi >> 63;
  u64 lo = x.lo, hi = x.hi;
  if (s) { lo = ~lo + 1ull; hi = ~hi + (u64)(lo == 0ull); }
  int lz = hi ? __clzll((i64)hi) : 64 + __clzll((i64)lo);
  u64 nh, nl;
  if (lz >= 64) { nh = lo << (lz - 64); nl = 0ull; }
  else if (lz == 0) { nh = hi; nl = lo; }
  else { nh = (hi << lz) | (lo >> (64 - lz)); nl = lo << lz; }
  u64 mant = nh >> 11;
  u64 rem = nh & 0x7ffull;
  u64 sticky = (u64)(nl != 0ull);
  mant += (u64)((rem > 0x400ull) | ((rem == 0x400ull) & ((mant & 1ull) | sticky)));
  i64 eb = 127 - lz - E + 1023;
  u64 bits = (s << 63) | (((u64)(eb - 1) << 52) + mant);
  return (lo | hi) ? __longlong_as_double((i64)bits) : 0.0;
}

// ---------------------------------------------------------------- load / store helpers

template <class T, int V> struct VecT;
template <> struct VecT<double, 1> { typedef double type; };
template <> struct VecT<double, 2> { typedef double2 type; };
template <> struct VecT<float, 1> { typedef float type; };
template <> struct VecT<float, 4> { typedef float4 type; };

// CG = true loads through L2 only (ld.global.cg): required where the same
// kernel launch writes the array (the persistent batched kernel), since the
// non-coherent and L1 paths may return stale lines there.
template <bool CG, class T> JD T ld1(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}
template <class T, int V, bool CG = false> JD void ldv(const T* __restrict__ p, T (&r)[V]) {
  if constexpr (V == 1) { r[0] = ld1<CG>(p); }
  else if constexpr (V == 2) {
    double2 t = ld1<CG>(reinterpret_cast<const double2*>(p)); r[0] = t.x; r[1] = t.y;
  } else {
    float4 t = ld1<CG>(reinterpret_cast<const float4*>(p)); r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
  }
}
template <class T, int V> JD void stv(T* __restrict__ p, const T (&r)[V]) {
  if constexpr (V == 1) { p[0] = r[0]; }
  else if constexpr (V == 2) { double2 t; t.x = r[0]; t.y = r[1]; *reinterpret_cast<double2*>(p) = t; }
  else { float4 t; t.x = r[0]; t.y = r[1]; t.z = r[2]; t.w = r[3]; *reinterpret_cast<float4*>(p) = t; }
}

// Arithmetic modes.
#define JM_NATIVE 0
#define JM_FIXED 1

// Internal value type: T for native, int64 fixed point for JM_FIXED.
template <class T, int MODE> struct WT { typedef T type; };
template <class T> struct WT<T, JM_FIXED> { typedef i64 type; };

template <class T, int MODE> JD typename WT<T, MODE>::type cvt_in(T x, int F) {
  if constexpr (MODE == JM_FIXED) return fx_from((double)x, F);
  else return x;
}

// Per-thread residual accumulator: the magnitude of a fixed-point
// difference (converted once at the end), or a non-negative T.
template <class T, int MODE> struct RT { typedef T type; };
template <class T> struct RT<T, JM_FIXED> { typedef u64 type; };

// ---------------------------------------------------------------- block reductions

// Maximum of a 64-bit word over the (converged) warp: the maximum of the high
// halves, then the maximum of the low halves of the lanes that hold it; two
// redux.sync operations instead of five shuffle rounds.
JD u64 warp_max_u64(u64 v) {
  const u32 hi = __reduce_max_sync(0xffffffffu, (u32)(v >> 32));
  const u32 lo = __reduce_max_sync(0xffffffffu, (u32)(v >> 32) == hi ? (u32)v : 0u);
  return ((u64)hi << 32) | lo;
}
JD double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Max over the block of a non-negative double given as its bit pattern, then
// one atomicMax per block (non-negative doubles order like their bit patterns).
template <int NT> JD void block_max_to(u64 bits, double* out) {
  __shared__ u64 red[NT / 32];
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  bits = warp_max_u64(bits);
  if ((t & 31) == 0) red[t >> 5] = bits;
  __syncthreads();
  if (t < 32) {
    u64 v = (t < NT / 32) ? red[t] : 0ull;
    v = warp_max_u64(v);
    if (t == 0 && out) atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)v);
  }
}

template <int NT> JD void block_sum_to(double s, double* out) {
  __shared__ double red[NT / 32];
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  s = warp_sum_f64(s);
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t < 32) {
    double v = (t < NT / 32) ? red[t] : 0.0;
    v = warp_sum_f64(v);
    if (t == 0 && out) atomicAdd(out, v);
  }
}

JD u64 dbits(double d) { return (u64)__double_as_longlong(d); }

// Programmatic dependent launch: a sweep kernel may be launched while the
// previous one still runs (its CTAs fill the SMs the previous grid frees);
// this waits until the previous grid has completed and its memory is
// visible, before the kernel touches any field.  A no-op when the launch
// did not ask for programmatic serialisation.
JD void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
JD double fabs_bits_free(double d) { return __longlong_as_double(__double_as_longlong(d) & 0x7fffffffffffffffLL); }

// FP32 error-free sum (Knuth TwoSum) accumulated as hi + lo.
JD void two_sum_acc(float& hi, float& lo, float x) {
  float s = hi + x;
  float bp = s - hi;
  float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

// ====================================================================== 5-point Jacobi (2D)
//
// One warp owns 32*V consecutive columns starting at its lane-0 column and
// marches rows [ys, ye), keeping rows y-1, y, y+1 in registers; the x
// neighbours come from warp shuffles (lanes 0 and 31 read the edge columns
// from memory).  Row y+3 is prefetched two iterations ahead.  All 32 lanes
// must call it with the same ys, ye (full-mask shuffles).

template <class T, int V, int MODE, bool CG>
JD void jacobi_march(const T* __restrict__ u, T* __restrict__ v, i64 nx, i64 ny, i64 x0, i64 ys, i64 ye, int F,
                     typename RT<T, MODE>::type& rmax) {
  typedef typename WT<T, MODE>::type W;
  const int lane = threadIdx.x & 31;
  const bool xin = x0 < nx;
  T rup[V], rcur[V], rdn[V], rnx[V];
  W up[V], cur[V], dn[V];
#pragma unroll
  for (int e = 0; e < V; ++e) { rup[e] = rcur[e] = rdn[e] = rnx[e] = T(0); }
  if (xin) {
    if (ys >= 1) ldv<T, V, CG>(u + (ys - 1) * nx + x0, rup);
    ldv<T, V, CG>(u + ys * nx + x0, rcur);
    if (ys + 1 < ny) ldv<T, V, CG>(u + (ys + 1) * nx + x0, rdn);
    if (ys + 2 < ny) ldv<T, V, CG>(u + (ys + 2) * nx + x0, rnx);
  }
#pragma unroll
  for (int e = 0; e < V; ++e) {
    up[e] = cvt_in<T, MODE>(rup[e], F);
    cur[e] = cvt_in<T, MODE>(rcur[e], F);
    dn[e] = cvt_in<T, MODE>(rdn[e], F);
  }
  for (i64 y = ys; y < ye; ++y) {
    // x neighbours of the row
    W left = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
    W right = __shfl_down_sync(0xffffffffu, cur[0], 1);
    if (lane == 0 && xin && x0 >= 1) left = cvt_in<T, MODE>(ld1<CG>(u + y * nx + x0 - 1), F);
    if (lane == 31 && xin && x0 + V < nx) right = cvt_in<T, MODE>(ld1<CG>(u + y * nx + x0 + V), F);
    // prefetch row y+3
    T rnn[V];
#pragma unroll
    for (int e = 0; e < V; ++e) rnn[e] = T(0);
    if (xin && y + 3 < ny) ldv<T, V, CG>(u + (y + 3) * nx + x0, rnn);

    const bool yint = (y >= 1) && (y <= ny - 2);
    T out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const i64 x = x0 + e;
      const W xl = (e == 0) ? left : cur[e - 1];
      const W xr = (e == V - 1) ? right : cur[e + 1];
      const bool in = yint && (x >= 1) && (x <= nx - 2);
      {
        const T s = (up[e] + dn[e]) + (xl + xr);
        const T r = T(0.25) * s;
        out[e] = in ? r : rcur[e];
        T d = r - rcur[e];
        d = d < T(0) ? -d : d;
        if (in && d > rmax) rmax = d;
      }
    }
    if (xin) stv<T, V>(v + y * nx + x0, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      up[e] = cur[e];
      cur[e] = dn[e];
      rcur[e] = rdn[e];
      rdn[e] = rnx[e];
      dn[e] = cvt_in<T, MODE>(rnx[e], F);
      rnx[e] = rnn[e];
    }
  }
}

// ====================================================================== 3D z-marching tiles
//
// CTA = BX x BY threads covering x in [bx0, bx0 + BX*V), y in [by0, by0 + BY),
// marching z over [cz0, cz0 + ZC).  The current plane lives in shared memory
// with a one-point halo in x and y (double-buffered, so one __syncthreads per
// plane); each thread keeps its own column's z-1, z, z+1 in registers.
// Loads for plane z+1 (halo) and z+2 (own) are issued one iteration ahead.

template <class W, int BX, int BY, int V> struct alignas(16) Plane {
  // row layout: [pad V-1][left halo][TX values][right halo][pad V-1]
  static constexpr int TX = BX * V;
  static constexpr int RW = TX + 2 * V;
  static constexpr int ROWS = BY + 2;
  W a[2][ROWS][RW];
};

template <class T, int BX, int BY, int V> struct HaloFetch {
  T yrow[V];  // thread rows 0 / BY-1: the row above / below the tile
  T xl, xr;   // threads tx 0 / BX-1: the column left / right of the tile
};

template <class T, int BX, int BY, int V, class P>
JD void fetch_halo(const T* __restrict__ u, const P& p, i64 z, i64 bx0, i64 by0, bool periodic,
                   HaloFetch<T, BX, BY, V>& h) {
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 x0 = bx0 + (i64)tx * V;
  const i64 y = by0 + ty;
  if (periodic) z = (z + nz) % nz;
  const T* pl = u + z * nx * ny;
#pragma unroll
  for (int e = 0; e < V; ++e) h.yrow[e] = T(0);
  h.xl = h.xr = T(0);
  // Periodic tiles that overhang the grid load the periodic image, so the
  // slot after the last column (row) holds column (row) 0.
  const i64 xl0 = periodic ? (x0 % nx) : x0;
  if (xl0 < nx) {
    if (ty == 0) {
      i64 yy = by0 - 1;
      if (periodic) yy = (yy + ny) % ny;
      if (yy >= 0) ldv<T, V>(pl + yy * nx + xl0, h.yrow);
    }
    if (ty == BY - 1) {
      i64 yy = by0 + BY;
      if (periodic) yy = yy % ny;
      if (yy < ny) ldv<T, V>(pl + yy * nx + xl0, h.yrow);
    }
  }
  // x halo: the thread at tx == 0 fetches for its own row (and the halo rows
  // through the diagonal corners below), tx == BX-1 likewise on the right.
  if (y < ny || periodic) {
    i64 yy = periodic ? (y % ny) : y;
    if (tx == 0) {
      i64 xx = bx0 - 1;
      if (periodic) xx = (xx + nx) % nx;
      if (xx >= 0 && yy < ny) h.xl = __ldg(pl + yy * nx + xx);
    }
    if (tx == BX - 1) {
      i64 xx = bx0 + BX * V;
      if (periodic) xx = xx % nx;
      if (xx < nx && yy < ny) h.xr = __ldg(pl + yy * nx + xx);
    }
  }
}

// Corner halo values (needed by the 27-point stencil only): the four points
// diagonal to the tile.  Fetched by thread (0,0) and friends; returned raw.
template <class T, class P>
JD T fetch_corner(const T* __restrict__ u, const P& p, i64 z, i64 xx, i64 yy) {
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  z = (z + nz) % nz;
  xx = (xx + nx) % nx;
  yy = (yy + ny) % ny;
  return __ldg(u + (z * ny + yy) * nx + xx);
}

// Write this thread's converted plane values and its halo share into buffer b.
template <class T, int BX, int BY, int V, int MODE>
JD void put_plane(Plane<typename WT<T, MODE>::type, BX, BY, V>& sm, int b, const typename WT<T, MODE>::type (&own)[V],
                  const HaloFetch<T, BX, BY, V>& h, int F) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  typedef typename WT<T, MODE>::type W;
  W* row = &sm.a[b][ty + 1][V + tx * V];
#pragma unroll
  for (int e = 0; e < V; ++e) row[e] = own[e];
  if (ty == 0) {
    W* hr = &sm.a[b][0][V + tx * V];
#pragma unroll
    for (int e = 0; e < V; ++e) hr[e] = cvt_in<T, MODE>(h.yrow[e], F);
  }
  if (ty == BY - 1) {
    W* hr = &sm.a[b][BY + 1][V + tx * V];
#pragma unroll
    for (int e = 0; e < V; ++e) hr[e] = cvt_in<T, MODE>(h.yrow[e], F);
  }
  if (tx == 0) sm.a[b][ty + 1][V - 1] = cvt_in<T, MODE>(h.xl, F);
  if (tx == BX - 1) sm.a[b][ty + 1][V + BX * V] = cvt_in<T, MODE>(h.xr, F);
}


// ---------------------------------------------------------------- 7-point heat
//
// Fixed path: with S the sum of the six faces and L = S - 6u (exact, scale F),
//   JACC_FP_SMALL (r = fb 2^-k, k <= 5): v 2^(F+k) = fa u + fb S,  fa = 2^k - 6 fb
//   JACC_FP_WIDE  (r = m 2^-k, m odd):   v 2^(F+k) = u 2^k + m L   (128-bit)
// and |v - u| = r |L|, so the residual only needs max |L|.

template <class T, int BX, int BY, int V, int ZC, int MODE, class P>
JD void heat3d_body(const T* __restrict__ u, T* __restrict__ v, const P& p, int F, typename RT<T, MODE>::type& rmax,
                    Plane<typename WT<T, MODE>::type, BX, BY, V>& sm, int ys_mul = 1, int ysub = 0) {
  typedef typename WT<T, MODE>::type W;
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const i64 sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 bx0 = (i64)blockIdx.x * (BX * V);
  const i64 by0 = ((i64)blockIdx.y * ys_mul + ysub) * BY;  // a CTA may cover ys_mul tiles of BY rows
  const i64 x0 = bx0 + (i64)tx * V;
  const i64 y = by0 + ty;
  const bool act = (x0 < nx) && (y < ny);
  const i64 cz0 = (i64)blockIdx.z * ZC;
  const i64 cz1 = (cz0 + ZC < nz) ? cz0 + ZC : nz;
  const T* urow = u + y * nx + x0;
  T* vrow = v + y * nx + x0;

  // Boundary planes are copied by the chunk that holds them.
  if (act && cz0 == 0) { T t[V]; ldv<T, V>(urow, t); stv<T, V>(vrow, t); }
  if (act && cz1 == nz) { T t[V]; ldv<T, V>(urow + (nz - 1) * sz, t); stv<T, V>(vrow + (nz - 1) * sz, t); }
  const i64 z0 = cz0 < 1 ? 1 : cz0;
  const i64 z1 = cz1 > nz - 1 ? nz - 1 : cz1;
  if (z0 >= z1) return;  // block-uniform

  const bool yint = (y >= 1) && (y <= ny - 2);
  T rcur[V], rzn[V], rzn2[V];
  W zp[V], cur[V], zn[V];
  {
    T t[V];
#pragma unroll
    for (int e = 0; e < V; ++e) t[e] = rcur[e] = rzn[e] = rzn2[e] = T(0);
    if (act) {
      ldv<T, V>(urow + (z0 - 1) * sz, t);
      ldv<T, V>(urow + z0 * sz, rcur);
      ldv<T, V>(urow + (z0 + 1) * sz, rzn);
      if (z0 + 2 < nz) ldv<T, V>(urow + (z0 + 2) * sz, rzn2);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) { zp[e] = cvt_in<T, MODE>(t[e], F); cur[e] = cvt_in<T, MODE>(rcur[e], F); }
  }
  HaloFetch<T, BX, BY, V> h, hn;
  fetch_halo<T, BX, BY, V>(u, p, z0, bx0, by0, false, h);
  hn = h;
  int b = 0;
  for (i64 z = z0; z < z1; ++z) {
#pragma unroll
    for (int e = 0; e < V; ++e) zn[e] = cvt_in<T, MODE>(rzn[e], F);
    T rn3[V];
#pragma unroll
    for (int e = 0; e < V; ++e) rn3[e] = T(0);
    if (act && z + 3 < nz) ldv<T, V>(urow + (z + 3) * sz, rn3);
    if (z + 1 < z1) fetch_halo<T, BX, BY, V>(u, p, z + 1, bx0, by0, false, hn);

    put_plane<T, BX, BY, V, MODE>(sm, b, cur, h, F);
    __syncthreads();
    const W* rm = &sm.a[b][ty][V + tx * V];
    const W* r0 = &sm.a[b][ty + 1][V + tx * V];
    const W* rp = &sm.a[b][ty + 2][V + tx * V];
    T out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const i64 x = x0 + e;
      const bool in = act && yint && (x >= 1) && (x <= nx - 2);
      const W xl = (e == 0) ? r0[-1] : cur[e - 1];
      const W xr = (e == V - 1) ? r0[V] : cur[e + 1];
      const W s = ((xl + xr) + (rm[e] + rp[e])) + (zp[e] + zn[e]);
      {
        const T r = (T)p.c0;
        const T o = cur[e] + r * (s - T(6) * cur[e]);
        out[e] = in ? o : rcur[e];
        T d = o - cur[e];
        d = d < T(0) ? -d : d;
        if (in && d > rmax) rmax = d;
      }
    }
    if (act) stv<T, V>(vrow + z * sz, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      zp[e] = cur[e];
      cur[e] = zn[e];
      rcur[e] = rzn[e];
      rzn[e] = rzn2[e];
      rzn2[e] = rn3[e];
    }
    h = hn;
    b ^= 1;
  }
}

// Residual of the heat sweep from max |L|: r max|L| scaled.
// r = fb 2^-k with 1 <= k <= 4 and fb <= 2 (r = 1/8, 1/16, ...): the
// constant-folded staged heat kernels form v 2^F directly as
// (fb S + (2^k - 6 fb) c + 2^(k-1)) >> k, which equals c + round(r L 2^F) bit
// for bit (2^k c is a multiple of 2^k); every term stays below 2^62 for
// |c| < 2^57 and |S| < 6 * 2^57.  (Every fixed-point heat kernel takes its
// residual from the increment v - c, so this changes no result.)
template <class P> JD bool heat_fold(const P& p) {
  return p.fpath == JACC_FP_SMALL && p.fk >= 1 && p.fk <= 4 && p.fb >= 1 && p.fb <= 2;
}


// ---------------------------------------------------------------- 27-point periodic box
//
// Per plane and own point: c = centre, f = the 4 in-plane faces, g = the 4
// in-plane diagonals.  With planes z-1 (m), z (0), z+1 (n):
//   v = w0 c0 + wf (f0 + cm + cn) + we (g0 + fm + fn) + wc (gm + gn).
// The shared-memory plane holds plane z+1 at iteration z.  Fixed path:
// v 2^(F+K) = sum_j fw_j * class_j exactly in 128 bits (w_j = fw_j 2^-K).

template <class T, int BX, int BY, int V, int MODE>
JD void plane_cfe(const Plane<typename WT<T, MODE>::type, BX, BY, V>& sm, int b, typename WT<T, MODE>::type (&c)[V],
                  typename WT<T, MODE>::type (&f)[V], typename WT<T, MODE>::type (&g)[V]) {
  typedef typename WT<T, MODE>::type W;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const W* rm = &sm.a[b][ty][V + tx * V];
  const W* r0 = &sm.a[b][ty + 1][V + tx * V];
  const W* rp = &sm.a[b][ty + 2][V + tx * V];
  W m[V + 2], z[V + 2], q[V + 2];
#pragma unroll
  for (int e = -1; e <= V; ++e) { m[e + 1] = rm[e]; z[e + 1] = r0[e]; q[e + 1] = rp[e]; }
#pragma unroll
  for (int e = 0; e < V; ++e) {
    c[e] = z[e + 1];
    f[e] = (z[e] + z[e + 2]) + (m[e + 1] + q[e + 1]);
    g[e] = (m[e] + m[e + 2]) + (q[e] + q[e + 2]);
  }
}

// The four halo corners of the tile (periodic wrap), fetched by thread (0,0).
template <class T, int BX, int BY, int V, class P>
JD void fetch_corners(const T* __restrict__ u, const P& p, i64 z, i64 bx0, i64 by0, T (&cr)[4]) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const i64 nx = p.nx, ny = p.ny, nz = p.nz;
    const i64 zz = (z % nz + nz) % nz;
    const i64 xl = (bx0 - 1 + nx) % nx, xr = (bx0 + BX * V) % nx;
    const i64 yt = (by0 - 1 + ny) % ny, yb = (by0 + BY) % ny;
    const T* pl = u + zz * nx * ny;
    cr[0] = __ldg(pl + yt * nx + xl);
    cr[1] = __ldg(pl + yt * nx + xr);
    cr[2] = __ldg(pl + yb * nx + xl);
    cr[3] = __ldg(pl + yb * nx + xr);
  }
}

template <class T, int BX, int BY, int V, int MODE>
JD void put_corners(Plane<typename WT<T, MODE>::type, BX, BY, V>& sm, int b, const T (&cr)[4], int F) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    sm.a[b][0][V - 1] = cvt_in<T, MODE>(cr[0], F);
    sm.a[b][0][V + BX * V] = cvt_in<T, MODE>(cr[1], F);
    sm.a[b][BY + 1][V - 1] = cvt_in<T, MODE>(cr[2], F);
    sm.a[b][BY + 1][V + BX * V] = cvt_in<T, MODE>(cr[3], F);
  }
}

// Sum accumulator: FP64 for FP64 data; an FP32 error-free (hi, lo) pair for
// FP32 data, combined in FP64 once per thread.
template <class T> struct SumAcc {
  double d = 0.0;
  JD void add(T x) { d += (double)x; }
  JD double total() const { return d; }
};
template <> struct SumAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  JD void add(float x) { two_sum_acc(hi, lo, x); }
  JD double total() const { return (double)hi + (double)lo; }
};

template <class T, int BX, int BY, int V, int MODE, class P>
JD void plane_load_put(const T* __restrict__ u, const P& p, i64 z, i64 bx0, i64 by0, bool act, const T* urow,
                       Plane<typename WT<T, MODE>::type, BX, BY, V>& sm, int b, int F) {
  typedef typename WT<T, MODE>::type W;
  const i64 nz = p.nz, sz = p.nx * p.ny;
  T r[V];
#pragma unroll
  for (int e = 0; e < V; ++e) r[e] = T(0);
  if (act) ldv<T, V>(urow + ((z % nz + nz) % nz) * sz, r);
  W own[V];
#pragma unroll
  for (int e = 0; e < V; ++e) own[e] = cvt_in<T, MODE>(r[e], F);
  HaloFetch<T, BX, BY, V> h;
  fetch_halo<T, BX, BY, V>(u, p, z, bx0, by0, true, h);
  T cr[4];
  fetch_corners<T, BX, BY, V>(u, p, z, bx0, by0, cr);
  put_plane<T, BX, BY, V, MODE>(sm, b, own, h, F);
  put_corners<T, BX, BY, V, MODE>(sm, b, cr, F);
}

template <class T, int BX, int BY, int V, int ZC, int MODE, class P>
JD void box27_body(const T* __restrict__ u, T* __restrict__ v, const P& p, int F, SumAcc<T>& acc,
                   Plane<typename WT<T, MODE>::type, BX, BY, V>& sm) {
  typedef typename WT<T, MODE>::type W;
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const i64 sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 bx0 = (i64)blockIdx.x * (BX * V);
  const i64 by0 = (i64)blockIdx.y * BY;
  const i64 x0 = bx0 + (i64)tx * V;
  const i64 y = by0 + ty;
  const bool act = (x0 < nx) && (y < ny);
  const i64 z0 = (i64)blockIdx.z * ZC;
  const i64 z1 = (z0 + ZC < nz) ? z0 + ZC : nz;
  const T* urow = u + (y % ny) * nx + (x0 % nx);  // periodic image for overhanging threads
  T* vrow = v + y * nx + x0;

  W cm[V], fm[V], gm[V], c0[V], f0[V], g0[V];
  int b = 0;
  plane_load_put<T, BX, BY, V, MODE>(u, p, z0 - 1, bx0, by0, true, urow, sm, b, F);
  __syncthreads();
  plane_cfe<T, BX, BY, V, MODE>(sm, b, cm, fm, gm);
  b ^= 1;
  plane_load_put<T, BX, BY, V, MODE>(u, p, z0, bx0, by0, true, urow, sm, b, F);
  __syncthreads();
  plane_cfe<T, BX, BY, V, MODE>(sm, b, c0, f0, g0);
  b ^= 1;
  for (i64 z = z0; z < z1; ++z) {
    plane_load_put<T, BX, BY, V, MODE>(u, p, z + 1, bx0, by0, true, urow, sm, b, F);
    __syncthreads();
    W cn[V], fn[V], gn[V];
    plane_cfe<T, BX, BY, V, MODE>(sm, b, cn, fn, gn);
    T out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const W F1 = (f0[e] + cm[e]) + cn[e];
      const W E2 = (g0[e] + fm[e]) + fn[e];
      const W C3 = gm[e] + gn[e];
      out[e] = ((T)p.c0 * c0[e] + (T)p.c1 * F1) + ((T)p.c2 * E2 + (T)p.c3 * C3);
    }
    if (act) {
      stv<T, V>(vrow + z * sz, out);
#pragma unroll
      for (int e = 0; e < V; ++e) acc.add(out[e]);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      cm[e] = c0[e]; fm[e] = f0[e]; gm[e] = g0[e];
      c0[e] = cn[e]; f0[e] = fn[e]; g0[e] = gn[e];
    }
    b ^= 1;
  }
}

// ---------------------------------------------------------------- 27-point periodic box, native arithmetic
//
// All periodic offsets are computed once per thread (no division in the
// plane loop); plane z+2 is fetched into registers one iteration ahead and
// stored to shared memory the next.  Row reads from shared memory use 16-byte
// vectors for the thread's own V columns.

template <class W, int V> JD void lds_row(const W* p, W (&r)[V + 2]) {
  r[0] = p[-1];
  if constexpr (V * sizeof(W) == 16 && V == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r[1] = t.x; r[2] = t.y; r[3] = t.z; r[4] = t.w;
  } else if constexpr (V * sizeof(W) == 16 && V == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r[1] = t.x; r[2] = t.y;
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) r[e + 1] = p[e];
  }
  r[V + 1] = p[V];
}

// Stores a thread's V values to a shared-memory row as one 16-byte vector
// where the width allows.
template <class W, int V> JD void sts_row(W* p, const W (&r)[V]) {
  if constexpr (V * sizeof(W) == 16 && V == 4) {
    float4 t;
    t.x = r[0]; t.y = r[1]; t.z = r[2]; t.w = r[3];
    *reinterpret_cast<float4*>(p) = t;
  } else if constexpr (V * sizeof(W) == 16 && V == 2) {
    double2 t;
    t.x = r[0]; t.y = r[1];
    *reinterpret_cast<double2*>(p) = t;
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) p[e] = r[e];
  }
}

template <class T, int BX, int BY, int V>
struct Box27Fetch {
  T own[V], hrow[V], hx, cr[4];
};

template <class T, int BX, int BY, int V, int ZC, class P>
JD void box27_body2(const T* __restrict__ u, T* __restrict__ v, const P& p, SumAcc<T>& acc, bool want_sum,
                    Plane<T, BX, BY, V>& sm) {
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const i64 sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 bx0 = (i64)blockIdx.x * (BX * V);
  const i64 by0 = (i64)blockIdx.y * BY;
  const i64 x0 = bx0 + (i64)tx * V;
  const i64 y = by0 + ty;
  const bool act = (x0 < nx) && (y < ny);
  const i64 z0 = (i64)blockIdx.z * ZC;
  const i64 z1 = (z0 + ZC < nz) ? z0 + ZC : nz;
  // periodic images, once per thread (threads overhanging the grid use them too)
  const i64 xo = x0 % nx, yo = y % ny;
  const i64 own_off = yo * nx + xo;
  const bool hy = (ty == 0) || (ty == BY - 1);
  const i64 hy_off = ((ty == 0) ? (by0 - 1 + ny) % ny : (by0 + BY) % ny) * nx + xo;
  const bool hx = (tx == 0) || (tx == BX - 1);
  const i64 hx_off = yo * nx + ((tx == 0) ? (bx0 - 1 + nx) % nx : (bx0 + BX * V) % nx);
  const bool corner = (tx == 0) && (ty == 0);
  i64 c_off[4] = {0, 0, 0, 0};
  if (corner) {
    const i64 xl = (bx0 - 1 + nx) % nx, xr = (bx0 + BX * V) % nx;
    const i64 yt = (by0 - 1 + ny) % ny, yb = (by0 + BY) % ny;
    c_off[0] = yt * nx + xl;
    c_off[1] = yt * nx + xr;
    c_off[2] = yb * nx + xl;
    c_off[3] = yb * nx + xr;
  }
  auto fetch = [&](i64 zoff, Box27Fetch<T, BX, BY, V>& f) {
    const T* pl = u + zoff;
    ldv<T, V>(pl + own_off, f.own);
    if (hy) ldv<T, V>(pl + hy_off, f.hrow);
    if (hx) f.hx = __ldg(pl + hx_off);
    if (corner) {
#pragma unroll
      for (int k = 0; k < 4; ++k) f.cr[k] = __ldg(pl + c_off[k]);
    }
  };
  auto put = [&](const Box27Fetch<T, BX, BY, V>& f, int b) {
    sts_row<T, V>(&sm.a[b][ty + 1][V + tx * V], f.own);
    if (hy) sts_row<T, V>(&sm.a[b][ty == 0 ? 0 : BY + 1][V + tx * V], f.hrow);
    if (tx == 0) sm.a[b][ty + 1][V - 1] = f.hx;
    if (tx == BX - 1) sm.a[b][ty + 1][V + BX * V] = f.hx;
    if (corner) {
      sm.a[b][0][V - 1] = f.cr[0];
      sm.a[b][0][V + BX * V] = f.cr[1];
      sm.a[b][BY + 1][V - 1] = f.cr[2];
      sm.a[b][BY + 1][V + BX * V] = f.cr[3];
    }
  };
  auto cfe = [&](int b, T (&c)[V], T (&f)[V], T (&g)[V]) {
    T m[V + 2], zz[V + 2], q[V + 2];
    lds_row<T, V>(&sm.a[b][ty][V + tx * V], m);
    lds_row<T, V>(&sm.a[b][ty + 1][V + tx * V], zz);
    lds_row<T, V>(&sm.a[b][ty + 2][V + tx * V], q);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      c[e] = zz[e + 1];
      f[e] = (zz[e] + zz[e + 2]) + (m[e + 1] + q[e + 1]);
      g[e] = (m[e] + m[e + 2]) + (q[e] + q[e + 2]);
    }
  };
  auto next_plane = [&](i64 zi) { return zi + 1 == nz ? (i64)0 : zi + 1; };

  const T w0 = (T)p.c0, wf = (T)p.c1, we = (T)p.c2, wc = (T)p.c3;
  T cm[V], fm[V], gm[V], c0[V], f0[V], g0[V];
  Box27Fetch<T, BX, BY, V> fa, fb;
  i64 zi = (z0 - 1 + nz) % nz;  // plane z0 - 1
  fetch(zi * sz, fa);
  zi = next_plane(zi);           // plane z0
  fetch(zi * sz, fb);
  put(fa, 0);
  __syncthreads();
  cfe(0, cm, fm, gm);
  put(fb, 1);
  zi = next_plane(zi);           // plane z0 + 1
  fetch(zi * sz, fa);
  __syncthreads();
  cfe(1, c0, f0, g0);
  int b = 0;
  for (i64 z = z0; z < z1; ++z) {
    put(fa, b);                   // plane z + 1
    if (z + 1 < z1) {
      zi = next_plane(zi);        // plane z + 2, one iteration ahead
      fetch(zi * sz, fa);
    }
    __syncthreads();
    T cn[V], fn[V], gn[V];
    cfe(b, cn, fn, gn);
    T out[V];
#pragma unroll
    for (int e = 0; e < V; ++e)
      out[e] = (w0 * c0[e] + wf * ((f0[e] + cm[e]) + cn[e])) + (we * ((g0[e] + fm[e]) + fn[e]) + wc * (gm[e] + gn[e]));
    if (act) {
      stv<T, V>(v + z * sz + y * nx + x0, out);
      if (want_sum) {
#pragma unroll
        for (int e = 0; e < V; ++e) acc.add(out[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      cm[e] = c0[e]; fm[e] = f0[e]; gm[e] = g0[e];
      c0[e] = cn[e]; f0[e] = fn[e]; g0[e] = gn[e];
    }
    b ^= 1;
  }
}

// ---------------------------------------------------------------- bulk-copy staged planes
//
// Plane staging with the bulk-copy engine: cp.async.bulk copies rows of the
// input field from global to shared memory and counts the bytes that landed
// on an mbarrier of the stage ("full"); no register holds data in flight, so
// a CTA keeps up to S planes outstanding at no register cost.  Each stage
// also has an "empty" mbarrier on which every warp arrives once it has read
// the stage; warp 0 waits on it before it reuses the stage.  Every wait gives
// up after JParams::timeout_ns (%globaltimer), records JACC_DEV_TIMEOUT and
// lets the CTA finish; before it returns, warp 0 waits (bounded too) for the
// copies it has issued, so no copy targets the shared memory of a CTA that
// has exited.

JD u32 smem_u32(const void* ptr) { return (u32)__cvta_generic_to_shared(ptr); }
JD u64 gtimer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
JD void mbar_init(u64* bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
JD void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
JD void mbar_expect_tx(u64* bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
JD void mbar_arrive(u64* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
JD bool mbar_try(u64* bar, u32 parity) {
  u32 done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// try_wait that may suspend the thread for up to `hint_ns` until the phase
// completes, so waiting warps take no issue slots.
JD bool mbar_try_suspend(u64* bar, u32 parity, u32 hint_ns) {
  u32 done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0;
}
// Waits for the completion of the phase with the given parity; false after
// limit_ns without it.
JD bool mbar_wait(u64* bar, u32 parity, i64 limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const u64 t0 = gtimer_ns();
  while (!mbar_try_suspend(bar, parity, 200000u))
    if ((i64)(gtimer_ns() - t0) > limit_ns) return false;
  return true;
}
// One bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completion counted in bytes on `bar`.
JD void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Geometry of the staged 27-point FP32 kernel: BX x BY threads, each owning 4
// consecutive columns (one 16-byte vector) of 2 consecutive rows, so a CTA
// computes a TW x TH tile per plane.  A stage holds R = TH + 2 rows of
// W = TW + 8 floats: slot i of staged row r is column (bx0 - 4 + i) mod nx of
// row (by0 - 1 + r) mod ny (the periodic images, so halo columns and rows need
// no special case).  The halo is 4 columns wide on each side because bulk
// copies move whole 16-byte units; columns bx0 - 1 and bx0 + TW are used.
template <int BX, int BY> struct Box27S {
  static constexpr int RY = 2;
  static constexpr int TW = BX * 4, TH = BY * RY;
  static constexpr int W = TW + 8, R = TH + 2;
  static constexpr int STAGE_BYTES = W * R * 4;
  static constexpr int S0 = 40960 / STAGE_BYTES;
  static constexpr int S = S0 < 2 ? 2 : (S0 > 4 ? 4 : S0);  // stages, 2..4, at most ~40 KB
  static constexpr int NW = BX * BY / 32;
};

template <int BX, int BY> struct alignas(128) Box27SSmem {
  float st[Box27S<BX, BY>::S][Box27S<BX, BY>::R][Box27S<BX, BY>::W];
  u64 full[Box27S<BX, BY>::S];
  u64 empty[Box27S<BX, BY>::S];
};

// Warp 0 requests staged plane zg into stage s: lane 0 posts the byte count,
// then lane r copies staged row r as one bulk copy, or as two or more where
// the row's slots wrap around the periodic x boundary.
template <int BX, int BY, class P>
JD void box27s_issue(Box27SSmem<BX, BY>& sm, int s, const float* __restrict__ u, const P& p, i64 zg, i64 bx0, i64 by0,
                     int weff) {
  typedef Box27S<BX, BY> G;
  const i64 nx = p.nx, ny = p.ny;
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_expect_tx(&sm.full[s], (u32)(G::R * weff * 4));
  __syncwarp();
  for (int r = lane; r < G::R; r += 32) {
    i64 yg = (by0 - 1 + r) % ny;
    if (yg < 0) yg += ny;
    const float* row = u + (zg * ny + yg) * nx;
    float* dst = &sm.st[s][r][0];
    i64 c = bx0 - 4;
    if (c < 0) c += nx;
    int i = 0;
    while (i < weff) {
      i64 len = nx - c;
      if (len > weff - i) len = weff - i;
      bulk_g2s(dst + i, row + c, (u32)(len * 4), &sm.full[s]);
      i += (int)len;
      c = 0;
    }
  }
}

// One staged plane -> the per-point plane terms of the thread's 2 x 4 points:
// A = wf c + we f + wc g (the plane's contribution as an upper or lower
// neighbour plane) and B = w0 c + wf f + we g (as the centre plane), where c
// is the point, f the sum of its 4 in-plane face neighbours and g of its 4
// in-plane diagonal neighbours.  Row sums r[x-1] + r[x+1] are shared by the
// two output rows.
template <int BX, int BY>
JD void box27s_terms(const float (*st)[Box27S<BX, BY>::W], float w0, float wf, float we, float wc, float (&A)[2][4],
                     float (&B)[2][4]) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  float r[4][6];
#pragma unroll
  for (int k = 0; k < 4; ++k) lds_row<float, 4>(&st[2 * ty + k][4 + 4 * tx], r[k]);
  float s[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int e = 0; e < 4; ++e) s[k][e] = r[k][e] + r[k][e + 2];
#pragma unroll
  for (int yy = 0; yy < 2; ++yy)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float c = r[yy + 1][e + 1];
      const float f = s[yy + 1][e] + (r[yy][e + 1] + r[yy + 2][e + 1]);
      const float g = s[yy][e] + s[yy + 2][e];
      A[yy][e] = fmaf(wc, g, fmaf(we, f, wf * c));
      B[yy][e] = fmaf(we, g, fmaf(wf, f, w0 * c));
    }
}

// The staged periodic 27-point FP32 sweep of one CTA tile: planes z0-1 ..
// z1 are staged (L = z1 - z0 + 2), output plane z = A(z-1) + B(z) + A(z+1)
// is formed as P + A(z+1) with P = A(z-1) + B(z) kept in registers.  Returns
// the thread's double-float sum of its outputs (want_sum).
template <int BX, int BY, int ZC, class P>
JD double box27s_body(const float* __restrict__ u, float* __restrict__ v, const P& p, const JParams& rt,
                      bool want_sum) {
  typedef Box27S<BX, BY> G;
  __shared__ Box27SSmem<BX, BY> sm;
  const i64 nx = p.nx, ny = p.ny, nz = p.nz, sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const bool warp0 = tid < 32;
  const i64 bx0 = (i64)blockIdx.x * G::TW, by0 = (i64)blockIdx.y * G::TH;
  const i64 z0 = (i64)blockIdx.z * ZC;
  const i64 z1 = (z0 + ZC < nz) ? z0 + ZC : nz;
  const int L = (int)(z1 - z0) + 2;
  const int weff = (int)((nx - bx0 < G::TW) ? nx - bx0 : G::TW) + 8;
  const i64 lim = rt.timeout_ns;
  const bool stall_cta = rt.stall_plane >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < G::S; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], G::NW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  auto plane_z = [&](int j) {
    i64 z = (z0 - 1 + j) % nz;
    return z < 0 ? z + nz : z;
  };
  auto request = [&](int j, int s) {
    if (!(stall_cta && j == rt.stall_plane)) box27s_issue<BX, BY>(sm, s, u, p, plane_z(j), bx0, by0, weff);
  };
  int issued = 0, consumed = 0;  // warp 0: planes requested, planes waited for
  if (warp0)
    for (; issued < G::S && issued < L; ++issued) request(issued, issued);

  const float w0 = (float)p.c0, wf = (float)p.c1, we = (float)p.c2, wc = (float)p.c3;
  const i64 x0 = bx0 + 4 * tx, y0 = by0 + 2 * ty;
  const bool ax = x0 < nx, ay0 = ax && y0 < ny, ay1 = ax && y0 + 1 < ny;
  float* vo = v + y0 * nx + x0 + z0 * sz;
  float hi = 0.0f, lo = 0.0f;
  // ring cursors (stage, phase parity): cn the next plane to wait for, cq
  // the plane whose stage warp 0 refills next (one step behind)
  int cn_s = 0, cq_s = 0;
  u32 cn_ph = 0, cq_ph = 0;
  auto adv = [&](int& s, u32& ph) {
    if (++s == G::S) {
      s = 0;
      ph ^= 1u;
    }
  };
  // consume plane j: wait for it, form its terms, release its stage, and let
  // warp 0 refill the stage of plane j - 1
  auto consume = [&](int j, float (&A)[2][4], float (&B)[2][4]) -> bool {
    if (!mbar_wait(&sm.full[cn_s], cn_ph, lim)) return false;
    ++consumed;
    box27s_terms<BX, BY>(sm.st[cn_s], w0, wf, we, wc, A, B);
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&sm.empty[cn_s]);
    adv(cn_s, cn_ph);
    if (j >= 1) {
      if (warp0 && issued < L) {
        if (!mbar_wait(&sm.empty[cq_s], cq_ph, lim)) return false;
        request(issued, cq_s);
        ++issued;
      }
      adv(cq_s, cq_ph);
    }
    return true;
  };
  // output plane of staged plane j - 1 from P = A(j-2) + B(j-1) and the
  // terms of plane j; Anew receives A(j), Aold holds A(j-1)
  float Pz[2][4];
  auto step = [&](int j, float (&Anew)[2][4], const float (&Aold)[2][4]) -> bool {
    float B[2][4];
    if (!consume(j, Anew, B)) return false;
    float o[2][4];
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        o[yy][e] = Pz[yy][e] + Anew[yy][e];
        Pz[yy][e] = Aold[yy][e] + B[yy][e];
      }
    if (ay0) stv<float, 4>(vo, o[0]);
    if (ay1) stv<float, 4>(vo + nx, o[1]);
    vo += sz;
    if (want_sum) {
      const float t0 = ay0 ? (o[0][0] + o[0][1]) + (o[0][2] + o[0][3]) : 0.0f;
      const float t1 = ay1 ? (o[1][0] + o[1][1]) + (o[1][2] + o[1][3]) : 0.0f;
      two_sum_acc(hi, lo, t0 + t1);
    }
    return true;
  };
  float Aa[2][4], Ab[2][4];
  bool ok;
  {
    float B[2][4];
    ok = consume(0, Aa, B) && consume(1, Ab, B);  // A of planes 0 and 1; B of plane 1
    if (ok) {
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
#pragma unroll
        for (int e = 0; e < 4; ++e) Pz[yy][e] = Aa[yy][e] + B[yy][e];
    }
  }
  if (ok) {
    // two steps per iteration: the A buffers swap roles without copies
    int j = 2;
    for (; j + 1 < L; j += 2) {
      if (!step(j, Aa, Ab) || !step(j + 1, Ab, Aa)) {
        ok = false;
        break;
      }
    }
    if (ok && j < L) ok = step(j, Aa, Ab);
  }
  if (!ok) {
    if (rt.status) atomicExch(rt.status, JACC_DEV_TIMEOUT);
    if (warp0)
      for (int j = consumed; j < issued; ++j)
        if (!(stall_cta && j == rt.stall_plane)) mbar_wait(&sm.full[j % G::S], (u32)((j / G::S) & 1), lim);
  }
  return (double)hi + (double)lo;
}

// ---------------------------------------------------------------- 27-point periodic box, temporal blocking (FP32)
//
// TT sweeps per launch.  A CTA of 32 x RY threads (4 floats each in x) loads
// an input region of 128 x RY points per plane: an output tile of 120 x
// (RY - 2 TT) points plus a halo of 4 columns (16-byte alignment) and TT rows
// on each side.  Planes stream in z; stage t (1..TT) computes sweep t for the
// plane t steps behind the input, from the three newest planes of stage t-1,
// over the region shrunk by t (values beyond it are never used).  Each stage's
// newest plane sits in shared memory, one 16-byte vector per thread and row;
// x-neighbours come from warp shuffles (a warp is one region row).  Only the
// last stage's plane is written to memory, so HBM traffic is 8/TT bytes per
// point-sweep.
constexpr int TB_BX = 32, TB_V = 4, TB_RX = TB_BX * TB_V, TB_HX = 4, TB_OX = TB_RX - 2 * TB_HX;

template <int RY> struct alignas(16) TbPlane {
  float a[RY + 2][TB_RX + 8];  // row r + 1, column c + 4 holds region point (c, r)
};

template <int RY> JD void tb_cfe(const TbPlane<RY>& sm, float (&c)[4], float (&f)[4], float (&g)[4]) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  float r[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 t = *reinterpret_cast<const float4*>(&sm.a[ty + k][4 + tx * 4]);
    r[k][1] = t.x; r[k][2] = t.y; r[k][3] = t.z; r[k][4] = t.w;
    r[k][0] = __shfl_up_sync(0xffffffffu, t.w, 1);
    r[k][5] = __shfl_down_sync(0xffffffffu, t.x, 1);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    c[e] = r[1][e + 1];
    f[e] = (r[1][e] + r[1][e + 2]) + (r[0][e + 1] + r[2][e + 1]);
    g[e] = (r[0][e] + r[0][e + 2]) + (r[2][e] + r[2][e + 2]);
  }
}

template <int RY> JD void tb_put(TbPlane<RY>& sm, const float (&o)[4]) {
  float4 t;
  t.x = o[0]; t.y = o[1]; t.z = o[2]; t.w = o[3];
  *reinterpret_cast<float4*>(&sm.a[threadIdx.y + 1][4 + threadIdx.x * 4]) = t;
}

template <int RY, int TT, int ZC, class P>
JD void box27_tb_body(const float* __restrict__ u, float* __restrict__ v, const P& p, SumAcc<float>& acc,
                      bool want_sum, TbPlane<RY> (&sm)[TT]) {
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const i64 sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  constexpr int OY = RY - 2 * TT;
  const i64 ox0 = (i64)blockIdx.x * TB_OX;
  const i64 oy0 = (i64)blockIdx.y * OY;
  const i64 z0 = (i64)blockIdx.z * ZC;
  const i64 z1 = (z0 + ZC < nz) ? z0 + ZC : nz;
  // this thread's 4 region columns and region row, wrapped once
  const i64 gx = ((ox0 - TB_HX + (i64)tx * 4) % nx + nx) % nx;
  const i64 gy = ((oy0 - TT + ty) % ny + ny) % ny;
  const i64 own = gy * nx + gx;
  // output: threads 1..30 hold the tile's 120 columns, rows TT..RY-TT-1
  const i64 outx = ox0 + (i64)(tx - 1) * 4;
  const i64 outy = oy0 + ty - TT;
  const bool out_ok = tx >= 1 && tx <= TB_BX - 2 && ty >= TT && ty < RY - TT && outx < nx && outy < ny;
  const float w0 = (float)p.c0, wf = (float)p.c1, we = (float)p.c2, wc = (float)p.c3;

  float cm[TT][4], fm[TT][4], gm[TT][4], c0[TT][4], f0[TT][4], g0[TT][4];
#pragma unroll
  for (int t = 0; t < TT; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) cm[t][e] = fm[t][e] = gm[t][e] = c0[t][e] = f0[t][e] = g0[t][e] = 0.f;

  const i64 zs = z0 - TT;  // first input plane
  i64 zi = ((zs - 1) % nz + nz) % nz;
  const int nsteps = (int)(z1 - z0) + 2 * TT;
  float nxt[4];
  zi = (zi + 1 == nz) ? 0 : zi + 1;
  ldv<float, 4>(u + zi * sz + own, nxt);
  for (int j = 0; j < nsteps; ++j) {
    float cur_in[4] = {nxt[0], nxt[1], nxt[2], nxt[3]};
    if (j + 1 < nsteps) {  // prefetch the next input plane
      zi = (zi + 1 == nz) ? 0 : zi + 1;
      ldv<float, 4>(u + zi * sz + own, nxt);
    }
    tb_put<RY>(sm[0], cur_in);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      float cn[4], fn[4], gn[4], o[4];
      tb_cfe<RY>(sm[t], cn, fn, gn);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        o[e] = (w0 * c0[t][e] + wf * ((f0[t][e] + cm[t][e]) + cn[e])) +
               (we * ((g0[t][e] + fm[t][e]) + fn[e]) + wc * (gm[t][e] + gn[e]));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        cm[t][e] = c0[t][e]; fm[t][e] = f0[t][e]; gm[t][e] = g0[t][e];
        c0[t][e] = cn[e]; f0[t][e] = fn[e]; g0[t][e] = gn[e];
      }
      if (t + 1 < TT) {
        tb_put<RY>(sm[t + 1], o);
        __syncthreads();
      } else if (j >= 2 * TT && out_ok) {
        const i64 z = zs + j - TT;  // output plane, in [z0, z1)
        stv<float, 4>(v + z * sz + outy * nx + outx, o);
        if (want_sum) {
#pragma unroll
          for (int e = 0; e < 4; ++e) acc.add(o[e]);
        }
      }
    }
  }
}

template <int RY, int TT, int ZC, class P>
JD void box27_tb_entry(const float* __restrict__ u, float* __restrict__ v, const P& p, double* resid) {
  griddep_wait();
  __shared__ TbPlane<RY> sm[TT];
  SumAcc<float> acc;
  box27_tb_body<RY, TT, ZC>(u, v, p, acc, resid != nullptr, sm);
  block_sum_to<TB_BX * RY>(acc.total(), resid);
}

// ====================================================================== resident fixed point (FP64 data)
//
// Within one sweep sequence the field stays in 64-bit fixed point in the two
// HBM buffers (the same 8 bytes per value): the first sweep reads FP64 and
// converts, intermediate sweeps read and write the int64 values directly, and
// the last sweep writes the exact stencil value correctly rounded to FP64.
// Intermediate values are rounded once per sweep to the 2^-F grid (F >= 57 -
// e(M), finer than an FP64 ulp of M).  Dirichlet boundary points keep their
// FP64 bits in both buffers throughout (the first sweep copies them; later
// sweeps write back the bits they read), so they are converted where they
// are read as neighbours.
#define JFX_IN_F64 1   // the sweep's input interior holds FP64
#define JFX_OUT_F64 2  // the sweep writes FP64 (else int64 fixed point)

JD i64 bits_i64(double d) { return (i64)__double_as_longlong(d); }
JD double i64_bits(i64 q) { return __longlong_as_double(q); }

// Raw 8-byte word -> fixed-point value: convert (FP64 input) or reinterpret
// (resident fixed point).
JD i64 fx_in(double raw, bool conv, int F) { return conv ? fx_from(raw, F) : bits_i64(raw); }

// Round q * 2^-k to the nearest integer (ties up), k in [0, 62].
JD i64 fx_round_shift(i64 q, int k) { return k ? ((q + ((i64)1 << (k - 1))) >> k) : q; }

// (x + 2^(k-1)) >> k for a 128-bit x whose result fits in int64, k in [0, 62].
JD i64 fx128_round_shift(s128 x, int k) {
  if (k == 0) return (i64)x.lo;
  s128 h;
  h.lo = (u64)1 << (k - 1);
  h.hi = 0;
  x = add128(x, h);
  return (i64)((x.lo >> k) | (x.hi << (64 - k)));
}

// Per-thread column facts of a tile: which of the thread's V columns are
// interior (bit set) and which are boundary columns (x == 0 or nx-1).
template <int V> JD void col_masks(i64 x0, i64 nx, unsigned& intm, unsigned& bndm) {
  intm = 0;
  bndm = 0;
#pragma unroll
  for (int e = 0; e < V; ++e) {
    const i64 x = x0 + e;
    if (x >= 1 && x <= nx - 2) intm |= 1u << e;
    if (x == 0 || x == nx - 1) bndm |= 1u << e;
  }
}

// ---------------------------------------------------------------- 5-point Jacobi, resident fixed point
//
// Same march as jacobi_march.  v 2^F = (S + 2) >> 2 with S the four
// neighbours (exact); the FP64 output is fx_to(S, F + 2).  Residual: max
// |S - 4u| (scale F, converted once per thread by the caller).  EDGE as for
// the 7-point kernel: intermediate sweeps (EDGE = false) convert nothing.
template <int V, bool CG, bool EDGE>
JD void jacobi_fx_march(const double* __restrict__ u, double* __restrict__ v, i64 nx, i64 ny, i64 x0, i64 ys, i64 ye,
                        int F, int flags, u64& rmax) {
  const int lane = threadIdx.x & 31;
  const bool xin = x0 < nx;
  const bool inf = EDGE && (flags & JFX_IN_F64);
  const bool outf = EDGE && (flags & JFX_OUT_F64);
  unsigned intm, bndm;
  col_masks<V>(x0, nx, intm, bndm);
  auto cvt = [&](double raw) -> i64 { return (EDGE && inf) ? fx_from(raw, F) : bits_i64(raw); };
  auto bnd_out = [&](double raw, i64 w) -> double {
    if constexpr (!EDGE) return i64_bits(w);
    if (inf && outf) return raw;
    if (outf) return fx_to(w, F);
    return i64_bits(w);
  };
  double rup[V], rcur[V], rdn[V], rnx[V];
  i64 up[V], cur[V], dn[V];
#pragma unroll
  for (int e = 0; e < V; ++e) rup[e] = rcur[e] = rdn[e] = rnx[e] = 0.0;
  if (xin) {
    if (ys >= 1) ldv<double, V, CG>(u + (ys - 1) * nx + x0, rup);
    ldv<double, V, CG>(u + ys * nx + x0, rcur);
    if (ys + 1 < ny) ldv<double, V, CG>(u + (ys + 1) * nx + x0, rdn);
    if (ys + 2 < ny) ldv<double, V, CG>(u + (ys + 2) * nx + x0, rnx);
  }
#pragma unroll
  for (int e = 0; e < V; ++e) {
    up[e] = cvt(rup[e]);
    cur[e] = cvt(rcur[e]);
    dn[e] = cvt(rdn[e]);
  }
  for (i64 y = ys; y < ye; ++y) {
    i64 left = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
    i64 right = __shfl_down_sync(0xffffffffu, cur[0], 1);
    if (lane == 0 && xin && x0 >= 1) left = cvt(ld1<CG>(u + y * nx + x0 - 1));
    if (lane == 31 && xin && x0 + V < nx) right = cvt(ld1<CG>(u + y * nx + x0 + V));
    double rnn[V];
#pragma unroll
    for (int e = 0; e < V; ++e) rnn[e] = 0.0;
    if (xin && y + 3 < ny) ldv<double, V, CG>(u + (y + 3) * nx + x0, rnn);
    const bool yint = (y >= 1) && (y <= ny - 2);
    double out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const i64 xl = (e == 0) ? left : cur[e - 1];
      const i64 xr = (e == V - 1) ? right : cur[e + 1];
      const bool in = yint && ((intm >> e) & 1u);
      const i64 s = (up[e] + dn[e]) + (xl + xr);
      const double o = outf ? fx_to(s, F + 2) : i64_bits((s + 2) >> 2);
      out[e] = in ? o : bnd_out(rcur[e], cur[e]);
      const i64 d = s - cur[e] * 4;
      const u64 ad = (u64)(d ^ (d >> 63));  // |d| (one less for negative d: below the tolerance by 2^-F)
      if (in && ad > rmax) rmax = ad;
    }
    if (xin) stv<double, V>(v + y * nx + x0, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      up[e] = cur[e];
      cur[e] = dn[e];
      rcur[e] = rdn[e];
      rdn[e] = rnx[e];
      dn[e] = cvt(rnx[e]);
      rnx[e] = rnn[e];
    }
  }
}

// ---------------------------------------------------------------- 5-point Jacobi, prefetching march
//
// The march of jacobi_march / jacobi_fx_march with loads issued PD rows
// ahead: a register ring holds the raw rows y+2 .. y+PD+1 in flight, and the
// x-edge values of lanes 0 and 31 (one column left of the warp's chunk for
// lane 0, one right for lane 31) for rows y+1 .. y+PD-1, so no load is
// consumed in the iteration that issues it.  The ring is indexed with
// compile-time slots (the row loop is unrolled by PD).  Rows past ye (the
// march end) are not prefetched beyond the one halo row the last step needs.
// FX: resident 64-bit fixed point (EDGE as for jacobi_fx_march); otherwise
// native arithmetic on T.
template <class T, int V, bool CG, bool FX, bool EDGE, int PD>
JD void jacobi_march_pf(const T* __restrict__ u, T* __restrict__ v, i64 nx, i64 ny, i64 x0, i64 ys, i64 ye, int F,
                        int flags, typename RT<T, FX ? JM_FIXED : JM_NATIVE>::type& rmax) {
  typedef typename WT<T, FX ? JM_FIXED : JM_NATIVE>::type W;
  const int lane = threadIdx.x & 31;
  const bool xin = x0 < nx;
  const bool inf = FX && EDGE && (flags & JFX_IN_F64);
  const bool outf = FX && EDGE && (flags & JFX_OUT_F64);
  // this lane's x-edge column (lane 0: x0 - 1, lane 31: x0 + V), if any
  const bool has_edge = xin && ((lane == 0 && x0 >= 1) || (lane == 31 && x0 + V < nx));
  const T* ecol = u + (lane == 0 ? x0 - 1 : x0 + V);
  const T* col = u + x0;
  auto cvt = [&](T raw) -> W {
    if constexpr (FX) return inf ? fx_from(raw, F) : bits_i64(raw);
    else return raw;
  };
  auto bnd_out = [&](T raw, W w) -> T {
    if constexpr (FX) {
      if constexpr (!EDGE) return i64_bits(w);
      if (inf && outf) return raw;
      if (outf) return fx_to(w, F);
      return i64_bits(w);
    } else {
      return raw;
    }
  };
  unsigned intm, bndm;
  col_masks<V>(x0, nx, intm, bndm);
  T ring[PD][V];  // slot j % PD: raw row ys + 1 + j (the "down" row of step j)
  T eg[PD];       // slot j % PD: this lane's x-edge value of row ys + j
  T rcur[V];
  W up[V], cur[V];
  {
    T t[V];
#pragma unroll
    for (int e = 0; e < V; ++e) t[e] = rcur[e] = T(0);
    if (xin) {
      if (ys >= 1) ldv<T, V, CG>(col + (ys - 1) * nx, t);
      ldv<T, V, CG>(col + ys * nx, rcur);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      up[e] = cvt(t[e]);
      cur[e] = cvt(rcur[e]);
    }
#pragma unroll
    for (int k = 0; k < PD; ++k) {
      const i64 r = ys + 1 + k;
#pragma unroll
      for (int e = 0; e < V; ++e) ring[k][e] = T(0);
      if (xin && r <= ye && r < ny) ldv<T, V, CG>(col + r * nx, ring[k]);
      eg[k] = T(0);
      if (has_edge && ys + k < ye) eg[k] = ld1<CG>(ecol + (ys + k) * nx);
    }
  }
  const i64 n = ye - ys;
  for (i64 j0 = 0; j0 < n; j0 += PD) {
#pragma unroll
    for (int i = 0; i < PD; ++i) {
      const i64 j = j0 + i;
      if (j >= n) break;
      const i64 y = ys + j;
      // consume slot i: the down row and this lane's edge of row y; refill it
      T rdn[V];
#pragma unroll
      for (int e = 0; e < V; ++e) rdn[e] = ring[i][e];
      const T edge = eg[i];
      {
        const i64 r = y + 1 + PD;
#pragma unroll
        for (int e = 0; e < V; ++e) ring[i][e] = T(0);
        if (xin && r <= ye && r < ny) ldv<T, V, CG>(col + r * nx, ring[i]);
        if (has_edge && y + PD < ye) eg[i] = ld1<CG>(ecol + (y + PD) * nx);
      }
      W dn[V];
#pragma unroll
      for (int e = 0; e < V; ++e) dn[e] = cvt(rdn[e]);
      W left = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
      W right = __shfl_down_sync(0xffffffffu, cur[0], 1);
      if (has_edge) {
        if (lane == 0) left = cvt(edge);
        else right = cvt(edge);
      }
      const bool yint = (y >= 1) && (y <= ny - 2);
      T out[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const W xl = (e == 0) ? left : cur[e - 1];
        const W xr = (e == V - 1) ? right : cur[e + 1];
        const bool in = yint && ((intm >> e) & 1u);
        if constexpr (FX) {
          const i64 s = (up[e] + dn[e]) + (xl + xr);
          const T o = outf ? fx_to(s, F + 2) : i64_bits((s + 2) >> 2);
          out[e] = in ? o : bnd_out(rcur[e], cur[e]);
          const i64 d = s - cur[e] * 4;
          const u64 ad = (u64)(d ^ (d >> 63));  // |d| (one less for negative d: below the tolerance by 2^-F)
          rmax = (in && ad > rmax) ? ad : rmax;
        } else {
          const T s = (up[e] + dn[e]) + (xl + xr);
          const T r = T(0.25) * s;
          out[e] = in ? r : rcur[e];
          T d = r - rcur[e];
          d = d < T(0) ? -d : d;
          rmax = (in && d > rmax) ? d : rmax;
        }
      }
      if (xin) stv<T, V>(v + y * nx + x0, out);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        up[e] = cur[e];
        cur[e] = dn[e];
        rcur[e] = rdn[e];
      }
    }
  }
}

// ---------------------------------------------------------------- 7-point heat, resident fixed point
//
// S = the six faces, L = S - 6u (exact, scale F):
//   JACC_FP_SMALL (r = fb 2^-k): v = u + round(fb L 2^-k)      (int64)
//   JACC_FP_WIDE  (r = m 2^-k):  v = u + round(m L 2^-k)       (128-bit product)
// FP64 output: u + r L correctly rounded.  The residual only needs max |L|.
//
// EDGE = false: an intermediate sweep.  Every value in both buffers, the
// Dirichlet boundary included, is already in fixed point, so the kernel does
// no conversion at all.  EDGE = true: the first and/or last sweep of a
// sequence (flags JFX_IN_F64 / JFX_OUT_F64): loads convert from FP64, stores
// convert to FP64, boundary points are converted (or copied when both).
template <bool EDGE, int BX, int BY, int V, int ZC, class P>
JD void heat3d_fx_body(const double* __restrict__ u, double* __restrict__ v, const P& p, int F, int flags, u64& rmax,
                       Plane<i64, BX, BY, V>& sm) {
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const i64 sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 bx0 = (i64)blockIdx.x * (BX * V);
  const i64 by0 = (i64)blockIdx.y * BY;
  const i64 x0 = bx0 + (i64)tx * V;
  const i64 y = by0 + ty;
  const bool act = (x0 < nx) && (y < ny);
  const i64 cz0 = (i64)blockIdx.z * ZC;
  const i64 cz1 = (cz0 + ZC < nz) ? cz0 + ZC : nz;
  const bool inf = EDGE && (flags & JFX_IN_F64);
  const bool outf = EDGE && (flags & JFX_OUT_F64);
  const double* urow = u + y * nx + x0;
  double* vrow = v + y * nx + x0;
  // boundary point written by this sweep, from its input word
  auto bnd_out = [&](double raw, i64 w) -> double {
    if constexpr (!EDGE) return i64_bits(w);    // fixed in, fixed out (raw holds the same bits)
    if (inf && outf) return raw;                // FP64 in, FP64 out: copy
    if (outf) return fx_to(w, F);               // fixed in, FP64 out
    return i64_bits(w);                         // FP64 in, fixed out
  };
  auto cvt = [&](double raw) -> i64 { return (EDGE && inf) ? fx_from(raw, F) : bits_i64(raw); };

  // Boundary planes are written by the chunk that holds them.
  if (act && (cz0 == 0 || cz1 == nz)) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if ((side == 0 && cz0 == 0) || (side == 1 && cz1 == nz)) {
        const i64 off = side ? (nz - 1) * sz : 0;
        double t[V];
        ldv<double, V>(urow + off, t);
#pragma unroll
        for (int e = 0; e < V; ++e) t[e] = bnd_out(t[e], cvt(t[e]));
        stv<double, V>(vrow + off, t);
      }
    }
  }
  const i64 z0 = cz0 < 1 ? 1 : cz0;
  const i64 z1 = cz1 > nz - 1 ? nz - 1 : cz1;
  if (z0 >= z1) return;  // block-uniform

  unsigned intm, bndm;
  col_masks<V>(x0, nx, intm, bndm);
  const bool rowb = (y == 0) || (y == ny - 1);
  const bool yint = act && !rowb;
  // halo sources of this thread (fixed per CTA and thread)
  const bool has_top = (ty == 0) && (by0 >= 1) && (x0 < nx);
  const bool has_bot = (ty == BY - 1) && (by0 + BY < ny) && (x0 < nx);
  const double* hyp = u + (has_top ? by0 - 1 : by0 + BY) * nx + x0;
  const bool has_xl = (tx == 0) && (bx0 >= 1) && (y < ny);
  const bool has_xr = (tx == BX - 1) && (bx0 + BX * V < nx) && (y < ny);
  const double* hxp = u + y * nx + (has_xl ? bx0 - 1 : bx0 + BX * V);

  double rcur[V], rzn[V], rzn2[V], hy[V], hyn[V];
  double hx = 0.0, hxn = 0.0;
  i64 zp[V], cur[V], zn[V];
  {
    double t[V];
#pragma unroll
    for (int e = 0; e < V; ++e) t[e] = rcur[e] = rzn[e] = rzn2[e] = hy[e] = hyn[e] = 0.0;
    if (act) {
      ldv<double, V>(urow + (z0 - 1) * sz, t);
      ldv<double, V>(urow + z0 * sz, rcur);
      ldv<double, V>(urow + (z0 + 1) * sz, rzn);
      if (z0 + 2 < nz) ldv<double, V>(urow + (z0 + 2) * sz, rzn2);
    }
    if (has_top || has_bot) ldv<double, V>(hyp + z0 * sz, hy);
    if (has_xl || has_xr) hx = __ldg(hxp + z0 * sz);
#pragma unroll
    for (int e = 0; e < V; ++e) { zp[e] = cvt(t[e]); cur[e] = cvt(rcur[e]); }
  }
  const i64 fb = p.fb, fw0 = p.fw0;
  const int k = p.fk;
  const bool small = p.fpath == JACC_FP_SMALL;
  int b = 0;
  i64 zoff = z0 * sz;
  for (i64 z = z0; z < z1; ++z, zoff += sz) {
#pragma unroll
    for (int e = 0; e < V; ++e) zn[e] = cvt(rzn[e]);
    // loads one plane ahead: own plane z+3, halo of plane z+1
    double rn3[V];
#pragma unroll
    for (int e = 0; e < V; ++e) rn3[e] = 0.0;
    if (act && z + 3 < nz) ldv<double, V>(urow + zoff + 3 * sz, rn3);
    if (z + 1 < z1) {
      if (has_top || has_bot) ldv<double, V>(hyp + zoff + sz, hyn);
      if (has_xl || has_xr) hxn = __ldg(hxp + zoff + sz);
    }
    // this plane into shared memory
    i64* row = &sm.a[b][ty + 1][V + tx * V];
#pragma unroll
    for (int e = 0; e < V; ++e) row[e] = cur[e];
    if (has_top || has_bot) {
      i64* hr = &sm.a[b][has_top ? 0 : BY + 1][V + tx * V];
#pragma unroll
      for (int e = 0; e < V; ++e) hr[e] = cvt(hy[e]);
    }
    if (has_xl) sm.a[b][ty + 1][V - 1] = cvt(hx);
    if (has_xr) sm.a[b][ty + 1][V + BX * V] = cvt(hx);
    __syncthreads();
    const i64* rm = &sm.a[b][ty][V + tx * V];
    const i64* r0 = &sm.a[b][ty + 1][V + tx * V];
    const i64* rp = &sm.a[b][ty + 2][V + tx * V];
    double out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const bool in = yint && ((intm >> e) & 1u);
      const i64 xl = (e == 0) ? r0[-1] : cur[e - 1];
      const i64 xr = (e == V - 1) ? r0[V] : cur[e + 1];
      const i64 sum = ((xl + xr) + (rm[e] + rp[e])) + (zp[e] + zn[e]);
      const i64 L = sum - 6 * cur[e];
      // the increment v - c in fixed point: v = c + round(r L)
      const i64 dv = small ? fx_round_shift(fb * L, k) : fx128_round_shift(mul_s64_u64(L, (u64)fw0), k);
      double o;
      if (outf) {
        if (small) o = fx_to(cur[e] * ((i64)1 << k) + fb * L, F + k);
        else o = fx128_to(add128(from_s64_shl(cur[e], k), mul_s64_u64(L, (u64)fw0)), F + k);
      } else {
        o = i64_bits(cur[e] + dv);
      }
      out[e] = in ? o : bnd_out(rcur[e], cur[e]);
      const u64 aL = (u64)(dv ^ (dv >> 63));  // |v - c| (one less for negative: 2^-F, below the tolerance)
      rmax = (in && aL > rmax) ? aL : rmax;
    }
    if (act) stv<double, V>(vrow + zoff, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      zp[e] = cur[e];
      cur[e] = zn[e];
      rcur[e] = rzn[e];
      rzn[e] = rzn2[e];
      rzn2[e] = rn3[e];
      hy[e] = hyn[e];
    }
    hx = hxn;
    b ^= 1;
  }
}

// Residual of the heat sweep from max |L|: r max|L| scaled.

// ---------------------------------------------------------------- 7-point heat, bulk-copy staged planes
//
// Same staging as the 27-point kernel (bulk copies on full/empty mbarriers,
// bounded waits), Dirichlet geometry: a thread owns one 16-byte column (V
// values) of 2 rows; a stage holds rows by0-1 .. by0+TH and columns
// bx0-V .. bx0+TW+V-1 of one plane, clipped to the grid (points outside are
// never needed: only interior points read neighbours).  Planes z0-1 .. z1 are
// staged; a thread keeps its own values of planes z-1 and z in registers,
// reads its own values of plane z+1 and the in-plane neighbours of plane z
// (rows y-1 and y+2, the columns left and right of its own) from the stage.
// The boundary planes z = 0 and nz-1 are written from the staged values.
//
// FX: FP64 storage in the resident 64-bit fixed point (EDGE: the first/last
// sweep converts on load/store); otherwise native arithmetic on T.
template <class T, int BX, int BY, int SC> struct Heat3S {
  static constexpr int V = 16 / (int)sizeof(T);
  static constexpr int RY = 2;
  static constexpr int TW = BX * V, TH = BY * RY;
  static constexpr int W = TW + 2 * V, R = TH + 2;
  static constexpr int STAGE_BYTES = W * R * (int)sizeof(T);
  static constexpr int S0 = 45056 / STAGE_BYTES;
  // stages: at most ~44 KB and SC (512^3 with 32 x 4 threads, 5.4 KB
  // stages: FP32 656 GLUP/s with 4 stages, 710 with 5, 713 with 6; FP64
  // precompiled 327.5 with 6, 295.6 with 5); larger tiles' stages fit fewer
  static constexpr int SMAX = SC;
  static constexpr int S = S0 < 2 ? 2 : (S0 > SMAX ? SMAX : S0);
  // A step needs planes z and z+1 staged.  With S >= 3 warp 0 refills the
  // stage released one step earlier (slack for lagging warps); with S = 2 it
  // refills the stage just released, and no plane is prefetched.
  static constexpr int D = S >= 3 ? 1 : 0;
  static constexpr int NW = BX * BY / 32;
};

template <class T, int BX, int BY, int SC> struct alignas(128) Heat3SSmem {
  T st[Heat3S<T, BX, BY, SC>::S][Heat3S<T, BX, BY, SC>::R][Heat3S<T, BX, BY, SC>::W];
  u64 full[Heat3S<T, BX, BY, SC>::S];
  u64 empty[Heat3S<T, BX, BY, SC>::S];
};

// Warp 0 requests plane zg into stage s: one bulk copy per staged row inside
// the grid; lane 0 first posts the byte count of the whole plane.
template <class T, int BX, int BY, int SC, class P>
JD void heat3s_issue(Heat3SSmem<T, BX, BY, SC>& sm, int s, const T* __restrict__ u, const P& p, i64 zg, i64 bx0,
                     i64 by0) {
  typedef Heat3S<T, BX, BY, SC> G;
  const i64 nx = p.nx, ny = p.ny;
  const int lane = threadIdx.x & 31;
  const i64 c0 = bx0 - G::V < 0 ? 0 : bx0 - G::V;
  const i64 c1 = bx0 + G::TW + G::V > nx ? nx : bx0 + G::TW + G::V;
  const i64 r0 = by0 - 1 < 0 ? 0 : by0 - 1;
  const i64 r1 = by0 + G::TH + 1 > ny ? ny : by0 + G::TH + 1;
  const u32 row_bytes = (u32)((c1 - c0) * (i64)sizeof(T));
  if (lane == 0) mbar_expect_tx(&sm.full[s], row_bytes * (u32)(r1 - r0));
  __syncwarp();
  for (i64 y = r0 + lane; y < r1; y += 32)
    bulk_g2s(&sm.st[s][y - (by0 - 1)][c0 - (bx0 - G::V)], u + (zg * ny + y) * nx + c0, row_bytes, &sm.full[s]);
}

// 16-byte shared-memory vector reads (bit patterns kept).
JD void lds_vec(const void* p, float (&r)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
}
JD void lds_vec(const void* p, double (&r)[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  r[0] = t.x; r[1] = t.y;
}
JD void lds_vec(const void* p, i64 (&r)[2]) {
  const longlong2 t = *reinterpret_cast<const longlong2*>(p);
  r[0] = t.x; r[1] = t.y;
}

template <class A, class B> struct SameT { static constexpr bool value = false; };
template <class A> struct SameT<A, A> { static constexpr bool value = true; };

template <class T, bool FX> struct HeatAcc { typedef T type; };
template <> struct HeatAcc<double, true> { typedef u64 type; };

template <class T, int BX, int BY, int ZC, bool FX, bool EDGE, int SC, class P>
JD void heat3s_body(const T* __restrict__ u, T* __restrict__ v, const P& p, const JParams& rt, int F, int flags,
                    typename HeatAcc<T, FX>::type& rmax, Heat3SSmem<T, BX, BY, SC>& sm) {
  typedef Heat3S<T, BX, BY, SC> G;
  constexpr int V = G::V;
  typedef typename WT<T, FX ? JM_FIXED : JM_NATIVE>::type Wt;  // working type: i64 (fixed) or T
  const i64 nx = p.nx, ny = p.ny, nz = p.nz, sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const bool warp0 = tid < 32;
  const i64 bx0 = (i64)blockIdx.x * G::TW, by0 = (i64)blockIdx.y * G::TH;
  const i64 x0 = bx0 + (i64)tx * V, y0 = by0 + 2 * ty;
  const bool ax = x0 < nx;
  const bool ay[2] = {ax && y0 < ny, ax && y0 + 1 < ny};
  // interior mask of the thread's 2 x V points: bit yy * V + e
  unsigned inm = 0;
#pragma unroll
  for (int yy = 0; yy < 2; ++yy)
#pragma unroll
    for (int e = 0; e < V; ++e)
      if (y0 + yy >= 1 && y0 + yy <= ny - 2 && x0 + e >= 1 && x0 + e <= nx - 2) inm |= 1u << (yy * V + e);
  const i64 cz0 = (i64)blockIdx.z * ZC;
  const i64 cz1 = (cz0 + ZC < nz) ? cz0 + ZC : nz;
  const i64 z0 = cz0 < 1 ? 1 : cz0;
  const i64 z1 = cz1 > nz - 1 ? nz - 1 : cz1;
  const bool inf = FX && EDGE && (flags & JFX_IN_F64);
  const bool outf = FX && EDGE && (flags & JFX_OUT_F64);
  // raw input word -> working value, working value -> output word, and a
  // boundary point's output word from its raw input word
  auto cvt = [&](T raw) -> Wt {
    if constexpr (FX) return inf ? fx_from(raw, F) : bits_i64(raw);
    else return raw;
  };
  auto as_out = [&](Wt w) -> T {
    if constexpr (FX) return i64_bits(w);
    else return w;
  };
  auto bnd_out = [&](T raw) -> T {
    if constexpr (FX && EDGE) {
      if (inf == outf) return raw;
      if (outf) return fx_to(bits_i64(raw), F);
      return i64_bits(fx_from(raw, F));
    } else {
      return raw;
    }
  };
  if (z0 >= z1) {  // a chunk holding only a boundary plane (block-uniform)
    for (i64 z = cz0; z < cz1; ++z)
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
        if (ay[yy]) {
          T t[V];
          ldv<T, V>(u + z * sz + (y0 + yy) * nx + x0, t);
#pragma unroll
          for (int e = 0; e < V; ++e) t[e] = bnd_out(t[e]);
          stv<T, V>(v + z * sz + (y0 + yy) * nx + x0, t);
        }
    return;
  }
  const int L = (int)(z1 - z0) + 2;  // staged planes z0-1 .. z1
  const i64 lim = rt.timeout_ns;
  const bool stall_cta = rt.stall_plane >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < G::S; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], G::NW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  auto request = [&](int j, int s) {
    if (!(stall_cta && j == rt.stall_plane)) heat3s_issue<T, BX, BY, SC>(sm, s, u, p, z0 - 1 + j, bx0, by0);
  };
  int issued = 0, consumed = 0;  // warp 0: planes requested, planes waited for
  if (warp0)
    for (; issued < G::S && issued < L; ++issued) request(issued, issued);
  // ring cursors (stage, phase parity): cn the next plane to wait for, cq the
  // plane whose stage warp 0 refills next
  int cn_s = 0, cq_s = 0;
  u32 cn_ph = 0, cq_ph = 0;
  auto adv = [&](int& s, u32& ph) {
    if (++s == G::S) {
      s = 0;
      ph ^= 1u;
    }
  };
  auto wait_next = [&]() -> bool {
    if (!mbar_wait(&sm.full[cn_s], cn_ph, lim)) return false;
    ++consumed;
    return true;
  };
  // this warp has read the plane in stage s for the last time (plane j);
  // warp 0 then refills the stage of plane j - D once every warp released it
  auto release = [&](int j, int s) -> bool {
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&sm.empty[s]);
    if (j >= G::D) {
      if (warp0 && issued < L) {
        if (!mbar_wait(&sm.empty[cq_s], cq_ph, lim)) return false;
        request(issued, cq_s);
        ++issued;
      }
      adv(cq_s, cq_ph);
    }
    return true;
  };
  auto own = [&](int s, T (&raw)[2][V]) {
#pragma unroll
    for (int yy = 0; yy < 2; ++yy) lds_vec(&sm.st[s][2 * ty + 1 + yy][V + V * tx], raw[yy]);
  };
  auto store_bnd = [&](T* dst, const T (&raw)[2][V], const Wt (&w)[2][V]) {
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
      if (ay[yy]) {
        T t[V];
#pragma unroll
        for (int e = 0; e < V; ++e) t[e] = (FX && EDGE) ? bnd_out(raw[yy][e]) : as_out(w[yy][e]);
        stv<T, V>(dst + yy * nx, t);
      }
  };
  constexpr bool RAW = FX && EDGE;  // raw words of plane z kept (converting sweeps only)
  T rcur[2][V];
  Wt wa[2][V], wb[2][V], wc[2][V];  // own values of planes z-1, z, z+1 (rotating roles)
  T* vo = v + y0 * nx + x0;
  bool ok = wait_next();
  if (ok) {  // plane z0-1
    T r0[2][V];
    own(cn_s, r0);
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int e = 0; e < V; ++e) wa[yy][e] = cvt(r0[yy][e]);
    if (cz0 == 0) store_bnd(vo, r0, wa);  // boundary plane 0
    const int s0 = cn_s;
    adv(cn_s, cn_ph);
    ok = release(0, s0) && wait_next();
  }
  int cc_s = cn_s;  // stage of the centre plane z
  if (ok) {  // plane z0
    own(cn_s, rcur);
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int e = 0; e < V; ++e) wb[yy][e] = cvt(rcur[yy][e]);
    adv(cn_s, cn_ph);
  }
  const T r = (T)p.c0;
  const i64 fb = p.fb, fw0 = p.fw0;
  const int k = p.fk;
  const bool small = p.fpath == JACC_FP_SMALL;
  const bool fold = heat_fold(p);
  constexpr bool folded = !SameT<P, JParams>::value;  // extents and coefficients are constants
  vo += z0 * sz;
  // one output plane (staged plane j, 1 <= j <= L-2) from the own values of
  // planes j-1 (zp) and j (cur); fills zn with those of plane j+1
  auto step = [&](int j, const Wt (&zp)[2][V], const Wt (&cur)[2][V], Wt (&zn)[2][V]) -> bool {
    if (!wait_next()) return false;
    T rzn[2][V];
    own(cn_s, rzn);
    const Wt(*pl)[G::W] = reinterpret_cast<const Wt(*)[G::W]>(sm.st[cc_s]);
    Wt ym[V], yp[V], xl[2], xr[2];
    lds_vec(&pl[2 * ty][V + V * tx], ym);
    lds_vec(&pl[2 * ty + 3][V + V * tx], yp);
#pragma unroll
    for (int yy = 0; yy < 2; ++yy) {
      xl[yy] = pl[2 * ty + 1 + yy][V + V * tx - 1];
      xr[yy] = pl[2 * ty + 1 + yy][V + V * tx + V];
    }
    if constexpr (FX && EDGE) {
      if (inf) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
          ym[e] = fx_from(i64_bits(ym[e]), F);
          yp[e] = fx_from(i64_bits(yp[e]), F);
        }
#pragma unroll
        for (int yy = 0; yy < 2; ++yy) {
          xl[yy] = fx_from(i64_bits(xl[yy]), F);
          xr[yy] = fx_from(i64_bits(xr[yy]), F);
        }
      }
    }
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int e = 0; e < V; ++e) zn[yy][e] = cvt(rzn[yy][e]);
#pragma unroll
    for (int yy = 0; yy < 2; ++yy) {
      T out[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const bool in = (inm >> (yy * V + e)) & 1u;
        const Wt a = (e == 0) ? xl[yy] : cur[yy][e - 1];
        const Wt b = (e == V - 1) ? xr[yy] : cur[yy][e + 1];
        const Wt c = yy == 0 ? ym[e] : cur[0][e];
        const Wt d = yy == 0 ? cur[1][e] : yp[e];
        const Wt sum = ((a + b) + (c + d)) + (zp[yy][e] + zn[yy][e]);
        const Wt ce = cur[yy][e];
        if constexpr (FX) {
          double o;
          i64 dv;  // the increment v - c in fixed point: v = c + round(r L)
          if (folded && fold) {
            const i64 vn = (fb * sum + ((((i64)1 << k) - 6 * fb) * ce + ((i64)1 << (k - 1)))) >> k;
            dv = vn - ce;
            o = outf ? fx_to(ce * ((i64)1 << k) + fb * (sum - 6 * ce), F + k) : i64_bits(vn);
          } else {
            const i64 Ld = sum - 6 * ce;
            if (small) dv = fx_round_shift(fb * Ld, k);
            else dv = fx128_round_shift(mul_s64_u64(Ld, (u64)fw0), k);
            if (outf) {
              if (small) o = fx_to(ce * ((i64)1 << k) + fb * Ld, F + k);
              else o = fx128_to(add128(from_s64_shl(ce, k), mul_s64_u64(Ld, (u64)fw0)), F + k);
            } else {
              o = i64_bits(ce + dv);
            }
          }
          const u64 aL = (u64)(dv ^ (dv >> 63));  // |v - c| (one less if negative)
          if constexpr (RAW) out[e] = in ? o : bnd_out(rcur[yy][e]);
          else out[e] = in ? o : as_out(ce);
          rmax = (in && aL > rmax) ? aL : rmax;
        } else {
          const T o = ce + r * (sum - T(6) * ce);
          out[e] = in ? o : ce;
          T dd = o - ce;
          dd = dd < T(0) ? -dd : dd;
          rmax = (in && dd > rmax) ? dd : rmax;
        }
      }
      if (ay[yy]) stv<T, V>(vo + yy * nx, out);
    }
    vo += sz;
    if (j == L - 2 && cz1 == nz) store_bnd(vo, rzn, zn);  // boundary plane nz-1 = staged plane L-1
    if (!release(j, cc_s)) return false;
    cc_s = cn_s;
    adv(cn_s, cn_ph);
    if constexpr (RAW) {
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
#pragma unroll
        for (int e = 0; e < V; ++e) rcur[yy][e] = rzn[yy][e];
    }
    return true;
  };
  if (ok) {
    // three steps per iteration: the buffers' roles rotate without copies
    int j = 1;
    for (; j + 2 <= L - 2; j += 3) {
      if (!step(j, wa, wb, wc) || !step(j + 1, wb, wc, wa) || !step(j + 2, wc, wa, wb)) {
        ok = false;
        break;
      }
    }
    if (ok && j <= L - 2) ok = step(j, wa, wb, wc);
    if (ok && j + 1 <= L - 2) ok = step(j + 1, wb, wc, wa);
  }
  if (!ok) {
    if (rt.status) atomicExch(rt.status, JACC_DEV_TIMEOUT);
    if (warp0)
      for (int j = consumed; j < issued; ++j)
        if (!(stall_cta && j == rt.stall_plane)) mbar_wait(&sm.full[j % G::S], (u32)((j / G::S) & 1), lim);
  }
}

// ---------------------------------------------------------------- 27-point box, resident fixed point
//
// v 2^F = round(sum_j fw_j class_j 2^-K) from the exact 128-bit sum; the FP64
// output is the 128-bit sum correctly rounded.  Periodic: no boundary, every
// point is updated.  The field sum accumulates the fixed outputs exactly in
// 128 bits per thread.
template <int BX, int BY, int V>
JD void fx_plane_load_put(const double* __restrict__ u, i64 nx, i64 ny, i64 nz, i64 z, i64 bx0, i64 by0,
                          const double* urow, Plane<i64, BX, BY, V>& sm, int b, int F, bool inf) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 zz = (z % nz + nz) % nz;
  const double* pl = u + zz * nx * ny;
  double r[V];
  ldv<double, V>(urow + zz * nx * ny, r);
  i64 w[V];
#pragma unroll
  for (int e = 0; e < V; ++e) w[e] = inf ? fx_from(r[e], F) : bits_i64(r[e]);
  i64* row = &sm.a[b][ty + 1][V + tx * V];
#pragma unroll
  for (int e = 0; e < V; ++e) row[e] = w[e];
  const i64 x0 = (bx0 + (i64)tx * V) % nx;
  if (ty == 0 || ty == BY - 1) {
    const i64 yy = ty == 0 ? (by0 - 1 + ny) % ny : (by0 + BY) % ny;
    double h[V];
    ldv<double, V>(pl + yy * nx + x0, h);
#pragma unroll
    for (int e = 0; e < V; ++e) w[e] = inf ? fx_from(h[e], F) : bits_i64(h[e]);
    i64* hr = &sm.a[b][ty == 0 ? 0 : BY + 1][V + tx * V];
#pragma unroll
    for (int e = 0; e < V; ++e) hr[e] = w[e];
  }
  const i64 yy = (by0 + ty) % ny;
  if (tx == 0) sm.a[b][ty + 1][V - 1] = fx_in(__ldg(pl + yy * nx + (bx0 - 1 + nx) % nx), inf, F);
  if (tx == BX - 1) sm.a[b][ty + 1][V + BX * V] = fx_in(__ldg(pl + yy * nx + (bx0 + BX * V) % nx), inf, F);
  if (tx == 0 && ty == 0) {
    const i64 xl = (bx0 - 1 + nx) % nx, xr = (bx0 + BX * V) % nx;
    const i64 yt = (by0 - 1 + ny) % ny, yb = (by0 + BY) % ny;
    sm.a[b][0][V - 1] = fx_in(__ldg(pl + yt * nx + xl), inf, F);
    sm.a[b][0][V + BX * V] = fx_in(__ldg(pl + yt * nx + xr), inf, F);
    sm.a[b][BY + 1][V - 1] = fx_in(__ldg(pl + yb * nx + xl), inf, F);
    sm.a[b][BY + 1][V + BX * V] = fx_in(__ldg(pl + yb * nx + xr), inf, F);
  }
}

template <bool EDGE, int BX, int BY, int V, int ZC, class P>
JD void box27_fx_body(const double* __restrict__ u, double* __restrict__ v, const P& p, int F, int flags, s128& acc,
                      Plane<i64, BX, BY, V>& sm) {
  const i64 nx = p.nx, ny = p.ny, nz = p.nz;
  const i64 sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const i64 bx0 = (i64)blockIdx.x * (BX * V);
  const i64 by0 = (i64)blockIdx.y * BY;
  const i64 x0 = bx0 + (i64)tx * V;
  const i64 y = by0 + ty;
  const bool act = (x0 < nx) && (y < ny);
  const i64 z0 = (i64)blockIdx.z * ZC;
  const i64 z1 = (z0 + ZC < nz) ? z0 + ZC : nz;
  const bool inf = EDGE && (flags & JFX_IN_F64);
  const bool outf = EDGE && (flags & JFX_OUT_F64);
  const double* urow = u + (y % ny) * nx + (x0 % nx);  // periodic image for overhanging threads
  double* vrow = v + y * nx + x0;
  const i64 w0 = p.fw0, w1 = p.fw1, w2 = p.fw2, w3 = p.fw3;
  const int K = p.fk;

  i64 cm[V], fm[V], gm[V], c0[V], f0[V], g0[V];
  int b = 0;
  fx_plane_load_put<BX, BY, V>(u, nx, ny, nz, z0 - 1, bx0, by0, urow, sm, b, F, inf);
  __syncthreads();
  plane_cfe<double, BX, BY, V, JM_FIXED>(sm, b, cm, fm, gm);
  b ^= 1;
  fx_plane_load_put<BX, BY, V>(u, nx, ny, nz, z0, bx0, by0, urow, sm, b, F, inf);
  __syncthreads();
  plane_cfe<double, BX, BY, V, JM_FIXED>(sm, b, c0, f0, g0);
  b ^= 1;
  for (i64 z = z0; z < z1; ++z) {
    fx_plane_load_put<BX, BY, V>(u, nx, ny, nz, z + 1, bx0, by0, urow, sm, b, F, inf);
    __syncthreads();
    i64 cn[V], fn[V], gn[V];
    plane_cfe<double, BX, BY, V, JM_FIXED>(sm, b, cn, fn, gn);
    double out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      s128 a = mul_s64_u64(c0[e], (u64)w0);
      a = add128(a, mul_s64_u64((f0[e] + cm[e]) + cn[e], (u64)w1));
      a = add128(a, mul_s64_u64((g0[e] + fm[e]) + fn[e], (u64)w2));
      a = add128(a, mul_s64_u64(gm[e] + gn[e], (u64)w3));
      const i64 q = fx128_round_shift(a, K);
      out[e] = outf ? fx128_to(a, F + K) : i64_bits(q);
      if (act) {
        s128 t;
        t.lo = (u64)q;
        t.hi = (u64)(q >> 63);
        acc = add128(acc, t);
      }
    }
    if (act) stv<double, V>(vrow + z * sz, out);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      cm[e] = c0[e]; fm[e] = f0[e]; gm[e] = g0[e];
      c0[e] = cn[e]; f0[e] = fn[e]; g0[e] = gn[e];
    }
    b ^= 1;
  }
}

// ====================================================================== kernels
//
// Every stencil kernel has the signature
//   (const T* u, T* v, JParams p, double* resid, const u64* maxword, int flags)
// and calls an entry below with P = JParams (precompiled) or P = a struct of
// constants (NVRTC); the runtime-only fields (status word, wait limits) are
// read from the JParams argument `rt` in both cases.
// resid (nullable) receives the fused reduction via one atomic per CTA (it
// must be zeroed before the launch); maxword (FP64 only, nullable) holds the
// bit pattern of max|u| written by jacc_k_maxabs, which selects the fixed
// point scale.  With maxword NULL or fpath NONE the native path runs.
// flags (JFX_*) say whether this sweep of a sequence reads and writes FP64
// or the resident fixed-point representation; native paths ignore them.
// EDGE = false instantiations run the intermediate sweeps of a fixed-point
// sequence and contain no conversion code; EDGE = true ones run the first and
// last sweeps and single launches.

// Whether the 5-point march prefetches rows and x-edges several rows ahead
// (jacobi_march_pf).  That pays on small, L2-resident grids, whose sweeps are
// latency-bound; on large grids its registers cost more occupancy than it
// gains, so the precompiled kernels (P = JParams) use the plain march and a
// constant-folded variant opts in by specialising this for its own P.
template <class P> struct JacobiPrefetch { static constexpr bool value = false; };

template <class T, int BX, int BY, int V, int ZC, bool EDGE, class P>
JD void jacobi2d_entry(const T* __restrict__ u, T* __restrict__ v, const P& p, const JParams& rt, double* resid,
                       const u64* maxword, int flags) {
  griddep_wait();
  u64 bits = 0;
  const i64 x0 = (i64)blockIdx.x * (BX * V) + (i64)threadIdx.x * V;
  const i64 ys = ((i64)blockIdx.y * BY + threadIdx.y) * ZC;
  const i64 ye = (ys + ZC < p.ny) ? ys + ZC : p.ny;
  if constexpr (sizeof(T) == 8) {
    const int F = (maxword && p.fpath != JACC_FP_NONE) ? fx_frac_bits(*maxword) : -1;
    if (F >= 0) {
      u64 m = 0;
      if (ys < p.ny) {
        if constexpr (JacobiPrefetch<P>::value)
          jacobi_march_pf<double, V, false, true, EDGE, 4>(u, v, p.nx, p.ny, x0, ys, ye, F, flags, m);
        else
          jacobi_fx_march<V, false, EDGE>(u, v, p.nx, p.ny, x0, ys, ye, F, flags, m);
      }
      bits = dbits(fx_to_u(m, F + 2));
    } else {
      double m = 0.0;
      if (ys < p.ny) {
        if constexpr (JacobiPrefetch<P>::value)
          jacobi_march_pf<T, V, false, false, false, 4>(u, v, p.nx, p.ny, x0, ys, ye, -1, 0, m);
        else
          jacobi_march<T, V, JM_NATIVE, false>(u, v, p.nx, p.ny, x0, ys, ye, -1, m);
      }
      bits = dbits(m);
    }
  } else {
    T m = T(0);
    if (ys < p.ny) {
      if constexpr (JacobiPrefetch<P>::value)
        jacobi_march_pf<T, V, false, false, false, 4>(u, v, p.nx, p.ny, x0, ys, ye, -1, 0, m);
      else
        jacobi_march<T, V, JM_NATIVE, false>(u, v, p.nx, p.ny, x0, ys, ye, -1, m);
    }
    bits = dbits((double)m);
  }
  block_max_to<BX * BY>(bits, resid);
}

template <class T, int BX, int BY, int V, int ZC, bool EDGE, class P>
JD void heat3d_entry(const T* __restrict__ u, T* __restrict__ v, const P& p, const JParams& rt, double* resid,
                     const u64* maxword, int flags) {
  griddep_wait();
  u64 bits = 0;
  if constexpr (sizeof(T) == 8) {
    // 16-byte columns: the staged kernel (2 rows per thread, so a CTA covers
    // 2 BY rows; the native fallback then runs two BY-row sub-tiles)
    constexpr bool STAGED = V == 2;
    constexpr size_t SM_PLANE = sizeof(Plane<i64, BX, BY, V>);
    // stage cap: 5 for the constant-folded intermediate sweeps (7 CTAs per SM,
    // SweepMinBlocks), else 6
    constexpr int SC = (!EDGE && !SameT<P, JParams>::value) ? 5 : 6;
    constexpr size_t SM_STAGED = STAGED ? sizeof(Heat3SSmem<double, BX, BY, SC>) : 0;
    __shared__ __align__(128) unsigned char raw[SM_PLANE > SM_STAGED ? SM_PLANE : SM_STAGED];
    const int F = (maxword && p.fpath != JACC_FP_NONE) ? fx_frac_bits(*maxword) : -1;
    if (F >= 0) {
      u64 m = 0;
      if constexpr (STAGED)
        heat3s_body<double, BX, BY, ZC, true, EDGE, SC>(u, v, p, rt, F, flags, m,
                                                        *reinterpret_cast<Heat3SSmem<double, BX, BY, SC>*>(raw));
      else
        heat3d_fx_body<EDGE, BX, BY, V, ZC>(u, v, p, F, flags, m, *reinterpret_cast<Plane<i64, BX, BY, V>*>(raw));
      bits = dbits(fx_to_u(m, F));  // max |v - c| in fixed point
    } else {
      double m = 0.0;
#pragma unroll 1
      for (int sub = 0; sub < (STAGED ? 2 : 1); ++sub)
        heat3d_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, m, *reinterpret_cast<Plane<double, BX, BY, V>*>(raw),
                                                 STAGED ? 2 : 1, sub);
      bits = dbits(m);
    }
  } else if constexpr (V == 4) {
    __shared__ Heat3SSmem<float, BX, BY, 6> sm;
    float m = 0.0f;
    heat3s_body<float, BX, BY, ZC, false, false, 6>(u, v, p, rt, -1, 0, m, sm);
    bits = dbits((double)m);
  } else {
    __shared__ Plane<T, BX, BY, V> sm;
    T m = T(0);
    heat3d_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, m, sm);
    bits = dbits((double)m);
  }
  block_max_to<BX * BY>(bits, resid);
}

template <class T, int BX, int BY, int V, int ZC, bool EDGE, class P>
JD void box27_entry(const T* __restrict__ u, T* __restrict__ v, const P& p, const JParams& rt, double* resid,
                    const u64* maxword, int flags) {
  griddep_wait();
  double total = 0.0;
  if constexpr (sizeof(T) == 8) {
    const int F = (maxword && p.fpath != JACC_FP_NONE) ? fx_frac_bits(*maxword) : -1;
    __shared__ __align__(16) unsigned char raw[sizeof(Plane<i64, BX, BY, V>)];
    if (F >= 0) {
      s128 acc;
      acc.lo = acc.hi = 0ull;
      box27_fx_body<EDGE, BX, BY, V, ZC>(u, v, p, F, flags, acc, *reinterpret_cast<Plane<i64, BX, BY, V>*>(raw));
      total = fx128_to(acc, F);
    } else {
      SumAcc<T> acc;
      box27_body2<T, BX, BY, V, ZC>(u, v, p, acc, resid != nullptr, *reinterpret_cast<Plane<double, BX, BY, V>*>(raw));
      total = acc.total();
    }
  } else if constexpr (V == 4) {
    total = box27s_body<BX, BY, ZC>(u, v, p, rt, resid != nullptr);
  } else {
    __shared__ Plane<T, BX, BY, V> sm;
    SumAcc<T> acc;
    box27_body2<T, BX, BY, V, ZC>(u, v, p, acc, resid != nullptr, sm);
    total = acc.total();
  }
  block_sum_to<BX * BY>(total, resid);
}

#ifdef JACC_AUX_KERNELS
// Pre-pass: atomicMax of the bit pattern of |u[i]| over n doubles.
// Any NaN orders above +Inf, so a NaN input selects the native path.
__global__ void __launch_bounds__(256) jacc_k_maxabs(const double* __restrict__ u, i64 n, u64* maxword) {
  griddep_wait();
  u64 m = 0;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 n2 = n / 2;
  const double2* u2 = reinterpret_cast<const double2*>(u);
  auto take = [&](double2 t) {
    const u64 a = dbits(t.x) & 0x7fffffffffffffffull, c = dbits(t.y) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
    m = c > m ? c : m;
  };
  i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  // four independent 16-byte loads in flight per thread (one resident wave)
  for (; i + 3 * stride < n2; i += 4 * stride) {
    double2 t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = __ldg(u2 + i + q * stride);
#pragma unroll
    for (int q = 0; q < 4; ++q) take(t[q]);
  }
  for (; i < n2; i += stride) take(__ldg(u2 + i));
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    u64 a = dbits(u[n - 1]) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
  }
  m = warp_max_u64(m);
  __shared__ u64 red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    u64 w = threadIdx.x < 8 ? red[threadIdx.x] : 0ull;
    w = warp_max_u64(w);
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long*>(maxword), (unsigned long long)w);
  }
}

// In-place conversion of an FP64 field to the resident 64-bit fixed point,
// q = u 2^F truncated toward zero with F from the max-abs word (the same
// conversion the first sweep of a sequence applies on load), so that the
// first sweep of a long sequence of a large field can run the intermediate
// kernel.  A field routed to native FP64 (F < 0) is left unchanged.
__global__ void __launch_bounds__(256) jacc_k_to_fixed(double* __restrict__ u, i64 n, const u64* maxword) {
  griddep_wait();
  const int F = fx_frac_bits(*maxword);
  if (F < 0) return;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 n2 = n / 2;
  double2* u2 = reinterpret_cast<double2*>(u);
  auto cvt = [&](double2 t) {
    double2 q;
    q.x = __longlong_as_double(fx_from(t.x, F));
    q.y = __longlong_as_double(fx_from(t.y, F));
    return q;
  };
  i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  // four independent 16-byte loads in flight per thread (one resident wave)
  for (; i + 3 * stride < n2; i += 4 * stride) {
    double2 t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = u2[i + q * stride];
#pragma unroll
    for (int q = 0; q < 4; ++q) u2[i + q * stride] = cvt(t[q]);
  }
  for (; i < n2; i += stride) u2[i] = cvt(u2[i]);
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) u[n - 1] = __longlong_as_double(fx_from(u[n - 1], F));
}

// Writes NaN to resid[i] for i in [0, n) with (i + 1) % T != 0 and i != n-1:
// the sweeps a temporally blocked launch does not materialise.
__global__ void jacc_k_fill_skipped(double* resid, int n, int T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && ((i + 1) % T) != 0 && i != n - 1) resid[i] = __longlong_as_double(0x7ff8000000000000LL);
}

#endif  // JACC_AUX_KERNELS

// Minimum resident CTAs per SM asked of the compiler (the second launch
// bound) for a sweep kernel.  For the staged FP64 7-point kernel with 32 x 4
// threads (512^3, 200 sweeps): the constant-folded intermediate sweeps at 7
// CTAs (at most 72 registers, 5 stages of 5.4 KB) run 384.7 GLUP/s against
// 378.8 at 6; the precompiled intermediate sweeps spill at that bound (298.9)
// and, unbounded, take 124 registers (4 CTAs), so they ask for 6 (80
// registers, 6 stages); the converting sweeps at 5 CTAs (at most 102
// registers, from 157) take 2.40 ms for a 2-sweep sequence against 2.83.
// Every other kernel: 0, no requirement (a bound of 1 is not neutral: it
// lets the compiler take registers for one CTA per SM, e.g. 111 instead of
// 80 for the staged FP32 7-point kernel).
template <int STENCIL, class T, int BX, int BY, int V, bool EDGE, bool FOLDED> struct SweepMinBlocks {
  static constexpr bool heat_staged_fp64 = STENCIL == 7 && sizeof(T) == 8 && BX == 32 && BY == 4 && V == 2;
  static constexpr int value = heat_staged_fp64 ? (EDGE ? 5 : (FOLDED ? 7 : 6)) : 0;
};

// The constant-folded last sweep of a sequence that does not convert on load
// (the flags are the constant JFX_OUT_F64, so the load conversion is compiled
// out): 80 registers at a bound of 6 CTAs per SM against 96 at 5 for the
// kernel that converts both ways (staged FP64 7-point, 32 x 4 threads).
template <int STENCIL, class T, int BX, int BY, int V> struct SweepMinBlocksLast {
  static constexpr int value = (STENCIL == 7 && sizeof(T) == 8 && BX == 32 && BY == 4 && V == 2) ? 6 : 0;
};

// Kernel templates instantiated by the precompiled library (P = JParams).
template <class T, int BX, int BY, int V, int ZC, bool EDGE>
__global__ void __launch_bounds__(BX * BY) jacc_k_jacobi2d(const T* __restrict__ u, T* __restrict__ v, JParams p,
                                                           double* resid, const u64* maxword, int flags) {
  jacobi2d_entry<T, BX, BY, V, ZC, EDGE>(u, v, p, p, resid, maxword, flags);
}
template <class T, int BX, int BY, int V, int ZC, bool EDGE>
__global__ void __launch_bounds__(BX * BY, (SweepMinBlocks<7, T, BX, BY, V, EDGE, false>::value))
    jacc_k_heat3d(const T* __restrict__ u, T* __restrict__ v, JParams p,
                                                         double* resid, const u64* maxword, int flags) {
  heat3d_entry<T, BX, BY, V, ZC, EDGE>(u, v, p, p, resid, maxword, flags);
}
template <int RY, int TT, int ZC>
__global__ void __launch_bounds__(TB_BX * RY) jacc_k_box27_tb(const float* __restrict__ u, float* __restrict__ v,
                                                              JParams p, double* resid, const u64* maxword, int flags) {
  box27_tb_entry<RY, TT, ZC>(u, v, p, resid);
}
template <class T, int BX, int BY, int V, int ZC, bool EDGE>
__global__ void __launch_bounds__(BX * BY) jacc_k_box27(const T* __restrict__ u, T* __restrict__ v, JParams p,
                                                        double* resid, const u64* maxword, int flags) {
  box27_entry<T, BX, BY, V, ZC, EDGE>(u, v, p, p, resid, maxword, flags);
}
