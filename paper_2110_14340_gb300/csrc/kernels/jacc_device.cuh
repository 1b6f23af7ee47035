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

JD u64 warp_max_u64(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u64 w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
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
      if constexpr (MODE == JM_FIXED) {
        const i64 s = (up[e] + dn[e]) + (xl + xr);  // exact; v = s * 2^-(F+2)
        out[e] = in ? (T)fx_to(s, F + 2) : rcur[e];
        const i64 d = s - cur[e] * 4;   // 4 (v - u) in scale F
        const u64 ad = (u64)(d < 0 ? -d : d);
        if (in && ad > rmax) rmax = ad;
      } else {
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

// CTA = BX x BY threads; thread row ty marches rows [ys, ys + ZC).
template <class T, int BX, int BY, int V, int ZC, int MODE, class P>
JD void jacobi2d_body(const T* __restrict__ u, T* __restrict__ v, const P& p, int F,
                      typename RT<T, MODE>::type& rmax) {
  const i64 nx = p.nx, ny = p.ny;
  const i64 x0 = (i64)blockIdx.x * (BX * V) + (i64)threadIdx.x * V;
  const i64 ys = ((i64)blockIdx.y * BY + threadIdx.y) * ZC;
  const i64 ye = (ys + ZC < ny) ? ys + ZC : ny;
  if (ys >= ny) return;  // whole warp (a warp lies within one thread row)
  jacobi_march<T, V, MODE, false>(u, v, nx, ny, x0, ys, ye, F, rmax);
}

// ====================================================================== 3D z-marching tiles
//
// CTA = BX x BY threads covering x in [bx0, bx0 + BX*V), y in [by0, by0 + BY),
// marching z over [cz0, cz0 + ZC).  The current plane lives in shared memory
// with a one-point halo in x and y (double-buffered, so one __syncthreads per
// plane); each thread keeps its own column's z-1, z, z+1 in registers.
// Loads for plane z+1 (halo) and z+2 (own) are issued one iteration ahead.

template <class W, int BX, int BY, int V> struct Plane {
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
      if constexpr (MODE == JM_FIXED) {
        const i64 L = s - 6 * cur[e];
        double o;
        if (p.fpath == JACC_FP_SMALL) {
          o = fx_to(p.fa * cur[e] + p.fb * s, F + p.fk);
        } else {
          o = fx128_to(add128(from_s64_shl(cur[e], p.fk), mul_s64_u64(L, (u64)p.fw0)), F + p.fk);
        }
        out[e] = in ? (T)o : rcur[e];
        const u64 aL = (u64)(L < 0 ? -L : L);
        if (in && aL > rmax) rmax = aL;
      } else {
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
template <class P> JD double heat_resid_fixed(const P& p, u64 maxL, int F) {
  const u64 m = (p.fpath == JACC_FP_SMALL) ? (u64)p.fb : (u64)p.fw0;
  return fx128_to(mul_s64_u64((i64)maxL, m), F + p.fk);
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
      if constexpr (MODE == JM_FIXED) {
        s128 a = mul_s64_u64(c0[e], (u64)p.fw0);
        a = add128(a, mul_s64_u64(F1, (u64)p.fw1));
        a = add128(a, mul_s64_u64(E2, (u64)p.fw2));
        a = add128(a, mul_s64_u64(C3, (u64)p.fw3));
        out[e] = (T)fx128_to(a, F + p.fk);
      } else {
        out[e] = ((T)p.c0 * c0[e] + (T)p.c1 * F1) + ((T)p.c2 * E2 + (T)p.c3 * C3);
      }
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

// ====================================================================== kernels
//
// Every stencil kernel has the signature
//   (const T* u, T* v, P p, double* resid, const u64* maxword)
// resid (nullable) receives the fused reduction via one atomic per CTA (it
// must be zeroed before the launch); maxword (FP64 only, nullable) holds the
// bit pattern of max|u| written by jacc_k_maxabs, which selects the fixed
// point scale.  With maxword NULL or fpath NONE the native path runs.

template <class T, int BX, int BY, int V, int ZC, class P>
JD void jacobi2d_entry(const T* __restrict__ u, T* __restrict__ v, const P& p, double* resid, const u64* maxword) {
  u64 bits = 0;
  if constexpr (sizeof(T) == 8) {
    const int F = (maxword && p.fpath != JACC_FP_NONE) ? fx_frac_bits(*maxword) : -1;
    if (F >= 0) {
      u64 m = 0;
      jacobi2d_body<T, BX, BY, V, ZC, JM_FIXED>(u, v, p, F, m);
      bits = dbits(fx_to_u(m, F + 2));
    } else {
      double m = 0.0;
      jacobi2d_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, m);
      bits = dbits(m);
    }
  } else {
    T m = T(0);
    jacobi2d_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, m);
    bits = dbits((double)m);
  }
  block_max_to<BX * BY>(bits, resid);
}

template <class T, int BX, int BY, int V, int ZC, class P>
JD void heat3d_entry(const T* __restrict__ u, T* __restrict__ v, const P& p, double* resid, const u64* maxword) {
  u64 bits = 0;
  if constexpr (sizeof(T) == 8) {
    const int F = (maxword && p.fpath != JACC_FP_NONE) ? fx_frac_bits(*maxword) : -1;
    __shared__ __align__(16) unsigned char raw[sizeof(Plane<i64, BX, BY, V>)];
    if (F >= 0) {
      u64 m = 0;
      heat3d_body<T, BX, BY, V, ZC, JM_FIXED>(u, v, p, F, m, *reinterpret_cast<Plane<i64, BX, BY, V>*>(raw));
      bits = dbits(heat_resid_fixed(p, m, F));
    } else {
      double m = 0.0;
      heat3d_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, m, *reinterpret_cast<Plane<double, BX, BY, V>*>(raw));
      bits = dbits(m);
    }
  } else {
    __shared__ Plane<T, BX, BY, V> sm;
    T m = T(0);
    heat3d_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, m, sm);
    bits = dbits((double)m);
  }
  block_max_to<BX * BY>(bits, resid);
}

template <class T, int BX, int BY, int V, int ZC, class P>
JD void box27_entry(const T* __restrict__ u, T* __restrict__ v, const P& p, double* resid, const u64* maxword) {
  SumAcc<T> acc;
  if constexpr (sizeof(T) == 8) {
    const int F = (maxword && p.fpath != JACC_FP_NONE) ? fx_frac_bits(*maxword) : -1;
    __shared__ __align__(16) unsigned char raw[sizeof(Plane<i64, BX, BY, V>)];
    if (F >= 0) {
      box27_body<T, BX, BY, V, ZC, JM_FIXED>(u, v, p, F, acc, *reinterpret_cast<Plane<i64, BX, BY, V>*>(raw));
    } else {
      box27_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, acc, *reinterpret_cast<Plane<double, BX, BY, V>*>(raw));
    }
  } else {
    __shared__ Plane<T, BX, BY, V> sm;
    box27_body<T, BX, BY, V, ZC, JM_NATIVE>(u, v, p, -1, acc, sm);
  }
  block_sum_to<BX * BY>(acc.total(), resid);
}

#ifdef JACC_AUX_KERNELS
// Pre-pass: atomicMax of the bit pattern of |u[i]| over n doubles.
// Any NaN orders above +Inf, so a NaN input selects the native path.
__global__ void __launch_bounds__(256) jacc_k_maxabs(const double* __restrict__ u, i64 n, u64* maxword) {
  u64 m = 0;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 n2 = n / 2;
  const double2* u2 = reinterpret_cast<const double2*>(u);
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    double2 t = __ldg(u2 + i);
    u64 a = dbits(t.x) & 0x7fffffffffffffffull, c = dbits(t.y) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
    m = c > m ? c : m;
  }
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

// Writes NaN to resid[i] for i in [0, n) with (i + 1) % T != 0 and i != n-1:
// the sweeps a temporally blocked launch does not materialise.
__global__ void jacc_k_fill_skipped(double* resid, int n, int T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && ((i + 1) % T) != 0 && i != n - 1) resid[i] = __longlong_as_double(0x7ff8000000000000LL);
}

#endif  // JACC_AUX_KERNELS

// Kernel templates instantiated by the precompiled library (P = JParams).
template <class T, int BX, int BY, int V, int ZC>
__global__ void __launch_bounds__(BX * BY) jacc_k_jacobi2d(const T* __restrict__ u, T* __restrict__ v, JParams p,
                                                           double* resid, const u64* maxword) {
  jacobi2d_entry<T, BX, BY, V, ZC>(u, v, p, resid, maxword);
}
template <class T, int BX, int BY, int V, int ZC>
__global__ void __launch_bounds__(BX * BY) jacc_k_heat3d(const T* __restrict__ u, T* __restrict__ v, JParams p,
                                                         double* resid, const u64* maxword) {
  heat3d_entry<T, BX, BY, V, ZC>(u, v, p, resid, maxword);
}
template <class T, int BX, int BY, int V, int ZC>
__global__ void __launch_bounds__(BX * BY) jacc_k_box27(const T* __restrict__ u, T* __restrict__ v, JParams p,
                                                        double* resid, const u64* maxword) {
  box27_entry<T, BX, BY, V, ZC>(u, v, p, resid, maxword);
}
