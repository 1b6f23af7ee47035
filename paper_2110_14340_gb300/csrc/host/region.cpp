// region.cpp - jacc_region_analyze: touched index ranges of an affine loop nest.
//
// The JACC runtime tracks the data range each kernel argument covers to
// decide synchronisation and placement (§3.2.1) and gives every updated array
// per-device write bounds a_lb/a_ub (§4.1); references to one array are
// merged to the widest range (§4.1).  For a rectangular nest every affine
// form sum_k c_k i_k + off is separable over the loops, so its extremes over
// the iteration domain are the sums of per-loop extremes, and each per-loop
// extreme sits at the loop's first or last iterate.
#include <cstring>

#include "jacc_internal.h"

namespace {

using wide = __int128;

constexpr wide kMin = -(static_cast<wide>(1) << 63);
constexpr wide kMax = (static_cast<wide>(1) << 63) - 1;

inline bool in64(wide v) { return v >= kMin && v <= kMax; }

// Iterates of one loop: first, last and whether there is any.
struct Span {
  wide first = 0, last = 0;
  bool empty = false;
};

Span span_of(const jacc_loop& L) {
  Span s;
  const wide lo = L.lo, hi = L.hi, st = L.step;
  const wide dist = (st > 0) ? hi - lo : lo - hi;
  const wide mag = (st > 0) ? st : -st;
  if (dist < 0) {
    s.empty = true;
    return s;
  }
  s.first = lo;
  s.last = lo + (dist / mag) * st;
  return s;
}

// [lo, hi] of off + sum_k c[k] i_k, or false on int64 overflow.
bool extremes(const Span* sp, int n, const int64_t* c, wide off, int64_t* lo, int64_t* hi) {
  wide a = off, b = off;
  for (int k = 0; k < n; ++k) {
    if (c[k] == 0) continue;
    const wide t0 = static_cast<wide>(c[k]) * sp[k].first;
    const wide t1 = static_cast<wide>(c[k]) * sp[k].last;
    if (!in64(t0) || !in64(t1)) return false;
    if (t0 <= t1) {
      a += t0;
      b += t1;
    } else {
      a += t1;
      b += t0;
    }
  }
  if (!in64(a) || !in64(b)) return false;
  *lo = static_cast<int64_t>(a);
  *hi = static_cast<int64_t>(b);
  return true;
}

void widen(int32_t* has, int64_t* lo, int64_t* hi, int nd, const int64_t* nlo, const int64_t* nhi) {
  for (int d = 0; d < nd; ++d) {
    if (!*has || nlo[d] < lo[d]) lo[d] = nlo[d];
    if (!*has || nhi[d] > hi[d]) hi[d] = nhi[d];
  }
}

}  // namespace

extern "C" jacc_status jacc_region_analyze(int32_t nloops, const jacc_loop* loops, int32_t nrefs, const jacc_ref* refs,
                                           int32_t narrays, const jacc_array* arrays, jacc_region* out) {
  using jacc::fail;
  if (nloops < 0 || nloops > JACC_MAX_LOOPS) return fail(JACC_ERR_INVALID_ARG, "nloops outside [0, JACC_MAX_LOOPS]");
  if (nrefs < 0 || narrays < 0) return fail(JACC_ERR_INVALID_ARG, "negative reference or array count");
  if ((nloops && !loops) || (nrefs && !refs) || (narrays && (!arrays || !out)))
    return fail(JACC_ERR_INVALID_ARG, "NULL array with a non-zero count");
  for (int k = 0; k < nloops; ++k)
    if (loops[k].step == 0) return fail(JACC_ERR_INVALID_ARG, "loop step 0");
  for (int a = 0; a < narrays; ++a) {
    if (arrays[a].ndim < 1 || arrays[a].ndim > JACC_MAX_DIMS)
      return fail(JACC_ERR_INVALID_ARG, "array ndim outside [1, JACC_MAX_DIMS]");
    for (int d = 0; d < arrays[a].ndim; ++d)
      if (arrays[a].extent[d] < 0) return fail(JACC_ERR_INVALID_ARG, "negative extent");
  }
  for (int r = 0; r < nrefs; ++r) {
    if (refs[r].array_id < 0 || refs[r].array_id >= narrays)
      return fail(JACC_ERR_INVALID_ARG, "reference array_id out of range");
    if (refs[r].ndim != arrays[refs[r].array_id].ndim)
      return fail(JACC_ERR_INVALID_ARG, "reference ndim differs from its array");
  }
  std::memset(out, 0, sizeof(jacc_region) * static_cast<size_t>(narrays));

  Span sp[JACC_MAX_LOOPS];
  for (int k = 0; k < nloops; ++k) {
    sp[k] = span_of(loops[k]);
    if (sp[k].empty) return jacc::ok();  // the nest never runs
  }

  for (int r = 0; r < nrefs; ++r) {
    const jacc_ref& R = refs[r];
    const jacc_array& A = arrays[R.array_id];
    const int nd = R.ndim;
    int64_t lo[JACC_MAX_DIMS], hi[JACC_MAX_DIMS];
    for (int d = 0; d < nd; ++d)
      if (!extremes(sp, nloops, R.coef[d], R.off[d], &lo[d], &hi[d]))
        return fail(JACC_ERR_OVERFLOW, "subscript bound overflows int64");

    // flattened offset: coefficients sum_d stride_d c[d][k], offset sum_d stride_d off[d]
    wide stride = 1;
    wide fc[JACC_MAX_LOOPS] = {0};
    wide foff = 0;
    for (int d = nd - 1; d >= 0; --d) {
      if (d < nd - 1) {
        stride *= A.extent[d + 1];
        if (!in64(stride)) return fail(JACC_ERR_OVERFLOW, "array stride overflows int64");
      }
      for (int k = 0; k < nloops; ++k) {
        const wide t = stride * R.coef[d][k];
        if (!in64(t)) return fail(JACC_ERR_OVERFLOW, "flattened coefficient overflows int64");
        fc[k] += t;
      }
      const wide t = stride * R.off[d];
      if (!in64(t)) return fail(JACC_ERR_OVERFLOW, "flattened offset overflows int64");
      foff += t;
    }
    int64_t fc64[JACC_MAX_LOOPS];
    for (int k = 0; k < nloops; ++k) {
      if (!in64(fc[k])) return fail(JACC_ERR_OVERFLOW, "flattened coefficient overflows int64");
      fc64[k] = static_cast<int64_t>(fc[k]);
    }
    if (!in64(foff)) return fail(JACC_ERR_OVERFLOW, "flattened offset overflows int64");
    int64_t llo, lhi;
    if (!extremes(sp, nloops, fc64, foff, &llo, &lhi)) return fail(JACC_ERR_OVERFLOW, "flattened bound overflows int64");

    jacc_region& O = out[R.array_id];
    if (R.is_write) {
      widen(&O.has_write, O.wlo, O.whi, nd, lo, hi);
      if (!O.has_write || llo < O.wlin_lo) O.wlin_lo = llo;
      if (!O.has_write || lhi > O.wlin_hi) O.wlin_hi = lhi;
      O.has_write = 1;
    } else {
      widen(&O.has_read, O.rlo, O.rhi, nd, lo, hi);
      if (!O.has_read || llo < O.rlin_lo) O.rlin_lo = llo;
      if (!O.has_read || lhi > O.rlin_hi) O.rlin_hi = lhi;
      O.has_read = 1;
    }
  }

  for (int a = 0; a < narrays; ++a) {
    const jacc_region& O = out[a];
    for (int d = 0; d < arrays[a].ndim; ++d) {
      const int64_t last = arrays[a].extent[d] - 1;
      if ((O.has_read && (O.rlo[d] < 0 || O.rhi[d] > last)) || (O.has_write && (O.wlo[d] < 0 || O.whi[d] > last)))
        return fail(JACC_ERR_OUT_OF_BOUNDS, "touched region leaves array " + std::to_string(a));
    }
  }
  return jacc::ok();
}
