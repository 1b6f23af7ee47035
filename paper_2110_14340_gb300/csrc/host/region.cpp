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
#include <string>
#include <vector>

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

namespace {

// Shared checks of references and arrays (jacc_region_analyze's rules).
jacc_status check_refs(int32_t nrefs, const jacc_ref* refs, int32_t narrays, const jacc_array* arrays) {
  using jacc::fail;
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
  return jacc::ok();
}

// The flattened row-major offset of a reference as an affine form.
bool flatten(const jacc_ref& R, const jacc_array& A, int nloops, wide* fc, wide* foff) {
  const int nd = R.ndim;
  wide stride = 1;
  for (int k = 0; k < nloops; ++k) fc[k] = 0;
  *foff = 0;
  for (int d = nd - 1; d >= 0; --d) {
    if (d < nd - 1) {
      stride *= A.extent[d + 1];
      if (!in64(stride)) return false;
    }
    for (int k = 0; k < nloops; ++k) {
      const wide t = stride * R.coef[d][k];
      if (!in64(t)) return false;
      fc[k] += t;
      if (!in64(fc[k])) return false;
    }
    const wide t = stride * R.off[d];
    if (!in64(t)) return false;
    *foff += t;
    if (!in64(*foff)) return false;
  }
  return true;
}

// Max (want_max) or min of off + sum_k c[k] i_k over an affine nest whose
// loops never run empty: eliminate the loops from the innermost out, the
// extreme of c i_k over [lo_k, hi_k] being c at hi_k or lo_k, an affine form
// in the outer indices.  False when a coefficient or constant leaves int64.
bool affine_extreme(const jacc_loop_affine* L, int n, const wide* c_in, wide off, bool want_max, wide* out) {
  wide c[JACC_MAX_LOOPS];
  for (int k = 0; k < n; ++k) c[k] = c_in[k];
  wide k0 = off;
  for (int k = n - 1; k >= 0; --k) {
    const wide a = c[k];
    if (a == 0) continue;
    const bool use_hi = (a > 0) == want_max;
    const int64_t base = use_hi ? L[k].hi : L[k].lo;
    const int64_t* bc = use_hi ? L[k].hi_coef : L[k].lo_coef;
    k0 += a * base;
    if (!in64(k0)) return false;
    for (int m = 0; m < k; ++m) {
      c[m] += a * bc[m];
      if (!in64(c[m])) return false;
    }
    c[k] = 0;
  }
  *out = k0;
  return true;
}

// The body runs only where every loop is non-empty.  An inner loop k whose
// extent hi_k - lo_k = a i_m + b depends on one outer index i_m with
// constant bounds is non-empty exactly for i_m >= ceil(-b / a) (a > 0) or
// i_m <= floor(b / -a) (a < 0): tightening i_m's bounds to that range drops
// only outer iterations in which the body never runs, so the elimination
// stays exact.  Repeated until no bound moves; emptiness that depends on
// several indices is unsupported.  L receives the tightened nest; *runs =
// false when no iteration runs at all.
jacc_status tighten_affine(int32_t nloops, const jacc_loop_affine* loops, jacc_loop_affine* L, bool* runs) {
  using jacc::fail;
  *runs = true;
  for (int k = 0; k < nloops; ++k) L[k] = loops[k];
  auto floor_div = [](wide p, wide q) { return p >= 0 ? p / q : -((-p + q - 1) / q); };  // q > 0
  for (int pass = 0; pass <= nloops; ++pass) {
    if (nloops > 0 && L[0].hi < L[0].lo) {
      *runs = false;
      return jacc::ok();
    }
    bool moved = false;
    for (int k = 1; k < nloops; ++k) {
      wide d[JACC_MAX_LOOPS];
      for (int m = 0; m < k; ++m) d[m] = static_cast<wide>(L[k].hi_coef[m]) - L[k].lo_coef[m];
      const wide b = static_cast<wide>(L[k].hi) - L[k].lo;
      wide mn;
      if (!affine_extreme(L, k, d, b, false, &mn)) return fail(JACC_ERR_OVERFLOW, "loop extent bound overflows int64");
      if (mn >= 0) continue;
      int var = -1, nvar = 0;
      for (int m = 0; m < k; ++m)
        if (d[m] != 0) {
          var = m;
          ++nvar;
        }
      if (nvar == 0) {  // loop k never runs
        *runs = false;
        return jacc::ok();
      }
      bool const_bounds = true;
      for (int m = 0; m < JACC_MAX_LOOPS; ++m)
        if (L[var].lo_coef[m] || L[var].hi_coef[m]) const_bounds = false;
      if (nvar > 1 || !const_bounds)
        return fail(JACC_ERR_UNSUPPORTED, "loop " + std::to_string(k) +
                                              " is empty for some outer iterations in a way that couples several indices");
      const wide a = d[var];
      if (a > 0) {
        const wide lo = -floor_div(b, a);  // ceil(-b / a)
        if (lo > L[var].lo) {
          L[var].lo = static_cast<int64_t>(lo);
          moved = true;
        }
      } else {
        const wide hi = floor_div(b, -a);
        if (hi < L[var].hi) {
          L[var].hi = static_cast<int64_t>(hi);
          moved = true;
        }
      }
      if (L[var].hi < L[var].lo) {  // no outer iteration runs loop k
        *runs = false;
        return jacc::ok();
      }
    }
    if (!moved) break;
  }
  for (int k = 1; k < nloops; ++k) {  // every loop now runs for every outer iteration left
    wide d[JACC_MAX_LOOPS];
    for (int m = 0; m < k; ++m) d[m] = static_cast<wide>(L[k].hi_coef[m]) - L[k].lo_coef[m];
    wide mn;
    if (!affine_extreme(L, k, d, static_cast<wide>(L[k].hi) - L[k].lo, false, &mn) || mn < 0)
      return fail(JACC_ERR_UNSUPPORTED, "loop " + std::to_string(k) + " is empty for some outer iterations");
  }
  return jacc::ok();
}

// Drops boxes inside another box of the same array and kind (keeping the
// first of equal ones) and writes the rest.
jacc_status emit_boxes(const std::vector<jacc_box>& all, const jacc_array* arrays, jacc_box* boxes, int32_t max_boxes,
                       int32_t* nboxes) {
  auto inside = [&](const jacc_box& a, const jacc_box& b) {
    for (int d = 0; d < arrays[a.array_id].ndim; ++d)
      if (a.lo[d] < b.lo[d] || a.hi[d] > b.hi[d]) return false;
    return true;
  };
  std::vector<jacc_box> keep;
  for (size_t i = 0; i < all.size(); ++i) {
    bool drop = false;
    for (size_t j = 0; j < all.size() && !drop; ++j) {
      if (i == j || all[i].array_id != all[j].array_id || all[i].is_write != all[j].is_write) continue;
      if (inside(all[i], all[j]) && (!inside(all[j], all[i]) || j < i)) drop = true;
    }
    if (!drop) keep.push_back(all[i]);
  }
  *nboxes = static_cast<int32_t>(keep.size());
  for (int32_t i = 0; i < *nboxes && i < max_boxes; ++i) boxes[i] = keep[static_cast<size_t>(i)];
  if (*nboxes > max_boxes) return jacc::fail(JACC_ERR_INVALID_ARG, "more boxes than max_boxes");
  return jacc::ok();
}

jacc_status bounds_check(const jacc_region* out, int32_t narrays, const jacc_array* arrays) {
  for (int a = 0; a < narrays; ++a) {
    const jacc_region& O = out[a];
    for (int d = 0; d < arrays[a].ndim; ++d) {
      const int64_t last = arrays[a].extent[d] - 1;
      if ((O.has_read && (O.rlo[d] < 0 || O.rhi[d] > last)) || (O.has_write && (O.wlo[d] < 0 || O.whi[d] > last)))
        return jacc::fail(JACC_ERR_OUT_OF_BOUNDS, "touched region leaves array " + std::to_string(a));
    }
  }
  return jacc::ok();
}

}  // namespace

extern "C" jacc_status jacc_region_analyze_affine(int32_t nloops, const jacc_loop_affine* loops, int32_t nrefs,
                                                  const jacc_ref* refs, int32_t narrays, const jacc_array* arrays,
                                                  jacc_region* out) {
  using jacc::fail;
  if (nloops < 0 || nloops > JACC_MAX_LOOPS) return fail(JACC_ERR_INVALID_ARG, "nloops outside [0, JACC_MAX_LOOPS]");
  if (nrefs < 0 || narrays < 0) return fail(JACC_ERR_INVALID_ARG, "negative reference or array count");
  if ((nloops && !loops) || (nrefs && !refs) || (narrays && (!arrays || !out)))
    return fail(JACC_ERR_INVALID_ARG, "NULL array with a non-zero count");
  for (int k = 0; k < nloops; ++k)
    for (int m = k; m < JACC_MAX_LOOPS; ++m)
      if (loops[k].lo_coef[m] || loops[k].hi_coef[m])
        return fail(JACC_ERR_INVALID_ARG, "a loop bound may depend only on outer loops");
  jacc_status st = check_refs(nrefs, refs, narrays, arrays);
  if (st) return st;
  std::memset(out, 0, sizeof(jacc_region) * static_cast<size_t>(narrays));
  jacc_loop_affine L[JACC_MAX_LOOPS];
  bool runs = true;
  st = tighten_affine(nloops, loops, L, &runs);
  if (st) return st;
  if (!runs) return jacc::ok();  // the nest never runs: nothing is touched
  loops = L;
  for (int r = 0; r < nrefs; ++r) {
    const jacc_ref& R = refs[r];
    const jacc_array& A = arrays[R.array_id];
    const int nd = R.ndim;
    int64_t lo[JACC_MAX_DIMS], hi[JACC_MAX_DIMS];
    for (int d = 0; d < nd; ++d) {
      wide c[JACC_MAX_LOOPS];
      for (int k = 0; k < nloops; ++k) c[k] = R.coef[d][k];
      wide a, b;
      if (!affine_extreme(loops, nloops, c, R.off[d], false, &a) || !affine_extreme(loops, nloops, c, R.off[d], true, &b))
        return fail(JACC_ERR_OVERFLOW, "subscript bound overflows int64");
      lo[d] = static_cast<int64_t>(a);
      hi[d] = static_cast<int64_t>(b);
    }
    wide fc[JACC_MAX_LOOPS], foff, fa, fb;
    if (!flatten(R, A, nloops, fc, &foff) || !affine_extreme(loops, nloops, fc, foff, false, &fa) ||
        !affine_extreme(loops, nloops, fc, foff, true, &fb))
      return fail(JACC_ERR_OVERFLOW, "flattened bound overflows int64");
    jacc_region& O = out[R.array_id];
    if (R.is_write) {
      widen(&O.has_write, O.wlo, O.whi, nd, lo, hi);
      if (!O.has_write || fa < O.wlin_lo) O.wlin_lo = static_cast<int64_t>(fa);
      if (!O.has_write || fb > O.wlin_hi) O.wlin_hi = static_cast<int64_t>(fb);
      O.has_write = 1;
    } else {
      widen(&O.has_read, O.rlo, O.rhi, nd, lo, hi);
      if (!O.has_read || fa < O.rlin_lo) O.rlin_lo = static_cast<int64_t>(fa);
      if (!O.has_read || fb > O.rlin_hi) O.rlin_hi = static_cast<int64_t>(fb);
      O.has_read = 1;
    }
  }
  return bounds_check(out, narrays, arrays);
}

extern "C" jacc_status jacc_region_boxes(int32_t nloops, const jacc_loop* loops, int32_t nrefs, const jacc_ref* refs,
                                         int32_t narrays, const jacc_array* arrays, jacc_box* boxes, int32_t max_boxes,
                                         int32_t* nboxes) {
  using jacc::fail;
  if (!nboxes || max_boxes < 0 || (max_boxes > 0 && !boxes)) return fail(JACC_ERR_INVALID_ARG, "NULL output");
  if (nloops < 0 || nloops > JACC_MAX_LOOPS) return fail(JACC_ERR_INVALID_ARG, "nloops outside [0, JACC_MAX_LOOPS]");
  if (nrefs < 0 || narrays < 0) return fail(JACC_ERR_INVALID_ARG, "negative reference or array count");
  if ((nloops && !loops) || (nrefs && !refs) || (narrays && !arrays))
    return fail(JACC_ERR_INVALID_ARG, "NULL array with a non-zero count");
  for (int k = 0; k < nloops; ++k)
    if (loops[k].step == 0) return fail(JACC_ERR_INVALID_ARG, "loop step 0");
  jacc_status st = check_refs(nrefs, refs, narrays, arrays);
  if (st) return st;
  *nboxes = 0;
  Span sp[JACC_MAX_LOOPS];
  for (int k = 0; k < nloops; ++k) {
    sp[k] = span_of(loops[k]);
    if (sp[k].empty) return jacc::ok();
  }
  std::vector<jacc_box> all;
  for (int r = 0; r < nrefs; ++r) {
    const jacc_ref& R = refs[r];
    jacc_box b{};
    b.array_id = R.array_id;
    b.is_write = R.is_write ? 1 : 0;
    bool exact = true;
    unsigned used = 0;  // loops a subscript of this reference depends on
    for (int d = 0; d < R.ndim; ++d) {
      if (!extremes(sp, nloops, R.coef[d], R.off[d], &b.lo[d], &b.hi[d]))
        return fail(JACC_ERR_OVERFLOW, "subscript bound overflows int64");
      int nz = 0, kk = -1;
      for (int k = 0; k < nloops; ++k)
        if (R.coef[d][k]) {
          ++nz;
          kk = k;
        }
      if (nz > 1) exact = false;
      if (nz == 1) {
        const int64_t c = R.coef[d][kk];
        if ((c != 1 && c != -1) || (loops[kk].step != 1 && loops[kk].step != -1) || (used >> kk & 1u)) exact = false;
        used |= 1u << kk;
      }
      const int64_t last = arrays[R.array_id].extent[d] - 1;
      if (b.lo[d] < 0 || b.hi[d] > last)
        return fail(JACC_ERR_OUT_OF_BOUNDS, "touched region leaves array " + std::to_string(R.array_id));
    }
    b.exact = exact ? 1 : 0;
    all.push_back(b);
  }
  return emit_boxes(all, arrays, boxes, max_boxes, nboxes);
}

extern "C" jacc_status jacc_region_boxes_affine(int32_t nloops, const jacc_loop_affine* loops, int32_t nrefs,
                                                const jacc_ref* refs, int32_t narrays, const jacc_array* arrays,
                                                jacc_box* boxes, int32_t max_boxes, int32_t* nboxes) {
  using jacc::fail;
  if (!nboxes || max_boxes < 0 || (max_boxes > 0 && !boxes)) return fail(JACC_ERR_INVALID_ARG, "NULL output");
  if (nloops < 0 || nloops > JACC_MAX_LOOPS) return fail(JACC_ERR_INVALID_ARG, "nloops outside [0, JACC_MAX_LOOPS]");
  if (nrefs < 0 || narrays < 0) return fail(JACC_ERR_INVALID_ARG, "negative reference or array count");
  if ((nloops && !loops) || (nrefs && !refs) || (narrays && !arrays))
    return fail(JACC_ERR_INVALID_ARG, "NULL array with a non-zero count");
  for (int k = 0; k < nloops; ++k)
    for (int m = k; m < JACC_MAX_LOOPS; ++m)
      if (loops[k].lo_coef[m] || loops[k].hi_coef[m])
        return fail(JACC_ERR_INVALID_ARG, "a loop bound may depend only on outer loops");
  jacc_status st = check_refs(nrefs, refs, narrays, arrays);
  if (st) return st;
  *nboxes = 0;
  jacc_loop_affine L[JACC_MAX_LOOPS];
  bool runs = true;
  st = tighten_affine(nloops, loops, L, &runs);
  if (st) return st;
  if (!runs) return jacc::ok();
  std::vector<jacc_box> all;
  for (int r = 0; r < nrefs; ++r) {
    const jacc_ref& R = refs[r];
    jacc_box b{};
    b.array_id = R.array_id;
    b.is_write = R.is_write ? 1 : 0;
    // exact when every subscript follows at most one loop, with coefficient
    // +-1, no two subscripts the same loop, and those loops have constant
    // bounds: then every combination of their values occurs (the loops in
    // between never run empty), and the touched set is the whole box
    bool exact = true;
    unsigned used = 0;
    for (int d = 0; d < R.ndim; ++d) {
      wide c[JACC_MAX_LOOPS];
      for (int k = 0; k < nloops; ++k) c[k] = R.coef[d][k];
      wide lo, hi;
      if (!affine_extreme(L, nloops, c, R.off[d], false, &lo) || !affine_extreme(L, nloops, c, R.off[d], true, &hi))
        return fail(JACC_ERR_OVERFLOW, "subscript bound overflows int64");
      b.lo[d] = static_cast<int64_t>(lo);
      b.hi[d] = static_cast<int64_t>(hi);
      int nz = 0, kk = -1;
      for (int k = 0; k < nloops; ++k)
        if (R.coef[d][k]) {
          ++nz;
          kk = k;
        }
      if (nz > 1) exact = false;
      if (nz == 1) {
        const int64_t cc = R.coef[d][kk];
        bool const_bounds = true;
        for (int m = 0; m < JACC_MAX_LOOPS; ++m)
          if (L[kk].lo_coef[m] || L[kk].hi_coef[m]) const_bounds = false;
        if ((cc != 1 && cc != -1) || !const_bounds || (used >> kk & 1u)) exact = false;
        used |= 1u << kk;
      }
      const int64_t last = arrays[R.array_id].extent[d] - 1;
      if (b.lo[d] < 0 || b.hi[d] > last)
        return fail(JACC_ERR_OUT_OF_BOUNDS, "touched region leaves array " + std::to_string(R.array_id));
    }
    b.exact = exact ? 1 : 0;
    all.push_back(b);
  }
  return emit_boxes(all, arrays, boxes, max_boxes, nboxes);
}
