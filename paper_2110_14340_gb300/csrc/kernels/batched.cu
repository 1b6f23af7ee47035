// batched.cu - many uneven 5-point Jacobi grids in one persistent launch.
//
// No counterpart in the paper (which overlaps independent kernels on 16
// OpenACC queues, §6.1).  All sweeps of all grids run inside one cooperative
// launch whose CTAs are co-resident.
//
// Work.  Each grid is cut into items: tiles of `rows` rows x `cols` columns
// (cols = 64 x the warps across a tile).  Grids are packed into groups whose
// two fields fit a budget of L2 bytes together.  Tickets run group by group,
// sweep-major inside a group: ticket t of a group names sweep t / I and item
// t % I of the group's I items.  A group's fields are read from HBM in its
// first sweep and stay in L2 for the rest; the next group's tickets follow,
// so CTAs that find no ready work in a group's last sweeps start the next one.
//
// Dependencies.  The 5-point item (b, c) of sweep s reads the rows above and
// below it and the columns left and right of it, written in sweep s-1 by
// items (b-1, c), (b+1, c), (b, c-1), (b, c+1) and itself, and overwrites
// what those items read in sweep s-1.  So it waits until each of these five
// items has finished s sweeps (a per-item counter), and then sets its own
// counter to s + 1.  Every wait targets strictly smaller tickets.  Tickets
// are handed out in order (one atomic counter; each CTA holds its current
// ticket and a prefetched next one), so the smallest unfinished ticket is
// always some CTA's current ticket, whose dependencies are finished: no
// deadlock.  Waits are bounded by %globaltimer; a wait that gives up writes
// JACC_ERR_TIMEOUT to the status word and every CTA leaves.
//
// Loads.  In the staged variant each warp streams its strip of an item's
// rows through a ring in shared memory: fixed-point units (every grid whose
// maximum allows it) fetch each row with one bulk copy issued by one lane
// and completed on the row slot's mbarrier, 8 rows in flight per warp, and
// intermediate sweeps give each lane 4 columns of a 128-column strip; the
// native FP64 path stages 64-column strips with 16-byte cp.async.cg copies
// (L2 only: the same launch writes the fields, and L1 is not coherent), 16
// rows in flight.  A row whose start is not 16-byte aligned (odd nx, odd
// row) is staged one element to the right.  The register variant marches
// rows through registers with ld.global.cg, as the single-grid kernels do.
#include <cuda_runtime.h>

#include "../host/jacc_internal.h"
#include "batched.h"
#include "jacc_device.cuh"

namespace {

JD void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
JD int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
JD u64 globaltimer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRing = 16;  // staged rows per warp (a power of two)
constexpr int kSlot = 68;  // doubles per staged row: columns x0-2 .. x0+65 (one more when shifted)
constexpr int kRingB = 8;  // staged rows per warp in the bulk-copy march
constexpr int kSlotB = 128 + 4;  // doubles per bulk-staged row of a 128-column strip
constexpr int kRingWords = kRing * kSlot > kRingB * kSlotB ? kRing * kSlot : kRingB * kSlotB;  // per warp
constexpr int kStagedSmem = kWarps * kRingWords * 8;

// ---------------------------------------------------------------- staged march

JD void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
JD void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> JD void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Staging layout.  Row r's columns [x0-1, x0+64] that lie in the grid are
// copied into a slot of 68 doubles: element x goes to slot[x - x0 + 2 + sh],
// sh = (r * nx) & 1, because 16-byte chunks start at even element indices;
// chunk l (columns x0 - sh + 2l and the next) lands at slot[2l + 2].  Lane l
// copies chunk l; lanes 0 and 1 also copy chunk -1 and chunk 32 (the halo
// columns) in the same instruction.  The array's last element, whose pair
// would run past the end of the field, is copied through a register.  The
// plan (which chunks a lane copies, for either parity) is fixed per unit, and
// row addresses advance by nx per row, so staging a row costs a few
// instructions per lane.
struct StagePlan {
  int cfa0, cfa1, cfb0, cfb1;  // first column of the lane's chunks, for sh = 0 and 1
  bool na0, na1, nb0, nb1;     // whether the chunk is needed
  int da, db;                  // slot index of each chunk
};

JD StagePlan stage_plan(int nx, int x0, int lane) {
  StagePlan P;
  const int clo = x0 >= 1 ? x0 - 1 : 0;
  const int chi = x0 + 64 <= nx - 1 ? x0 + 64 : nx - 1;
  const int la = lane, lb = lane == 0 ? -1 : 32;
  P.da = 2 * la + 2;
  P.db = 2 * lb + 2;
  P.cfa0 = x0 + 2 * la;
  P.cfa1 = P.cfa0 - 1;
  P.cfb0 = x0 + 2 * lb;
  P.cfb1 = P.cfb0 - 1;
  P.na0 = P.cfa0 <= chi && P.cfa0 + 1 >= clo;
  P.na1 = P.cfa1 <= chi && P.cfa1 + 1 >= clo;
  P.nb0 = lane < 2 && P.cfb0 <= chi && P.cfb0 + 1 >= clo;
  P.nb1 = lane < 2 && P.cfb1 <= chi && P.cfb1 + 1 >= clo;
  return P;
}

// Copies one row (row pointer rp = u + r nx, parity sh) into slot sp; `last`
// marks the field's last row.
JD void stage_row(const StagePlan& P, double* sp, const double* rp, int sh, bool last, int nx) {
  const bool na = sh ? P.na1 : P.na0, nb = sh ? P.nb1 : P.nb0;
  const int ca = sh ? P.cfa1 : P.cfa0, cb = sh ? P.cfb1 : P.cfb0;
  if (na) {
    if (!last || ca + 1 < nx) cp_async16(sp + P.da, rp + ca);
    else sp[P.da] = __ldcg(rp + ca);
  }
  if (nb) {
    if (!last || cb + 1 < nx) cp_async16(sp + P.db, rp + cb);
    else sp[P.db] = __ldcg(rp + cb);
  }
}

// One warp: output rows [ya, yb) of columns [x0, x0 + 64) (lane: x0 + 2 lane
// and the next column).  Arithmetic and outputs are those of jacobi_fx_march
// (FX: resident 64-bit fixed point, EDGE: first or last sweep) or of the
// native jacobi_march, value for value.  Row r lives in slot (r - ya + 1)
// mod kRing; rows ya-1 .. yb are staged (those inside the grid).  The
// kernel runs fixed-point units through bulk_march_fx below and uses this
// one for the native FP64 path (grids with a non-finite or tiny maximum).
template <bool FX, bool EDGE>
JD void staged_march(double* ring, const double* __restrict__ u, double* __restrict__ v, i64 nx64, i64 ny, i64 x064,
                     i64 ya, i64 yb, int F, int flags, u64& rfx, double& rnat) {
  const int lane = threadIdx.x & 31;
  const int nx = (int)nx64, x0 = (int)x064;  // extents below 2^31
  const int xa = x0 + 2 * lane;
  const bool inf = EDGE && (flags & JFX_IN_F64);
  const bool outf = EDGE && (flags & JFX_OUT_F64);
  const bool c0 = xa < nx, c1 = xa + 1 < nx;
  const bool in0 = xa >= 1 && xa <= nx - 2, in1 = xa + 1 >= 1 && xa + 1 <= nx - 2;
  const int odd = nx & 1;
  const StagePlan P = stage_plan(nx, x0, lane);
  // staging cursor: next row to stage, its offset, parity and ring position
  i64 rs = ya - 1;
  i64 offs = (ya - 1) * nx64;
  int shs = odd ? (int)(rs & 1) : 0;
  int js = 0;
  auto stage_next = [&]() {
    if (rs >= 0 && rs < ny && rs <= yb)
      stage_row(P, ring + (js & (kRing - 1)) * kSlot, u + offs, shs, rs == ny - 1, nx);
    cp_async_commit();
    ++rs;
    offs += nx64;
    shs ^= odd;
    ++js;
  };
  auto own = [&](const double* sp, int sh, bool inside, double (&o)[2]) {
    o[0] = o[1] = 0.0;
    if (!inside || !c0) return;
    const double* p = sp + 2 * lane + 2 + sh;
    if (sh == 0 && c1) {
      const double2 t = *reinterpret_cast<const double2*>(p);
      o[0] = t.x;
      o[1] = t.y;
    } else {
      o[0] = p[0];
      if (c1) o[1] = p[1];
    }
  };
  auto cvt = [&](double raw) -> i64 { return inf ? fx_from(raw, F) : bits_i64(raw); };

#pragma unroll 1
  for (int j = 0; j < kRing; ++j) stage_next();
  cp_async_wait<kRing - 2>();  // rows ya-1 and ya
  __syncwarp();
  int shy = odd ? (int)(ya & 1) : 0;  // parity of row y
  double rup[2], rcur[2];
  own(ring + 0 * kSlot, shy ^ odd, ya >= 1, rup);
  own(ring + 1 * kSlot, shy, true, rcur);
  __syncwarp();
  stage_next();  // into the slot of row ya-1
  double* out = v + ya * nx64 + xa;
  int jy = 1;  // ring position of row y
#pragma unroll 1
  for (i64 y = ya; y < yb; ++y) {
    cp_async_wait<kRing - 2>();  // row y+1
    __syncwarp();
    const double* sy = ring + (jy & (kRing - 1)) * kSlot;
    const double* sn = ring + ((jy + 1) & (kRing - 1)) * kSlot;
    double rdn[2];
    own(sn, shy ^ odd, y + 1 < ny, rdn);
    const double* cs = sy + 2 * lane + 2 + shy;
    const double rl = in0 ? cs[-1] : 0.0;
    const double rr = in1 ? cs[2] : 0.0;
    const bool yint = y >= 1 && y <= ny - 2;
    const bool a0 = yint && in0, a1 = yint && in1;
    double o0, o1;
    if constexpr (FX) {
      const i64 cu0 = cvt(rcur[0]), cu1 = cvt(rcur[1]);
      const i64 s0 = (cvt(rup[0]) + cvt(rdn[0])) + (cvt(rl) + cu1);
      const i64 s1 = (cvt(rup[1]) + cvt(rdn[1])) + (cu0 + cvt(rr));
      auto bnd = [&](double raw, i64 w) -> double {
        if constexpr (!EDGE) return i64_bits(w);
        if (inf && outf) return raw;
        if (outf) return fx_to(w, F);
        return i64_bits(w);
      };
      o0 = a0 ? (outf ? fx_to(s0, F + 2) : i64_bits((s0 + 2) >> 2)) : bnd(rcur[0], cu0);
      o1 = a1 ? (outf ? fx_to(s1, F + 2) : i64_bits((s1 + 2) >> 2)) : bnd(rcur[1], cu1);
      const i64 d0 = s0 - cu0 * 4, d1 = s1 - cu1 * 4;
      const u64 ad0 = (u64)(d0 ^ (d0 >> 63)), ad1 = (u64)(d1 ^ (d1 >> 63));
      if (a0 && ad0 > rfx) rfx = ad0;
      if (a1 && ad1 > rfx) rfx = ad1;
    } else {
      const double s0 = (rup[0] + rdn[0]) + (rl + rcur[1]);
      const double s1 = (rup[1] + rdn[1]) + (rcur[0] + rr);
      const double q0 = 0.25 * s0, q1 = 0.25 * s1;
      o0 = a0 ? q0 : rcur[0];
      o1 = a1 ? q1 : rcur[1];
      double e0 = q0 - rcur[0], e1 = q1 - rcur[1];
      e0 = e0 < 0.0 ? -e0 : e0;
      e1 = e1 < 0.0 ? -e1 : e1;
      if (a0 && e0 > rnat) rnat = e0;
      if (a1 && e1 > rnat) rnat = e1;
    }
    if (c1 && shy == 0) {
      double2 t;
      t.x = o0;
      t.y = o1;
      *reinterpret_cast<double2*>(out) = t;
    } else if (c0) {
      out[0] = o0;
      if (c1) out[1] = o1;
    }
    out += nx64;
    rup[0] = rcur[0];
    rup[1] = rcur[1];
    rcur[0] = rdn[0];
    rcur[1] = rdn[1];
    shy ^= odd;
    ++jy;
    __syncwarp();
    stage_next();  // into the slot of row y
  }
  cp_async_wait<0>();  // no copy may land in the ring after the next unit starts with it
  __syncwarp();
}

// ---------------------------------------------------------------- bulk-copy march
//
// The fixed-point march of the staged variant.  A warp's unit is W = 32 CPL
// columns (CPL = 4 in intermediate sweeps of items at least 128 columns
// wide; 2 in narrower items and in the converting first and last sweeps,
// whose conversions need the registers); lane l owns
// columns x0 + CPL l .. x0 + CPL l + CPL - 1.  Rows stream through a ring of
// kRingB slots of W + 4 doubles, each slot with its own mbarrier: lane 0
// fetches row r with ONE bulk copy (cp.async.bulk) of the 16-byte-aligned
// span that covers columns [max(x0 - 1, 0), min(x0 + W, nx - 1)], counted in
// bytes on the slot's barrier.  Element x of row r lands at
// slot[x - x0 + 2 + sh], sh = (r nx) & 1, which puts the span's even start on
// an even slot index.  The field's last element, whose pair would run past
// the end of the field, goes through a register.  A row outside the grid or
// past the unit's halo row is not fetched, but lane 0 still arrives on its
// slot's barrier, so every slot completes one phase per staged row and the
// warp's running row count `gq` (kept across units) gives each wait its
// slot and parity.  Staging a row costs a few instructions on one lane, and
// the row loop handles CPL columns per lane, so the per-row bookkeeping is
// spread over 2 CPL updates.  Outputs and residual are those of
// jacobi_fx_march, value for value.  False if a wait ran out (after a
// bounded wait for the copies still in flight).  stall > 0 is a test hook:
// the warp never stages its stall-th row (counted by gq from 1).
JD void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int CPL, bool EDGE>
JD bool bulk_march_fx(double* ring, u64* bars, u32& gq, const double* __restrict__ u, double* __restrict__ v,
                      i64 nx64, int ny, int x0, int ya, int yb, int F, int flags, u64 timeout_ns, int stall, u64& rfx) {
  constexpr int W = 32 * CPL, SLOT = W + 4;
  const int lane = threadIdx.x & 31;
  const int nx = (int)nx64;
  const i64 ntot = nx64 * ny;
  const int xl = x0 + CPL * lane;  // the lane's first column
  const bool inf = EDGE && (flags & JFX_IN_F64);
  const bool outf = EDGE && (flags & JFX_OUT_F64);
  bool cin[CPL], cint[CPL];  // column inside the grid; interior column
  bool call = true, iall = true;
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
    cin[e] = xl + e < nx;
    cint[e] = xl + e >= 1 && xl + e <= nx - 2;
    call = call && cin[e];
    iall = iall && cint[e];
  }
  const bool ufast = __all_sync(0xffffffffu, iall);  // no boundary column in the unit
  const int odd = nx & 1;
  const int clo = x0 >= 1 ? x0 - 1 : 0;
  const int chi = x0 + W <= nx - 1 ? x0 + W : nx - 1;
  const u32 g0 = gq;  // running count of row ya - 1
  int rs = ya - 1;    // next row to stage
  __syncwarp();
  if (lane == 0) fence_proxy_async_smem();  // the ring's earlier generic-proxy use precedes these copies
  // the test hook: the stall-th staged row is neither fetched nor arrived
  // on, so the wait for it runs out (no row has this count otherwise)
  const u32 stall_q = stall > 0 ? (u32)(stall - 1) : 0xffffffffu;
  auto stage_next = [&]() {
    if (lane == 0 && gq != stall_q) {
      const int j = (int)(gq % kRingB);
      u64* bar = bars + j;
      double* slot = ring + j * SLOT;
      i64 es = 0, ee = 0, base = 0;
      if (rs >= 0 && rs <= yb && rs < ny) {
        const i64 rb = (i64)rs * nx64;
        base = rb + x0 - 2 - (rb & 1);  // the element at slot[0]
        es = (rb + clo) & ~1ll;
        ee = (rb + chi + 2) & ~1ll;
        if (ee > ntot) {  // the span ends at the field's odd last element
          ee = ntot - 1;
          slot[ntot - 1 - base] = __ldcg(u + ntot - 1);
        }
      }
      if (ee > es) {
        const u32 bytes = (u32)(ee - es) * 8u;
        mbar_expect_tx(bar, bytes);
        bulk_g2s(slot + (es - base), u + es, bytes, bar);
      } else {
        mbar_arrive(bar);
      }
    }
    ++rs;
    ++gq;
  };
  auto slot_of = [&](int r) -> const double* { return ring + ((g0 + (u32)(r - ya + 1)) % kRingB) * SLOT; };
  auto wait_row = [&](int r) -> bool {
    const u32 q = g0 + (u32)(r - ya + 1);
    return mbar_wait(bars + (q % kRingB), (q / kRingB) & 1u, (i64)timeout_ns);
  };
  // the lane's CPL raw words of a staged row (zero outside the grid's rows)
  auto own = [&](const double* sp, int sh, bool inside, double (&o)[CPL]) {
    if (!inside) {
#pragma unroll
      for (int e = 0; e < CPL; ++e) o[e] = 0.0;
      return;
    }
    const double* p = sp + CPL * lane + 2 + sh;
    if (sh == 0) {
#pragma unroll
      for (int e = 0; e < CPL; e += 2) {
        const double2 t = *reinterpret_cast<const double2*>(p + e);
        o[e] = t.x;
        o[e + 1] = t.y;
      }
    } else {
      o[0] = p[0];
#pragma unroll
      for (int e = 1; e + 1 < CPL; e += 2) {
        const double2 t = *reinterpret_cast<const double2*>(p + e);
        o[e] = t.x;
        o[e + 1] = t.y;
      }
      o[CPL - 1] = p[CPL - 1];
    }
  };
  auto cvt = [&](double raw) -> i64 { return inf ? fx_from(raw, F) : bits_i64(raw); };
  auto bnd = [&](double raw, i64 w) -> double {
    if constexpr (!EDGE) return i64_bits(w);
    if (inf && outf) return raw;
    if (outf) return fx_to(w, F);
    return i64_bits(w);
  };
  // bounded wait for the copies still in flight (the last kRingB staged rows)
  auto drain = [&]() {
    for (u32 q = gq - kRingB; q != gq; ++q) mbar_wait(bars + (q % kRingB), (q / kRingB) & 1u, 1000000);
  };

#pragma unroll 1
  for (int j = 0; j < kRingB; ++j) stage_next();
  if (!wait_row(ya - 1) || !wait_row(ya)) {
    drain();
    return false;
  }
  int shy = odd & ya;  // parity of row y
  double ra[CPL], rb[CPL], rc[CPL];
  own(slot_of(ya - 1), shy ^ odd, ya >= 1, ra);
  own(slot_of(ya), shy, true, rb);
  __syncwarp();
  stage_next();
  double* out = v + (i64)ya * nx64 + xl;
  int y = ya;
  bool ok = true;
  // one row: up, cur -> dn (raw words); writes row y
  auto step = [&](const double (&up)[CPL], const double (&cur)[CPL], double (&dn)[CPL]) {
    if (!ok || !wait_row(y + 1)) {
      ok = false;
      return;
    }
    own(slot_of(y + 1), shy ^ odd, y + 1 < ny, dn);
    const double* cs = slot_of(y) + CPL * lane + 2 + shy;
    const double rl = cs[-1], rr = cs[CPL];  // columns left and right of the lane's (any value outside)
    const bool yint = y >= 1 && y <= ny - 2;
    i64 c[CPL], sm[CPL];
#pragma unroll
    for (int e = 0; e < CPL; ++e) c[e] = cvt(cur[e]);
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
      const i64 w = e == 0 ? cvt(rl) : c[e - 1];
      const i64 z = e == CPL - 1 ? cvt(rr) : c[e + 1];
      sm[e] = (cvt(up[e]) + cvt(dn[e])) + (w + z);
    }
    double o[CPL];
    if (!EDGE && ufast && yint) {
#pragma unroll
      for (int e = 0; e < CPL; ++e) {
        o[e] = i64_bits((sm[e] + 2) >> 2);
        const i64 d = sm[e] - c[e] * 4;
        const u64 ad = (u64)(d ^ (d >> 63));  // |d| (one less if negative)
        rfx = ad > rfx ? ad : rfx;
      }
    } else {
#pragma unroll
      for (int e = 0; e < CPL; ++e) {
        const bool a = yint && cint[e];
        o[e] = a ? (outf ? fx_to(sm[e], F + 2) : i64_bits((sm[e] + 2) >> 2)) : bnd(cur[e], c[e]);
        const i64 d = sm[e] - c[e] * 4;
        const u64 ad = a ? (u64)(d ^ (d >> 63)) : 0ull;
        rfx = ad > rfx ? ad : rfx;
      }
    }
    if (call && shy == 0) {
#pragma unroll
      for (int e = 0; e < CPL; e += 2) {
        double2 t;
        t.x = o[e];
        t.y = o[e + 1];
        *reinterpret_cast<double2*>(out + e) = t;
      }
    } else {
#pragma unroll
      for (int e = 0; e < CPL; ++e)
        if (cin[e]) out[e] = o[e];
    }
    out += nx64;
    shy ^= odd;
    ++y;
    __syncwarp();
    stage_next();  // into the slot of the row just finished
  };
#pragma unroll 1
  while (ok && y + 2 < yb) {
    step(ra, rb, rc);
    step(rb, rc, ra);
    step(rc, ra, rb);
  }
  if (y < yb) step(ra, rb, rc);
  if (y < yb) step(rb, rc, ra);
  if (!ok) drain();
  return ok;
}

// ---------------------------------------------------------------- register march

template <bool EDGE>
JD void register_units(const JBGrid& G, const double* src, double* dst, i64 x0, i64 ya, i64 yb, int F, int flags,
                       u64& rfx, double& rnat) {
  if (G.nx % 2 == 0) {
    if (F >= 0) jacobi_fx_march<2, true, EDGE>(src, dst, G.nx, G.ny, x0 + 2 * (threadIdx.x & 31), ya, yb, F, flags, rfx);
    else jacobi_march<double, 2, JM_NATIVE, true>(src, dst, G.nx, G.ny, x0 + 2 * (threadIdx.x & 31), ya, yb, F, rnat);
  } else {
    for (int half = 0; half < 2; ++half) {
      const i64 xl = x0 + 32 * half + (threadIdx.x & 31);
      if (F >= 0) jacobi_fx_march<1, true, EDGE>(src, dst, G.nx, G.ny, xl, ya, yb, F, flags, rfx);
      else jacobi_march<double, 1, JM_NATIVE, true>(src, dst, G.nx, G.ny, xl, ya, yb, F, rnat);
    }
  }
}

// ---------------------------------------------------------------- the persistent kernel
//
// A CTA is 8 compute warps and one scheduler warp, which hand items over
// through two mailbox slots on mbarriers: the scheduler fills slot i & 1
// with the CTA's i-th item and arrives on the slot's `ready` barrier; each
// compute warp runs its unit of item i, arrives on the slot's `done` barrier
// and goes straight on to item i + 1 once that is published, so warps that
// finish early do not wait for the slowest one.  The scheduler resolves item
// i + 1 (ticket, item, grid, and the five dependency counters polled by five
// lanes with relaxed loads in parallel) while item i runs.  It signals a
// finished item (fence, release store of its counter) as soon as the item's
// `done` barrier completes — also from inside its wait for the next item's
// dependencies — so it never blocks while it holds a finished, unsignalled
// item: the smallest unfinished ticket is always some CTA's item in progress
// or a published item whose dependencies are all signalled, and the launch
// cannot deadlock.  A slot is refilled only after every compute warp has
// finished the item it held two steps before, so no warp can miss a phase.

constexpr int kCTA = kThreads + 32;  // compute warps + the scheduler warp

JD unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The item the compute warps run next, with its grid's descriptor and
// fixed-point scale, so they load nothing but field data.
struct Mailbox {
  int stop;
  int s;  // sweep
  int F;  // fraction bits of the grid's fixed-point form, -1: native FP64
  int first;  // the item is the launch's first ticket (the row-stall test hook's warp)
  JBItem it;
  JBGrid G;
};

struct BatchShared {
  Mailbox mb[2];
  u64 ready[2];              // count 1: the scheduler filled the slot
  u64 done[2];               // count kWarps: every compute warp finished the slot's item
  u64 rows[kWarps][kRingB];  // count 1 + bytes: a compute warp's staged row (bulk-copy march)
};

// Scheduler-side view of one ticket.
struct Tk {
  long long t;
  int s, self, F;
  int dep;  // this lane's counter (lanes 0..4: self, up, down, left, right), -1 if none
  JBItem it;
  JBGrid G;
};

// Decodes ticket t (all lanes of the scheduler warp; grp is the group cursor).
JD bool decode(const JBatchParams& bp, long long t, int& grp, int base_item, Tk& k) {
  k.t = t;
  if (t >= bp.total_tickets) return false;
  while (grp + 1 < bp.ngroups && t >= (long long)(bp.groups[grp + 1].item_begin - base_item) * bp.nsweeps) ++grp;
  const JBGroup Q = bp.groups[grp];
  const long long lt = t - (long long)(Q.item_begin - base_item) * bp.nsweeps;
  k.s = (int)(lt / Q.nitems);
  k.it = bp.items[Q.item_begin + (int)(lt % Q.nitems)];
  const JBItem it = k.it;
  k.G = bp.grids[it.g];
  const JBGrid& G = k.G;
  k.F = bp.maxwords ? fx_frac_bits(bp.maxwords[it.g]) : -1;
  k.self = G.item_base + it.b * G.nc + it.c;
  const int lane = threadIdx.x & 31;
  k.dep = -1;
  if (lane == 0) k.dep = k.self;
  if (lane == 1 && it.b > 0) k.dep = k.self - G.nc;
  if (lane == 2 && it.b + 1 < G.nb) k.dep = k.self + G.nc;
  if (lane == 3 && it.c > 0) k.dep = k.self - 1;
  if (lane == 4 && it.c + 1 < G.nc) k.dep = k.self + 1;
  return true;
}

// One round of dependency loads: true when all five counters reach k.s.
JD bool deps_ready(const JBatchParams& bp, const Tk& k) {
  const bool ok = k.dep < 0 || ld_relaxed_u32(bp.done + k.dep) >= (unsigned)k.s;
  return __all_sync(0xffffffffu, ok);
}

// What the scheduler keeps of an item after publishing it: enough to signal it.
struct Sig {
  long long t;
  int s, self;
};

JD Sig sig_of(const Tk& k) { return Sig{k.t, k.s, k.self}; }

JD void signal_done(const JBatchParams& bp, const Sig& k) {
  if ((threadIdx.x & 31) == 0 && k.t != bp.stall_ticket) {
    __threadfence();
    st_release_u32(bp.done + k.self, (unsigned)(k.s + 1));
  }
  __syncwarp();
}

// Polls the dependencies of `nxt` until they are ready; meanwhile signals
// `cur` (the CTA's item i) as soon as its done barrier completes.  False if
// the batch is abandoned (this wait ran out, or another CTA's did).
JD bool deps_wait_serving(const JBatchParams& bp, const Tk& nxt, const Sig& cur, BatchShared& sh, int i, bool& sig) {
  const u64 t0 = globaltimer_ns();
  for (;;) {
    if (deps_ready(bp, nxt)) return true;
    if (!sig && mbar_try(&sh.done[i & 1], (u32)((i >> 1) & 1))) {
      signal_done(bp, cur);
      sig = true;
    }
    int bad = 0;
    if ((threadIdx.x & 31) == 0) {
      bad = ld_relaxed_i32(bp.status) != 0;
      if (!bad && globaltimer_ns() - t0 > bp.timeout_ns) {
        atomicCAS(bp.status, 0, JACC_ERR_TIMEOUT);
        bad = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, bad, 0)) return false;
    __nanosleep(64);
  }
}

// Fills slot i & 1 and marks it ready (all lanes of the scheduler warp).
JD void publish(BatchShared& sh, int i, int stop, const Tk& k) {
  Mailbox& mb = sh.mb[i & 1];
  if ((threadIdx.x & 31) == 0) {
    mb.stop = stop;
    mb.first = k.t == 0;
    mb.s = k.s;
    mb.F = k.F;
    mb.it = k.it;
    mb.G = k.G;
  }
  __threadfence();  // acquire side of the relaxed dependency loads (every lane)
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&sh.ready[i & 1]);
}

template <int STAGED>
__global__ void __launch_bounds__(kCTA, STAGED ? 2 : 3) jacc_k_batched(JBatchParams bp) {
  extern __shared__ __align__(16) double s_ring[];
  __shared__ __align__(16) BatchShared sh;
  const int warp = threadIdx.x >> 5;
  const int base_item = bp.groups[0].item_begin;
  if (threadIdx.x == 0) {
    mbar_init(&sh.ready[0], 1);
    mbar_init(&sh.ready[1], 1);
    mbar_init(&sh.done[0], kWarps);
    mbar_init(&sh.done[1], kWarps);
    for (int w = 0; w < kWarps; ++w)
      for (int j = 0; j < kRingB; ++j) mbar_init(&sh.rows[w][j], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (warp == kWarps) {
    // ------------------------------------------------------------ scheduler warp
    int grp = 0;
    Sig cur;
    bool live;
    {
      Tk first;
      long long t = 0;
      if ((threadIdx.x & 31) == 0) t = (long long)atomicAdd(bp.ticket, 1ull);
      t = __shfl_sync(0xffffffffu, t, 0);
      bool none_pending = true;  // no item of this CTA is running yet
      live = decode(bp, t, grp, base_item, first) && deps_wait_serving(bp, first, sig_of(first), sh, 0, none_pending);
      publish(sh, 0, live ? 0 : 1, first);
      cur = sig_of(first);
    }
    for (int i = 0; live; ++i) {
      // item i runs; resolve item i + 1, serving item i's completion meanwhile
      Tk nxt;
      long long tn = 0;
      if ((threadIdx.x & 31) == 0) tn = (long long)atomicAdd(bp.ticket, 1ull);
      tn = __shfl_sync(0xffffffffu, tn, 0);
      bool sig = false;
      const bool has = decode(bp, tn, grp, base_item, nxt);
      const bool ok = has && deps_wait_serving(bp, nxt, cur, sh, i, sig);
      publish(sh, i + 1, ok ? 0 : 1, nxt);  // slot (i+1) & 1 held item i-1, finished before cur was signalled
      if (!sig) {
        if (!mbar_wait(&sh.done[i & 1], (u32)((i >> 1) & 1), (i64)bp.timeout_ns)) {
          if ((threadIdx.x & 31) == 0) atomicCAS(bp.status, 0, JACC_ERR_TIMEOUT);
          break;
        }
        signal_done(bp, cur);
      }
      cur = sig_of(nxt);
      live = ok;
    }
    return;
  }
  // -------------------------------------------------------------- compute warps
  double* ring = s_ring + warp * kRingWords;
  u32 gq = 0;  // rows this warp has staged through its bulk-copy ring
  bool stall_armed = false;
  for (int i = 0;; ++i) {
    if (!mbar_wait(&sh.ready[i & 1], (u32)((i >> 1) & 1), (i64)bp.timeout_ns)) {
      if ((threadIdx.x & 31) == 0) atomicCAS(bp.status, 0, JACC_ERR_TIMEOUT);
      break;
    }
    const Mailbox& mb = sh.mb[i & 1];
    if (mb.stop) break;
    const int s = mb.s;
    const int F = mb.F;
    const JBItem it = mb.it;
    const JBGrid G = mb.G;
    // the row-stall test hook acts in warp 0 of the CTA that runs the first
    // ticket (its first item), which counts its staged rows from there on
    if (mb.first && warp == 0) stall_armed = true;
    const double* src = (s & 1) ? G.u[1] : G.u[0];
    double* dst = (s & 1) ? G.u[0] : G.u[1];
    const int flags = (s == 0 ? JFX_IN_F64 : 0) | (s == bp.nsweeps - 1 ? JFX_OUT_F64 : 0);
    // this warp's unit of the item: a strip of Wu columns (128 in the
    // bulk-copy march of intermediate sweeps of items at least 128 wide, else
    // 64) of a slice of its rows
    const int Wu = (STAGED && F >= 0 && G.cols >= 128 && !flags) ? 128 : 64;
    const int across = G.cols / Wu;
    const int slices = kWarps / across;
    const i64 x0 = (i64)it.c * G.cols + Wu * (warp % across);
    const i64 r0 = (i64)it.b * G.rows;
    const i64 r1 = r0 + G.rows < G.ny ? r0 + G.rows : G.ny;
    const i64 h = (r1 - r0 + slices - 1) / slices;
    const i64 ya = r0 + (warp / across) * h;
    const i64 yb = ya + h < r1 ? ya + h : r1;
    u64 rfx = 0;
    double rnat = 0.0;
    // after a wait anywhere ran out the batch is abandoned: items still
    // handed out are passed through without work
    if (x0 < G.nx && ya < yb && ld_relaxed_i32(bp.status) == 0) {
      if constexpr (STAGED) {
        if (F >= 0) {
          const int nyi = (int)G.ny, x0i = (int)x0, yai = (int)ya, ybi = (int)yb;
          const u64 tmo = bp.timeout_ns;
          const int stall = stall_armed ? bp.stall_row : 0;
          u64* bars = sh.rows[warp];
          bool ok;
          if (Wu == 128)
            ok = bulk_march_fx<4, false>(ring, bars, gq, src, dst, G.nx, nyi, x0i, yai, ybi, F, flags, tmo, stall, rfx);
          else if (flags)
            ok = bulk_march_fx<2, true>(ring, bars, gq, src, dst, G.nx, nyi, x0i, yai, ybi, F, flags, tmo, stall, rfx);
          else
            ok = bulk_march_fx<2, false>(ring, bars, gq, src, dst, G.nx, nyi, x0i, yai, ybi, F, flags, tmo, stall, rfx);
          if (!ok && (threadIdx.x & 31) == 0) atomicCAS(bp.status, 0, JACC_ERR_TIMEOUT);
        } else {
          staged_march<false, false>(ring, src, dst, G.nx, G.ny, x0, ya, yb, F, flags, rfx, rnat);
        }
      } else {
        if (flags) register_units<true>(G, src, dst, x0, ya, yb, F, flags, rfx, rnat);
        else register_units<false>(G, src, dst, x0, ya, yb, F, flags, rfx, rnat);
      }
    }
    // the warp's residual maximum: one atomic per warp (non-negative doubles
    // order like their bit patterns)
    const u64 bits = warp_max_u64(F >= 0 ? dbits(fx_to_u(rfx, F + 2)) : dbits(rnat));
    if ((threadIdx.x & 31) == 0 && bp.resid)
      atomicMax(reinterpret_cast<unsigned long long*>(bp.resid + (i64)it.g * bp.nsweeps + s), (unsigned long long)bits);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&sh.done[i & 1]);
  }
}

// Max |u0| per grid: blockIdx.y = grid.
__global__ void __launch_bounds__(256) jacc_k_maxabs_batched(const JBGrid* grids, u64* maxwords) {
  const JBGrid G = grids[blockIdx.y];
  const i64 n = G.nx * G.ny;
  const double* u = G.u[0];
  u64 m = 0;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const u64 a = dbits(__ldg(u + i)) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
  }
  m = warp_max_u64(m);
  __shared__ u64 red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    u64 w = threadIdx.x < 8 ? red[threadIdx.x] : 0ull;
    w = warp_max_u64(w);
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long*>(maxwords + blockIdx.y), (unsigned long long)w);
  }
}

}  // namespace

namespace jacc {

cudaError_t batched_occupancy(int staged, int* blocks_per_sm) {
  if (staged) {
    cudaError_t e = cudaFuncSetAttribute(jacc_k_batched<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, jacc_k_batched<1>, kCTA, kStagedSmem);
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, jacc_k_batched<0>, kCTA, 0);
}

cudaError_t launch_batched(const JBatchParams& bp, int nctas, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(kCTA);
  cfg.dynamicSmemBytes = bp.staged ? kStagedSmem : 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (bp.staged) return cudaLaunchKernelEx(&cfg, jacc_k_batched<1>, bp);
  return cudaLaunchKernelEx(&cfg, jacc_k_batched<0>, bp);
}

cudaError_t launch_maxabs_batched(const JBGrid* d_grids, int ngrids, i64 max_n, u64* maxwords, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(maxwords, 0, sizeof(u64) * (size_t)ngrids, s);
  if (e != cudaSuccess) return e;
  i64 bx = (max_n + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  jacc_k_maxabs_batched<<<dim3((unsigned)bx, (unsigned)ngrids), 256, 0, s>>>(d_grids, maxwords);
  return cudaGetLastError();
}

}  // namespace jacc
