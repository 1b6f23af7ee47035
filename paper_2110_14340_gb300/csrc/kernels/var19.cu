// var19.cu - the variable-coefficient 19-point Jacobi step (FP32): the
// iteration of the paper's Himeno workload (§5.2), written from the stencil's
// definition.  For each interior point, p(dx,dy,dz) the neighbour at an offset
// and a0..wrk1, bnd the twelve coefficient fields at the point:
//   s0 = a0 p(+x) + a1 p(+y) + a2 p(+z)
//      + b0 (p(+x+y) - p(+x-y) - p(-x+y) + p(-x-y))
//      + b1 (p(+y+z) - p(-y+z) - p(+y-z) + p(-y-z))
//      + b2 (p(+x+z) - p(-x+z) - p(+x-z) + p(-x-z))
//      + c0 p(-x) + c1 p(-y) + c2 p(-z) + wrk1
//   ss = (s0 a3 - p) bnd,   v = p + omega ss,   residual = sum of ss^2.
// Boundary points keep p.
//
// The iterate p is staged plane by plane in shared memory by bulk copies
// (the same scheme as the 7-point kernel: full/empty mbarriers, bounded
// waits, warp 0 issues one copy per staged row); a step reads planes z-1, z
// and z+1 from the ring.  The twelve coefficient fields are read once each,
// straight from global memory with 16-byte loads issued at the start of the
// step, so their latency overlaps the shared-memory work.  A CTA of 32 x 4
// threads owns a 128 x 4 tile (one 16-byte column per thread) and marches
// ZC planes.  HBM bytes per update: 13 reads + 1 write of 4 bytes = 56.
#include <cuda_runtime.h>

#include "../host/jacc_internal.h"
#include "jacc_device.cuh"

namespace {

JD float fmul(float a, float b) { return __fmul_rn(a, b); }
JD float fadd(float a, float b) { return __fadd_rn(a, b); }
JD float fsub(float a, float b) { return __fsub_rn(a, b); }

constexpr int BX = 32, BY = 4, V = 4, ZC = 40;  // 40 planes: 125.3 against 124.2 GLUP/s with 64 (512 x 512 x 1024)
constexpr int TW = BX * V, TH = BY;
constexpr int W = TW + 2 * V, R = TH + 2;
constexpr int S = 6;                 // stages: planes z-1, z, z+1 plus prefetch
constexpr int NW = BX * BY / 32;

struct alignas(128) Smem {
  float st[S][R][W];  // staged row r <-> grid row by0 - 1 + r, slot i <-> column bx0 - V + i
  u64 full[S];
  u64 empty[S];
};

// Warp 0 requests plane zg into stage s (rows and columns clipped to the grid).
JD void issue_plane(Smem& sm, int s, const float* __restrict__ u, const JParams& p, i64 zg, i64 bx0, i64 by0) {
  const i64 nx = p.nx, ny = p.ny;
  const int lane = threadIdx.x & 31;
  const i64 c0 = bx0 - V < 0 ? 0 : bx0 - V;
  const i64 c1 = bx0 + TW + V > nx ? nx : bx0 + TW + V;
  const i64 r0 = by0 - 1 < 0 ? 0 : by0 - 1;
  const i64 r1 = by0 + TH + 1 > ny ? ny : by0 + TH + 1;
  const u32 row_bytes = (u32)((c1 - c0) * 4);
  if (lane == 0) mbar_expect_tx(&sm.full[s], row_bytes * (u32)(r1 - r0));
  __syncwarp();
  for (i64 y = r0 + lane; y < r1; y += 32)
    bulk_g2s(&sm.st[s][y - (by0 - 1)][c0 - (bx0 - V)], u + (zg * ny + y) * nx + c0, row_bytes, &sm.full[s]);
}

__global__ void __launch_bounds__(BX * BY) jacc_k_var19(const float* __restrict__ u, float* __restrict__ v,
                                                         JParams p, double* resid) {
  __shared__ Smem sm;
  const i64 nx = p.nx, ny = p.ny, nz = p.nz, sz = nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const bool warp0 = tid < 32;
  const i64 bx0 = (i64)blockIdx.x * TW, by0 = (i64)blockIdx.y * TH;
  const i64 x0 = bx0 + (i64)tx * V, y = by0 + ty;
  const bool act = x0 < nx && y < ny;
  unsigned inm = 0;  // interior columns of the thread's 4 points
#pragma unroll
  for (int e = 0; e < V; ++e)
    if (y >= 1 && y <= ny - 2 && x0 + e >= 1 && x0 + e <= nx - 2) inm |= 1u << e;
  const i64 cz0 = (i64)blockIdx.z * ZC;
  const i64 cz1 = (cz0 + ZC < nz) ? cz0 + ZC : nz;
  const i64 z0 = cz0 < 1 ? 1 : cz0;
  const i64 z1 = cz1 > nz - 1 ? nz - 1 : cz1;
  float hi = 0.0f, lo = 0.0f;
  if (z0 >= z1) {  // a chunk holding only a boundary plane (block-uniform)
    if (act)
      for (i64 z = cz0; z < cz1; ++z) {
        float t[V];
        ldv<float, V>(u + z * sz + y * nx + x0, t);
        stv<float, V>(v + z * sz + y * nx + x0, t);
      }
    block_sum_to<BX * BY>(0.0, resid);
    return;
  }
  const int L = (int)(z1 - z0) + 2;  // staged planes z0-1 .. z1
  const i64 lim = p.timeout_ns;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], NW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  int issued = 0, consumed = 0;  // warp 0: planes requested, planes waited for
  if (warp0)
    for (; issued < S && issued < L; ++issued) issue_plane(sm, issued, u, p, z0 - 1 + issued, bx0, by0);
  // ring cursors: cn = next plane to wait for; cq = plane whose stage warp 0 refills next
  int cn_s = 0, cq_s = 0;
  u32 cn_ph = 0, cq_ph = 0;
  auto adv = [&](int& s, u32& ph) {
    if (++s == S) {
      s = 0;
      ph ^= 1u;
    }
  };
  auto wait_next = [&]() -> bool {
    if (!mbar_wait(&sm.full[cn_s], cn_ph, lim)) return false;
    ++consumed;
    return true;
  };
  bool ok = wait_next();  // plane z0 - 1
  int sm1 = cn_s;
  adv(cn_s, cn_ph);
  if (ok) ok = wait_next();  // plane z0
  int s0 = cn_s;
  adv(cn_s, cn_ph);
  const float omega = (float)p.c0;
  const float* const* cf = p.cf;
  const i64 off0 = y * nx + x0;
  if (ok && cz0 == 0 && act) {  // boundary plane 0 from the staged plane z0 - 1 = 0
    float t[V];
    lds_vec(&sm.st[sm1][ty + 1][V + V * tx], t);
    stv<float, V>(v + off0, t);
  }
  for (int j = 1; ok && j <= L - 2; ++j) {
    const i64 off = (z0 - 1 + j) * sz + off0;
    // the twelve coefficients of the row, issued before any wait
    float c[12][V];
#pragma unroll
    for (int f = 0; f < 12; ++f) {
#pragma unroll
      for (int e = 0; e < V; ++e) c[f][e] = 0.0f;
      if (act) ldv<float, V>(cf[f] + off, c[f]);
    }
    if (!wait_next()) {
      ok = false;
      break;
    }
    const int sp1 = cn_s;
    adv(cn_s, cn_ph);
    const float(*Pm)[W] = sm.st[sm1];
    const float(*P0)[W] = sm.st[s0];
    const float(*Pp)[W] = sm.st[sp1];
    const int cx = V + V * tx;  // slot of the thread's first column
    float r0m[V + 2], r00[V + 2], r0p[V + 2], rm0[V + 2], rp0[V + 2];
    float rmm[V], rmp[V], rpm[V], rpp[V];
    lds_row<float, V>(&P0[ty][cx], r0m);
    lds_row<float, V>(&P0[ty + 1][cx], r00);
    lds_row<float, V>(&P0[ty + 2][cx], r0p);
    lds_row<float, V>(&Pm[ty + 1][cx], rm0);
    lds_row<float, V>(&Pp[ty + 1][cx], rp0);
    lds_vec(&Pm[ty][cx], rmm);
    lds_vec(&Pm[ty + 2][cx], rmp);
    lds_vec(&Pp[ty][cx], rpm);
    lds_vec(&Pp[ty + 2][cx], rpp);
    float out[V];
    float g = 0.0f;
#pragma unroll
    for (int e = 0; e < V; ++e) {
      // every product and sum rounded as written (no contraction into
      // fused multiply-adds): the step is the stencil's definition evaluated
      // left to right in IEEE FP32, term by term
      const float pc = r00[e + 1];
      float s = fadd(fadd(fmul(c[0][e], r00[e + 2]), fmul(c[1][e], r0p[e + 1])), fmul(c[2][e], rp0[e + 1]));
      s = fadd(s, fmul(c[4][e], fadd(fsub(fsub(r0p[e + 2], r0m[e + 2]), r0p[e]), r0m[e])));
      s = fadd(s, fmul(c[5][e], fadd(fsub(fsub(rpp[e], rpm[e]), rmp[e]), rmm[e])));
      s = fadd(s, fmul(c[6][e], fadd(fsub(fsub(rp0[e + 2], rp0[e]), rm0[e + 2]), rm0[e])));
      s = fadd(fadd(fadd(fadd(s, fmul(c[7][e], r00[e])), fmul(c[8][e], r0m[e + 1])), fmul(c[9][e], rm0[e + 1])),
               c[10][e]);
      const float ss = fmul(fsub(fmul(s, c[3][e]), pc), c[11][e]);
      const bool in = (inm >> e) & 1u;
      out[e] = in ? fadd(pc, fmul(omega, ss)) : pc;
      g += in ? ss * ss : 0.0f;
    }
    if (act) stv<float, V>(v + off, out);
    two_sum_acc(hi, lo, g);
    // plane j-1 is no longer needed: release it; warp 0 refills the stage of
    // plane j-2, which every warp released one step ago
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&sm.empty[sm1]);
    if (j >= 2) {
      if (warp0 && issued < L) {
        if (!mbar_wait(&sm.empty[cq_s], cq_ph, lim)) {
          ok = false;
          break;
        }
        issue_plane(sm, cq_s, u, p, z0 - 1 + issued, bx0, by0);
        ++issued;
      }
      adv(cq_s, cq_ph);
    }
    sm1 = s0;
    s0 = sp1;
    if (j == L - 2 && cz1 == nz && act) {  // boundary plane nz-1 = staged plane L-1
      float t[V];
      lds_vec(&sm.st[sp1][ty + 1][V + V * tx], t);
      stv<float, V>(v + (nz - 1) * sz + off0, t);
    }
  }
  if (!ok) {
    if (p.status) atomicExch(p.status, JACC_DEV_TIMEOUT);
    if (warp0)
      for (int j = consumed; j < issued; ++j) mbar_wait(&sm.full[j % S], (u32)((j / S) & 1), lim);
  }
  block_sum_to<BX * BY>((double)hi + (double)lo, resid);
}

}  // namespace

namespace jacc {

void var19_geometry(long long nx, long long ny, long long nz, dim3* grid, dim3* block) {
  *grid = dim3((unsigned)((nx + TW - 1) / TW), (unsigned)((ny + TH - 1) / TH), (unsigned)((nz + ZC - 1) / ZC));
  *block = dim3(BX, BY, 1);
}

cudaError_t launch_var19(const float* u, float* v, const JParams& p, double* resid, dim3 grid, dim3 block,
                         cudaStream_t s) {
  jacc_k_var19<<<grid, block, 0, s>>>(u, v, p, resid);
  return cudaGetLastError();
}

}  // namespace jacc
