// box27_tb2.cu - two sweeps of the periodic 27-point FP32 stencil per launch
// (temporal blocking, T = 2), staged in shared memory.
//
// One CTA owns an output tile of 128 x 16 points and marches a chunk of z
// planes.  Input planes (with a halo of 8 columns and 2 rows, periodic
// images included) arrive by bulk copies into a ring of 4 stages on
// mbarriers, as in the single-sweep staged kernel.  Stage 1 computes sweep 1
// over the tile plus a 1-point halo in x (4 columns, for 16-byte vectors) and
// y, from each input plane: per point the plane terms A = wf c + we f + wc g
// and B = w0 c + wf f + we g (c the point, f its 4 in-plane faces, g its 4
// in-plane diagonals), and sweep-1 value of plane z-1 = A(z-2) + B(z-1) + A(z),
// kept as a running P = A(z-2) + B(z-1) per point in registers.  Each
// sweep-1 plane goes to a shared-memory plane (two, alternating), which stage
// 2 reads the same way to form sweep 2 of the plane behind it and write it
// to memory.  One barrier per plane separates the stages.  The per-point
// arithmetic is the single-sweep staged kernel's, in the same order, so two
// sweeps here give the bits of two single sweeps; HBM traffic is 8 bytes per
// point per two sweeps.
#include <cuda_runtime.h>

#include "../host/jacc_internal.h"
#include "jacc_device.cuh"

namespace {

constexpr int QX = 32, RP = 8;            // output tile: 32 quads x 8 row pairs = 128 x 16 points
constexpr int TW = 4 * QX, TH = 2 * RP;
constexpr int U1X = QX + 2, U1Y = RP + 1;  // stage-1 units: 34 x 9 (136 x 18 points)
constexpr int W2 = TW + 8, R2 = TH + 2;    // sweep-1 plane: columns bx0-4 .., rows by0-1 ..
constexpr int W1 = TW + 16, R1 = TH + 4;   // input plane: columns bx0-8 .., rows by0-2 ..
constexpr int NT = 320;                    // threads: 306 stage-1 units, 256 stage-2 units
constexpr int NW = NT / 32;
constexpr int S = 4;                       // input stages
constexpr int ZC = 64;                     // output planes per CTA
static_assert(U1X * U1Y <= NT && QX * RP <= NT, "units per CTA");
static_assert(R1 <= 32, "one row per lane of warp 0");

struct alignas(128) Tb2Smem {
  float in[S][R1][W1];
  float s1[2][R2][W2];
  u64 full[S];
  u64 empty[S];
};

// Plane terms of a 4 x 2 unit whose points start at `p` (row stride
// `stride`): rows -1 .. 2 and columns -1 .. 4 around it are read.  The
// arithmetic of box27s_terms.
JD void tb2_terms(const float* p, int stride, float w0, float wf, float we, float wc, float (&A)[2][4],
                  float (&B)[2][4]) {
  float r[4][6];
#pragma unroll
  for (int k = 0; k < 4; ++k) lds_row<float, 4>(p + (k - 1) * stride, r[k]);
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

// Warp 0 requests input plane zg into stage s: lane 0 posts the byte count,
// lane r copies staged row r (row (by0 - 2 + r) mod ny), as one bulk copy or
// several where its columns (bx0 - 8 + i) mod nx wrap around.
JD void tb2_issue(Tb2Smem& sm, int s, const float* __restrict__ u, i64 nx, i64 ny, i64 zg, i64 bx0, i64 by0,
                  int weff) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_expect_tx(&sm.full[s], (u32)(R1 * weff * 4));
  __syncwarp();
  if (lane < R1) {
    i64 yg = (by0 - 2 + lane) % ny;
    if (yg < 0) yg += ny;
    const float* row = u + (zg * ny + yg) * nx;
    float* dst = &sm.in[s][lane][0];
    i64 c = (bx0 - 8) % nx;
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

__global__ void __launch_bounds__(NT, 2) jacc_k_box27_tb2s(const float* __restrict__ u, float* __restrict__ v,
                                                           JParams p, double* resid, const u64* maxword, int flags) {
  (void)maxword;
  (void)flags;
  griddep_wait();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Tb2Smem& sm = *reinterpret_cast<Tb2Smem*>(smem_raw);
  const i64 nx = p.nx, ny = p.ny, nz = p.nz, sz = nx * ny;
  const int t = threadIdx.x;
  const bool warp0 = t < 32;
  const i64 bx0 = (i64)blockIdx.x * TW, by0 = (i64)blockIdx.y * TH;
  const i64 z0 = (i64)blockIdx.z * ZC;
  const i64 z1 = (z0 + ZC < nz) ? z0 + ZC : nz;
  const int L = (int)(z1 - z0) + 4;  // input planes z0-2 .. z1+1
  const int weff = (int)((nx - bx0 < TW) ? nx - bx0 : TW) + 16;
  const i64 lim = p.timeout_ns;
  const bool stall_cta = p.stall_plane >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  if (t == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], NW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  auto plane_z = [&](int j) {
    i64 z = (z0 - 2 + j) % nz;
    return z < 0 ? z + nz : z;
  };
  auto request = [&](int j, int s) {
    if (!(stall_cta && j == p.stall_plane)) tb2_issue(sm, s, u, nx, ny, plane_z(j), bx0, by0, weff);
  };
  int issued = 0, consumed = 0;
  if (warp0)
    for (; issued < S && issued < L; ++issued) request(issued, issued);

  const float w0 = (float)p.c0, wf = (float)p.c1, we = (float)p.c2, wc = (float)p.c3;
  // stage-1 unit: columns bx0-4+4ux .., rows by0-1+2uy ..
  const bool has1 = t < U1X * U1Y;
  const int ux = t % U1X, uy = t / U1X;
  // stage-2 unit: columns bx0+4tx .., rows by0+2ty ..
  const bool has2 = t < QX * RP;
  const int tx = t % QX, ty = t / QX;
  const i64 ox = bx0 + 4 * tx, oy = by0 + 2 * ty;
  const bool ax = has2 && ox < nx, ay0 = ax && oy < ny, ay1 = ax && oy + 1 < ny;
  float* vo = v + oy * nx + ox;
  float hi = 0.0f, lo = 0.0f;
  float P1[2][4], A1[2][4], P2[2][4], A2[2][4];
#pragma unroll
  for (int yy = 0; yy < 2; ++yy)
#pragma unroll
    for (int e = 0; e < 4; ++e) P1[yy][e] = A1[yy][e] = P2[yy][e] = A2[yy][e] = 0.0f;
  int cn_s = 0, cq_s = 0;
  u32 cn_ph = 0, cq_ph = 0;
  auto adv = [&](int& s, u32& ph) {
    if (++s == S) {
      s = 0;
      ph ^= 1u;
    }
  };
  bool ok = true, refill_ok = true;
  for (int j = 0; j < L; ++j) {
    // ---- stage 1: input plane j (z0-2+j) -> sweep-1 plane j-1 (z0-3+j)
    const bool got = mbar_wait(&sm.full[cn_s], cn_ph, lim);
    if (got && has1) {
      float A[2][4], B[2][4];
      tb2_terms(&sm.in[cn_s][2 * uy + 1][4 * ux + 4], W1, w0, wf, we, wc, A, B);
      if (j >= 2) {
        float o[2][4];
#pragma unroll
        for (int yy = 0; yy < 2; ++yy)
#pragma unroll
          for (int e = 0; e < 4; ++e) o[yy][e] = P1[yy][e] + A[yy][e];
        float* dst = &sm.s1[(j - 1) & 1][2 * uy][4 * ux];
        sts_row<float, 4>(dst, o[0]);
        sts_row<float, 4>(dst + W2, o[1]);
      }
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          P1[yy][e] = A1[yy][e] + B[yy][e];
          A1[yy][e] = A[yy][e];
        }
    }
    __syncwarp();
    if ((t & 31) == 0) mbar_arrive(&sm.empty[cn_s]);
    adv(cn_s, cn_ph);
    if (got) ++consumed;
    if (j >= 1) {  // refill the stage of plane j-1 (released one step ago)
      if (warp0 && issued < L && refill_ok) {
        // plane `issued` goes to stage issued % S == cq_s; after a wait that
        // ran out no further plane is requested, so that mapping holds for
        // every copy in flight
        if (mbar_wait(&sm.empty[cq_s], cq_ph, lim)) {
          request(issued, cq_s);
          ++issued;
        } else {
          refill_ok = false;
        }
      }
      adv(cq_s, cq_ph);
    }
    // sweep-1 plane j-1 complete (two planes alternate, so one barrier per
    // plane also keeps stage 1 from overwriting what stage 2 reads); a wait
    // that ran out in any thread ends the CTA's march for all of them
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    // ---- stage 2: sweep-1 plane k = j-1 -> sweep-2 plane k-1 (z0-4+j)
    if (j >= 2 && has2) {
      float A[2][4], B[2][4];
      tb2_terms(&sm.s1[(j - 1) & 1][2 * ty + 1][4 * tx + 4], W2, w0, wf, we, wc, A, B);
      if (j >= 4) {
        float o[2][4];
#pragma unroll
        for (int yy = 0; yy < 2; ++yy)
#pragma unroll
          for (int e = 0; e < 4; ++e) o[yy][e] = P2[yy][e] + A[yy][e];
        const i64 z = z0 - 4 + j;
        float* q = vo + z * sz;
        if (ay0) stv<float, 4>(q, o[0]);
        if (ay1) stv<float, 4>(q + nx, o[1]);
        if (resid) {
          const float t0 = ay0 ? (o[0][0] + o[0][1]) + (o[0][2] + o[0][3]) : 0.0f;
          const float t1 = ay1 ? (o[1][0] + o[1][1]) + (o[1][2] + o[1][3]) : 0.0f;
          two_sum_acc(hi, lo, t0 + t1);
        }
      }
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          P2[yy][e] = A2[yy][e] + B[yy][e];
          A2[yy][e] = A[yy][e];
        }
    }
  }
  if (!ok) {
    if (p.status) atomicExch(p.status, JACC_DEV_TIMEOUT);
    if (warp0)
      for (int j = consumed; j < issued; ++j)
        if (!(stall_cta && j == p.stall_plane)) mbar_wait(&sm.full[j % S], (u32)((j / S) & 1), lim);
  }
  block_sum_to<NT>((double)hi + (double)lo, resid);
}

}  // namespace

namespace jacc {

const void* box27_tb2_kernel() { return (const void*)jacc_k_box27_tb2s; }
int box27_tb2_smem() { return (int)sizeof(Tb2Smem); }
dim3 box27_tb2_grid(i64 nx, i64 ny, i64 nz) {
  return dim3((unsigned)((nx + TW - 1) / TW), (unsigned)((ny + TH - 1) / TH), (unsigned)((nz + ZC - 1) / ZC));
}
dim3 box27_tb2_block() { return dim3(NT); }
cudaError_t box27_tb2_setup() {
  return cudaFuncSetAttribute(jacc_k_box27_tb2s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Tb2Smem));
}

}  // namespace jacc
