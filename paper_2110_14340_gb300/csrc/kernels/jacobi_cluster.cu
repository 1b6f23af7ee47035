// jacobi_cluster.cu - all sweeps of a small 5-point FP64 grid in one launch of
// one thread-block cluster, the field resident in the cluster's shared memory.
//
// A 256 x 256 FP64 grid is 512 KB per field: too large for one SM, small
// enough for the distributed shared memory of a cluster of 8 or 16 CTAs.  A
// sweep of such a grid is a few microseconds of launch latency and a fraction
// of that of work, so one launch per sweep (even replayed from a CUDA graph)
// is latency-bound.  Here CTA r of the cluster keeps rows [r*rows, (r+1)*rows)
// of both ping-pong fields plus one halo row above and below in its shared
// memory.  A sweep writes its first and last own rows also into the
// neighbours' halo rows (st.shared::cluster), then one cluster barrier
// (release/acquire) orders every CTA's writes before the next sweep.  The
// barrier is split: each warp reduces its residual maximum between the
// arrive and the wait, and warp 0 combines a sweep's per-warp partials after
// the next sweep's barrier, so a sweep costs one barrier and no other
// synchronisation.  HBM is touched once to load the field and once to store
// the result.
//
// The arithmetic is that of the resident fixed-point path (and of its native
// FP64 fallback) bit for bit: max|u| over the grid picks F, the first sweep
// converts on load, intermediate sweeps keep v 2^F = (S + 2) >> 2, the last
// writes fx_to(S, F + 2) and, if there were two sweeps or more, the other
// buffer receives sweep n-1 in the internal form, exactly as jacc_sweep's
// launch-per-sweep sequence leaves it.
#include "jacc_device.cuh"

#include <cuda_runtime.h>

#include "jacobi_cluster.h"

namespace {

constexpr int kThreads = 1024;  // threads per CTA (512 for small grids, see launch_jacobi_cluster)
constexpr int kResChunk = 512;  // sweeps whose residuals are held in shared memory before a flush
// Column-pair items per thread held in registers.  A CTA's two fields fit in
// at most 227 KB, 2 (rows + 2) pitch words, so rows * pitch / 2 / 1024 < 7;
// with 512 threads a CTA of more than 4096 pairs takes the unhoisted loop.
constexpr int kMaxItems = 8;

JD u32 cluster_rank() {
  u32 r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// All threads of all CTAs of the cluster; orders shared and global memory.
JD void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The two halves of cluster_sync, for work that needs neither the barrier's
// release (done after the arrive) nor its acquire (done before the wait).
JD void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
JD void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// Shared-memory address of `p` (this CTA) in CTA `rank` of the cluster.
JD u32 map_rank(const void* p, u32 rank) {
  u32 out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}
JD void st_cluster_u64(u32 addr, u64 v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
JD u64 ld_cluster_u64(u32 addr) {
  u64 v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}

// One intermediate fixed-point sweep over a thread's hoisted items (column
// pairs at shared-memory word offsets ioff[i]).  An item whose warp-uniform
// bit in `fast` is set has both columns interior on every lane of the warp
// and no edge-row push, so it runs without selects; the others keep the
// boundary columns unchanged.  src and dst are the two fields, which never
// overlap, so the loads of one item may be issued ahead of the stores of the
// one before.  Returns the thread's maximum of |4(v - u)| (one less for
// negative differences), the form the residual is reduced in.
JD u64 fx_items(const u64* __restrict__ src, u64* __restrict__ dst, i64 pitch, const int (&ioff)[kMaxItems],
                u32 ikind, u32 fast, int nit) {
  u64 rmax = 0;
#pragma unroll
  for (int i = 0; i < kMaxItems; ++i) {
    if (i >= nit) break;
    const u64* rc = src + ioff[i];
    const longlong2 c = *reinterpret_cast<const longlong2*>(rc);
    const longlong2 up = *reinterpret_cast<const longlong2*>(rc - pitch);
    const longlong2 dn = *reinterpret_cast<const longlong2*>(rc + pitch);
    const i64 xl = (i64)rc[-1], xr = (i64)rc[2];
    const i64 s0 = (up.x + dn.x) + (xl + c.y);
    const i64 s1 = (up.y + dn.y) + (c.x + xr);
    const i64 d0 = s0 - c.x * 4, d1 = s1 - c.y * 4;
    const u64 a0 = (u64)(d0 ^ (d0 >> 63)), a1 = (u64)(d1 ^ (d1 >> 63));  // |d| (one less if negative)
    longlong2 v;
    if (fast & (1u << i)) {
      v.x = (s0 + 2) >> 2;
      v.y = (s1 + 2) >> 2;
      rmax = max(rmax, max(a0, a1));
    } else {
      const u32 kd = ikind >> (4 * i);
      const bool in0 = kd & 1u, in1 = kd & 2u;
      v.x = in0 ? (s0 + 2) >> 2 : c.x;
      v.y = in1 ? (s1 + 2) >> 2 : c.y;
      rmax = max(rmax, max(in0 ? a0 : 0ull, in1 ? a1 : 0ull));
    }
    *reinterpret_cast<longlong2*>(dst + ioff[i]) = v;
  }
  return rmax;
}

template <int NC, int NT>
__global__ void __launch_bounds__(NT) jacc_k_jacobi_cluster(JClusterArgs a) {
  extern __shared__ __align__(16) u64 smem[];
  __shared__ u64 part_max;
  const i64 nx = a.nx, ny = a.ny, rows = a.rows, pitch = a.pitch;
  const int t = threadIdx.x;
  const u32 rank = cluster_rank();
  const i64 r0 = (i64)rank * rows;
  const i64 r1 = (r0 + rows < ny) ? r0 + rows : ny;
  const i64 nr = (r1 > r0) ? r1 - r0 : 0;  // own rows (0 for a CTA past the grid)
  u64* const bufA = smem;                       // local row lr <-> grid row r0 - 1 + lr
  u64* const bufB = smem + (rows + 2) * pitch;

  // max |u| over the grid: this CTA's rows, then every CTA's partial
  u64 m = 0;
  for (i64 i = t; i < nr * nx; i += NT) {
    const u64 b = dbits(a.u[r0 * nx + i]) & 0x7fffffffffffffffull;
    m = b > m ? b : m;
  }
  m = warp_max_u64(m);
  __shared__ u64 red[NT / 32];
  if ((t & 31) == 0) red[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    u64 w = 0;
    for (int k = 0; k < NT / 32; ++k) w = red[k] > w ? red[k] : w;
    part_max = w;
  }
  cluster_sync();
  u64 gmax = 0;
  for (int k = 0; k < NC; ++k) {
    const u64 w = ld_cluster_u64(map_rank(&part_max, (u32)k));
    gmax = w > gmax ? w : gmax;
  }
  const int F = a.native ? -1 : fx_frac_bits(gmax);
  const bool fixed = F >= 0;

  // load own rows and the two halo rows, converted to the working form
  for (i64 lr = 0; lr < nr + 2; ++lr) {
    const i64 g = r0 - 1 + lr;
    if (g < 0 || g >= ny) continue;
    for (i64 x = t; x < nx; x += NT) {
      const double d = a.u[g * nx + x];
      bufA[lr * pitch + x] = fixed ? (u64)fx_from(d, F) : dbits(d);
    }
  }
  __syncthreads();

  const int n = a.nsweeps;
  // this thread's items: column pair cp of local row lr, advanced by
  // NT items per step (32-bit index arithmetic, no division per item)
  const int half = (int)((nx + 1) / 2);  // column pairs per row
  const int step_rows = NT / half, step_cols = NT % half;
  const int nitems = (int)nr * half;
  // x-neighbour rows of the cluster neighbours, for pushing edge rows
  const bool push_up = rank > 0 && nr > 0 && r0 >= 1;  // first own row -> previous CTA's lower halo row
  const bool push_dn = nr > 0 && r1 < ny;              // last own row -> next CTA's upper halo row
  __shared__ u64 wred[3][NT / 32];               // per-warp residual partials of sweeps k % 3
  __shared__ u64 rres[kResChunk];                      // this CTA's residual maxima of the current chunk
  // The items of a thread are the same in every sweep: their shared-memory
  // offsets and point kinds are worked out once (at most kMaxItems per thread,
  // which the shared-memory budget guarantees for every grid that fits)
  int ioff[kMaxItems];
  u32 ikind = 0;  // per item i, bits 4i..4i+3: column 0 interior, column 1 interior, push up, push down
  int nit = 0;
  {
    int lr = 1 + t / half, cp = t % half;
    for (int it = t; it < nitems && nit < kMaxItems; it += NT, ++nit) {
      const i64 x0 = 2 * (i64)cp;
      const i64 g = r0 - 1 + lr;
      const bool yin = g >= 1 && g <= ny - 2;
      ioff[nit] = (int)(lr * pitch + x0);
      ikind |= (u32)((yin && x0 >= 1 && x0 <= nx - 2) | ((yin && x0 + 1 <= nx - 2) << 1) |
                     ((push_up && lr == 1) << 2) | ((push_dn && lr == nr) << 3))
               << (4 * nit);
      cp += step_cols;
      lr += step_rows;
      if (cp >= half) {
        cp -= half;
        ++lr;
      }
    }
  }
  const bool hoisted = nitems <= kMaxItems * NT;
  // per item, one bit for the whole warp: every lane holds the item, both its
  // columns are interior and it pushes no edge row
  u32 fast = 0;
#pragma unroll
  for (int i = 0; i < kMaxItems; ++i) {
    const u32 kd = (ikind >> (4 * i)) & 15u;
    fast |= (u32)__all_sync(0xffffffffu, i < nit && kd == 3u) << i;
  }
  const u32 pushes = ikind & 0xccccccccu;  // this thread's push bits
  int slot = 0;                            // wred slot of sweep k: k % 3
  for (int k = 0; k < n; ++k) {
    const u64* src = (k & 1) ? bufB : bufA;
    u64* dst = (k & 1) ? bufA : bufB;
    const bool last = k == n - 1;
    u64 rmax_fx = 0;
    double rmax_nat = 0.0;
    int lr = 1 + t / half, cp = t % half;
    if (fixed && !last && hoisted) {
      // intermediate fixed-point sweeps: hoisted items, 16-byte shared-memory
      // accesses, no per-sweep index arithmetic; then the edge rows (their
      // values re-read from this thread's own stores) into the neighbours'
      // halo rows
      rmax_fx = fx_items(src, dst, pitch, ioff, ikind, fast, nit);
      if (pushes) {
#pragma unroll
        for (int i = 0; i < kMaxItems; ++i) {
          if (i >= nit) break;
          const u32 kd = ikind >> (4 * i);
          if (!(kd & 12u)) continue;
          const longlong2 v = *reinterpret_cast<const longlong2*>(dst + ioff[i]);
          if (kd & 4u) {  // first own row -> the previous CTA's lower halo row
            const u32 ra = map_rank(dst + ioff[i] + rows * pitch, rank - 1);
            st_cluster_u64(ra, (u64)v.x);
            st_cluster_u64(ra + 8, (u64)v.y);
          }
          if (kd & 8u) {  // last own row -> the next CTA's upper halo row
            const u32 ra = map_rank(dst + ioff[i] - nr * pitch, rank + 1);
            st_cluster_u64(ra, (u64)v.x);
            st_cluster_u64(ra + 8, (u64)v.y);
          }
        }
      }
    } else if (fixed && !last) {
      // intermediate fixed-point sweeps: a column pair per item, 16-byte
      // shared-memory accesses (pitch is even, so every pair is aligned; an
      // odd nx pads each row by one word, which is written but never used)
      for (int it = t; it < nitems; it += NT) {
        const i64 x0 = 2 * (i64)cp;
        const i64 g = r0 - 1 + lr;
        const bool yin = g >= 1 && g <= ny - 2;
        const bool in0 = yin && x0 >= 1 && x0 <= nx - 2, in1 = yin && x0 + 1 <= nx - 2;
        const u64* rc = src + lr * pitch + x0;
        const longlong2 c = *reinterpret_cast<const longlong2*>(rc);
        const longlong2 up = *reinterpret_cast<const longlong2*>(rc - pitch);
        const longlong2 dn = *reinterpret_cast<const longlong2*>(rc + pitch);
        const i64 xl = (i64)rc[-1], xr = (i64)rc[2];
        const i64 s0 = (up.x + dn.x) + (xl + c.y);
        const i64 s1 = (up.y + dn.y) + (c.x + xr);
        longlong2 v;
        v.x = in0 ? (s0 + 2) >> 2 : c.x;
        v.y = in1 ? (s1 + 2) >> 2 : c.y;
        const i64 d0 = s0 - c.x * 4, d1 = s1 - c.y * 4;
        const u64 a0 = (u64)(d0 ^ (d0 >> 63)), a1 = (u64)(d1 ^ (d1 >> 63));  // |d| (one less if negative)
        rmax_fx = (in0 && a0 > rmax_fx) ? a0 : rmax_fx;
        rmax_fx = (in1 && a1 > rmax_fx) ? a1 : rmax_fx;
        *reinterpret_cast<longlong2*>(dst + lr * pitch + x0) = v;
        // edge rows also go straight into the neighbours' halo rows
        if (push_up && lr == 1) {
          const u32 ra = map_rank(dst + (rows + 1) * pitch + x0, rank - 1);
          st_cluster_u64(ra, (u64)v.x);
          st_cluster_u64(ra + 8, (u64)v.y);
        }
        if (push_dn && lr == nr) {
          const u32 ra = map_rank(dst + x0, rank + 1);
          st_cluster_u64(ra, (u64)v.x);
          st_cluster_u64(ra + 8, (u64)v.y);
        }
        cp += step_cols;
        lr += step_rows;
        if (cp >= half) {
          cp -= half;
          ++lr;
        }
      }
    } else {
      for (int it = t; it < nitems; it += NT) {
        const i64 x0 = 2 * (i64)cp;
        const i64 g = r0 - 1 + lr;
        const bool yin = g >= 1 && g <= ny - 2;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const i64 x = x0 + e;
          if (x >= nx) break;
          const bool in = yin && x >= 1 && x <= nx - 2;
          const u64 cw = src[lr * pitch + x];
          u64 vw = cw;       // next working word (boundary: unchanged)
          double out = 0.0;  // FP64 result (last sweep)
          if (fixed) {
            const i64 c = (i64)cw;
            if (in) {
              const i64 s = ((i64)src[(lr - 1) * pitch + x] + (i64)src[(lr + 1) * pitch + x]) +
                            ((i64)src[lr * pitch + x - 1] + (i64)src[lr * pitch + x + 1]);
              vw = (u64)((s + 2) >> 2);
              if (last) out = fx_to(s, F + 2);
              const i64 d = s - c * 4;
              const u64 ad = (u64)(d ^ (d >> 63));  // |d| (one less for negative d), as the sweep kernels
              rmax_fx = ad > rmax_fx ? ad : rmax_fx;
            } else if (last) {
              out = (n == 1) ? a.u[g * nx + x] : fx_to(c, F);
            }
          } else {
            const double c = __longlong_as_double((i64)cw);
            if (in) {
              const double s = (__longlong_as_double((i64)src[(lr - 1) * pitch + x]) +
                                __longlong_as_double((i64)src[(lr + 1) * pitch + x])) +
                               (__longlong_as_double((i64)src[lr * pitch + x - 1]) +
                                __longlong_as_double((i64)src[lr * pitch + x + 1]));
              const double r = 0.25 * s;
              vw = dbits(r);
              out = r;
              double d = r - c;
              d = d < 0.0 ? -d : d;
              rmax_nat = d > rmax_nat ? d : rmax_nat;
            } else {
              out = c;
            }
          }
          if (last) {
            a.res[g * nx + x] = out;
            if (n >= 2) a.oth[g * nx + x] = __longlong_as_double((i64)cw);
          } else {
            dst[lr * pitch + x] = vw;
            // edge rows also go straight into the neighbours' halo rows
            if (push_up && lr == 1) st_cluster_u64(map_rank(dst + (rows + 1) * pitch + x, rank - 1), vw);
            if (push_dn && lr == nr) st_cluster_u64(map_rank(dst + x, rank + 1), vw);
          }
        }
        cp += step_cols;
        lr += step_rows;
        if (cp >= half) {
          cp -= half;
          ++lr;
        }
      }
    }
    // One cluster barrier per sweep, split in two: its arrive releases this
    // sweep's field writes (local and pushed), and the warp's residual
    // maximum (the maximum magnitude in fixed point, or the bits of the
    // non-negative maximum, which order alike) is reduced while the other
    // CTAs arrive.  The per-warp partials of sweep k go to wred[k % 3]; they
    // are read after the next sweep's barrier, whose arrive releases them,
    // and the slot is next written two sweeps later, after warp 0 has
    // arrived past its read.
    cluster_arrive();
    const u64 bits = warp_max_u64(fixed ? rmax_fx : dbits(rmax_nat));
    if ((t & 31) == 0) wred[slot][t >> 5] = bits;
    cluster_wait();
    const int prev = slot == 0 ? 2 : slot - 1;
    // warp 0: this CTA's residual of sweep k - 1 (unless a flush took it)
    if (t < 32 && k >= 1 && (k - 1) % kResChunk != kResChunk - 1) {
      u64 w = t < NT / 32 ? wred[prev][t] : 0ull;
      w = warp_max_u64(w);
      if (t == 0) rres[(k - 1) % kResChunk] = fixed ? dbits(fx_to_u(w, F + 2)) : w;
    }
    // Residuals leave the cluster in chunks: a global write before a barrier
    // would make the barrier's release wait for it, so each sweep's CTA
    // maxima stay in shared memory until the chunk ends; then CTA 0 takes
    // the maximum over the cluster and stores it (plain stores, no atomics).
    if (k % kResChunk == kResChunk - 1 || last) {
      __syncthreads();  // this sweep's per-warp partials
      if (t < 32) {
        u64 w = t < NT / 32 ? wred[slot][t] : 0ull;
        w = warp_max_u64(w);
        if (t == 0) rres[k % kResChunk] = fixed ? dbits(fx_to_u(w, F + 2)) : w;
      }
      cluster_sync();  // every CTA's maxima of this chunk are written
      const int k0 = k - k % kResChunk;
      if (rank == 0 && a.resid) {
        for (int i = t; i <= k - k0; i += NT) {
          u64 w = 0;
          for (int r = 0; r < NC; ++r) {
            const u64 v = ld_cluster_u64(map_rank(&rres[i], (u32)r));
            w = v > w ? v : w;
          }
          a.resid[k0 + i] = __longlong_as_double((i64)w);
        }
      }
      if (last) cluster_sync();  // CTA 0's remote reads precede every exit
    }
    slot = slot == 2 ? 0 : slot + 1;
  }
}

template <int NC, int NT> cudaError_t launch_nc(const JClusterArgs& a, size_t smem, cudaStream_t s) {
  const void* f = (const void*)jacc_k_jacobi_cluster<NC, NT>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (NC > 8) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = NC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacc_k_jacobi_cluster<NC, NT>, a);
}

template <int NC> bool fits_nc(const JClusterArgs& a, size_t smem) {
  const void* f = (const void*)jacc_k_jacobi_cluster<NC, kThreads>;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
  if (NC > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = NC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

size_t smem_bytes(i64 ny, i64 pitch, int nc, i64* rows) {
  *rows = (ny + nc - 1) / nc;
  return (size_t)(2 * (*rows + 2) * pitch) * sizeof(u64);
}

}  // namespace

int jacobi_cluster_plan(long long nx, long long ny, int* nc_out) {
  const i64 pitch = (nx + 1) & ~1ll;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  const size_t budget = (size_t)optin - 8192;  // static shared memory of the kernel
  for (int nc : {16, 8}) {
    i64 rows = 0;
    const size_t smem = smem_bytes(ny, pitch, nc, &rows);
    if (smem > budget || rows < 1) continue;
    JClusterArgs a = {};
    a.nx = nx;
    a.ny = ny;
    a.rows = rows;
    a.pitch = pitch;
    if (nc == 16 ? fits_nc<16>(a, smem) : fits_nc<8>(a, smem)) {
      *nc_out = nc;
      return 1;
    }
  }
  return 0;
}

cudaError_t launch_jacobi_cluster(JClusterArgs a, int nc, cudaStream_t s) {
  a.pitch = (a.nx + 1) & ~1ll;
  const size_t smem = smem_bytes(a.ny, a.pitch, nc, &a.rows);
  // 512 threads when a CTA has at most 1024 column pairs (up to two per
  // thread rather than one or none), 1024 otherwise: measured 1.00 against
  // 1.21 us per sweep at 128^2, 1.95 against 1.73 at 256^2 (1000 sweeps)
  const long long pairs = a.rows * ((a.nx + 1) / 2);
  if (pairs <= 1024) return nc == 16 ? launch_nc<16, 512>(a, smem, s) : launch_nc<8, 512>(a, smem, s);
  return nc == 16 ? launch_nc<16, kThreads>(a, smem, s) : launch_nc<8, kThreads>(a, smem, s);
}
