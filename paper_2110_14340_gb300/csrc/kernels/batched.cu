// batched.cu - many uneven 5-point Jacobi grids in one persistent launch.
//
// No counterpart in the paper (which overlaps independent kernels on 16
// OpenACC queues, §6.1).  All sweeps of all grids run inside one
// cooperative launch whose CTAs are co-resident.  Work is a sequence of
// tickets in sweep-major order: ticket t names sweep s = t / I and item
// j = t % I of the schedule's item table (item = one band of rows of one
// grid).  A CTA takes the next ticket, waits until every item of sweep s-1 of
// that grid has finished (a per-grid completion counter), runs its band and
// bumps the counter.  Every wait targets strictly smaller tickets, which were
// handed to running CTAs earlier, so the smallest unfinished ticket always
// progresses: no deadlock.  Waits are bounded by %globaltimer; a wait that
// gives up writes JACC_ERR_TIMEOUT to the status word and every CTA leaves.
#include <cuda_runtime.h>

#include "../host/jacc_internal.h"
#include "batched.h"
#include "jacc_device.cuh"

namespace {

JD unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
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

// Bounded wait for *done >= target.  Returns 0 on success, 1 if the batch is
// being abandoned (this wait timed out, or another CTA's did).
JD int wait_done(const unsigned* done, unsigned target, int* status, u64 timeout_ns) {
  if (ld_acquire_u32(done) >= target) return 0;
  const u64 t0 = globaltimer_ns();
  for (;;) {
    if (ld_acquire_u32(done) >= target) return 0;
    if (ld_relaxed_i32(status) != 0) return 1;
    if (globaltimer_ns() - t0 > timeout_ns) {
      atomicCAS(status, 0, JACC_ERR_TIMEOUT);
      return 1;
    }
    __nanosleep(256);
  }
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// One band: warps take 32*V-column chunks; the fixed-point path keeps the
// field resident in fixed point between sweeps (flags: first sweep reads
// FP64, last sweep writes FP64).
template <int V, int MODE>
JD void run_band(const JBGrid& G, const double* src, double* dst, i64 r0, i64 r1, int F, int flags,
                 typename RT<double, MODE>::type& m) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const i64 chunk = 32 * V;
  const i64 nchunks = (G.nx + chunk - 1) / chunk;
  for (i64 c = warp; c < nchunks; c += kWarps) {
    const i64 x0 = c * chunk + lane * V;
    if constexpr (MODE == JM_FIXED) {
      if (flags) jacobi_fx_march<V, true, true>(src, dst, G.nx, G.ny, x0, r0, r1, F, flags, m);
      else jacobi_fx_march<V, true, false>(src, dst, G.nx, G.ny, x0, r0, r1, F, flags, m);
    } else {
      jacobi_march<double, V, MODE, true>(src, dst, G.nx, G.ny, x0, r0, r1, F, m);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 3) jacc_k_batched(JBatchParams bp) {
  __shared__ long long s_ticket;
  __shared__ int s_stop;
  const long long total = (long long)bp.total_items * bp.nsweeps;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(bp.ticket, 1ull);
      int stop = t >= total;
      if (!stop) {
        const int s = (int)(t / bp.total_items);
        const JBItem it = bp.items[t % bp.total_items];
        stop = wait_done(bp.done + it.g, (unsigned)s * (unsigned)bp.grids[it.g].nitems, bp.status, bp.timeout_ns);
      }
      s_ticket = t;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    const long long t = s_ticket;
    const int s = (int)(t / bp.total_items);
    const JBItem it = bp.items[t % bp.total_items];
    const JBGrid G = bp.grids[it.g];
    const i64 r0 = (i64)it.item * G.rows;
    const i64 r1 = (r0 + G.rows < G.ny) ? r0 + G.rows : G.ny;
    const double* src = G.u[s & 1];
    double* dst = G.u[(s + 1) & 1];
    const int F = bp.maxwords ? fx_frac_bits(bp.maxwords[it.g]) : -1;
    const int flags = (s == 0 ? JFX_IN_F64 : 0) | (s == bp.nsweeps - 1 ? JFX_OUT_F64 : 0);
    u64 bits;
    if (F >= 0) {
      u64 m = 0;
      if (G.vec == 2) run_band<2, JM_FIXED>(G, src, dst, r0, r1, F, flags, m);
      else run_band<1, JM_FIXED>(G, src, dst, r0, r1, F, flags, m);
      bits = dbits(fx_to_u(m, F + 2));
    } else {
      double m = 0.0;
      if (G.vec == 2) run_band<2, JM_NATIVE>(G, src, dst, r0, r1, F, flags, m);
      else run_band<1, JM_NATIVE>(G, src, dst, r0, r1, F, flags, m);
      bits = dbits(m);
    }
    block_max_to<kThreads>(bits, bp.resid ? bp.resid + (i64)it.g * bp.nsweeps + s : nullptr);
    __syncthreads();  // every thread's stores of this band precede the signal
    if (threadIdx.x == 0 && t != bp.stall_ticket) {
      __threadfence();
      atomicAdd(bp.done + it.g, 1u);
    }
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

cudaError_t batched_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, jacc_k_batched, kThreads, 0);
}

cudaError_t launch_batched(const JBatchParams& bp, int nctas, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacc_k_batched, bp);
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
