// jacc_internal.h - shared declarations of the host runtime (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../../include/jacc.h"
#include "../kernels/jacc_params.h"

namespace jacc {

// Records `msg` as the calling thread's last error and returns `st`.
jacc_status fail(jacc_status st, const std::string& msg);
jacc_status ok();
// Wraps a CUDA runtime status: JACC_OK or JACC_ERR_CUDA with the CUDA message.
jacc_status cuda_check(cudaError_t e, const char* what);

struct TileCfg {
  int bx, by, vec16, zc;
};
const TileCfg& tile_cfg(int id);

// One cached sweep graph.
struct SweepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  u64* scratch = nullptr;  // max-abs word of this graph (device)
};

using GraphKey = std::tuple<const void*, const void*, int32_t, const double*>;

// One cached jacc_sweep_until graph (device-side loop with conditional nodes).
struct UntilGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  u64* scratch = nullptr;  // [0] max-abs word, [1] residual slot, [2] sweep counter, [3] spare residual slot
};
using UntilKey = std::tuple<const void*, const void*, int32_t, double, const double*, const int32_t*>;

// A specialised kernel (the object behind a jacc_kernel handle).
struct Kernel {
  jacc_kernel_desc desc{};
  std::string key;
  JParams params{};
  int tile = 0;
  int elem = 8;                 // bytes per element
  int vec = 1;                  // elements per thread in x
  bool jit = false;
  double compile_ms = 0.0;
  const void* func = nullptr;   // kernel entry (host stub or cudaKernel_t)
  const void* func_out = nullptr;  // entry for the first/last sweep of a fixed-point sequence (FP64 in or out)
  const void* func_last = nullptr;  // constant-folded FP64 last sweep that converts only on store (or null)
  cudaLibrary_t lib = nullptr;  // NVRTC module, if jit
  dim3 grid, block;
  int smem = 0;                 // dynamic shared memory per CTA of `func`
  int tblock = 1;
  int cluster_nc = 0;           // JACC_SPEC_CLUSTER: CTAs of the cluster-resident sweep launch
  int refcount = 0;
  u64* scratch = nullptr;       // max-abs word for direct launches (device)
  std::map<GraphKey, SweepGraph> graphs;
  std::map<UntilKey, UntilGraph> until_graphs;
  std::map<std::string, SweepGraph> coeff_graphs;  // jacc_sweep_coeffs graphs, keyed by all pointers
};

// The two-sweep staged 27-point FP32 kernel (temporal blocking, T = 2;
// rows of 16-byte multiples).
const void* box27_tb2_kernel();
int box27_tb2_smem();
dim3 box27_tb2_grid(long long nx, long long ny, long long nz);
dim3 box27_tb2_block();
cudaError_t box27_tb2_setup();

// The variable-coefficient 19-point kernel (one fixed tile).
void var19_geometry(long long nx, long long ny, long long nz, dim3* grid, dim3* block);
cudaError_t launch_var19(const float* u, float* v, const JParams& p, double* resid, dim3 grid, dim3 block,
                         cudaStream_t s);

// Validates a pair of field pointers for kernel k (non-null, 16-byte aligned,
// not overlapping).
jacc_status check_buffers(const Kernel& k, const void* a, const void* b);
// Destroys k's cached jacc_sweep_until graphs.
void free_until_graphs(Kernel& k);
cudaError_t launch_until_check(double* slot, int* counter, double* resid, double tol, int max_sweeps,
                               cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_odd, cudaStream_t s);
cudaError_t launch_until_final(const int* counter, int* status, int recompute, cudaGraphConditionalHandle h_final,
                               cudaStream_t s);

// Launch one sweep of `k` (no validation).  maxword may be null.  flags:
// JFX_* bits (first sweep of a sequence reads FP64, last writes FP64).
cudaError_t launch_sweep_kernel(const Kernel& k, const void* u, void* v, double* resid, const u64* maxword, int flags,
                                cudaStream_t s);
constexpr int kFxIn = 1, kFxOut = 2;  // JFX_IN_F64, JFX_OUT_F64
// Default limit of one bounded device wait (staged kernels): 2 s.
constexpr int64_t kDefaultTimeoutNs = 2000000000;
// Enqueue the max-abs pre-pass of `n` doubles into maxword (zeroing it first).
cudaError_t launch_maxabs(const double* u, long long n, u64* maxword, cudaStream_t s);
cudaError_t launch_fill_skipped(double* resid, int n, int T, cudaStream_t s);
// u (n FP64 values) -> the resident fixed point in place, F from *maxword
cudaError_t launch_to_fixed(double* u, long long n, const u64* maxword, cudaStream_t s);
// Drops the cached per-device address of jacc_launch_static's scratch array.
void static_scratch_forget();

// NVRTC: compile `src` (plus jacc_params.h) for sm_103a, load it, return
// kernel `name`.  Uses the on-disk cache under $JACC_CACHE_DIR if set.
jacc_status jit_compile(const std::string& src, const char* const* names, int nnames, cudaLibrary_t* lib,
                        const void** funcs, double* ms);
// The device-code text embedded at build time.
const char* device_source();
const char* params_source();

std::mutex& global_mutex();

// Tile validity for a descriptor (vector width and grid limits) and the
// default tile; the autotuner's remembered pick for a shape (-1 if none).
bool tile_valid(const jacc_kernel_desc& d, int t);
// Tiles that run a bulk-copy staged kernel (2 rows per thread).
bool staged_tile(const jacc_kernel_desc& d, int t);
int default_tile(const jacc_kernel_desc& d);
int tuned_tile(const jacc_kernel_desc& d);
void remember_tile(const jacc_kernel_desc& d, int tile);

}  // namespace jacc
