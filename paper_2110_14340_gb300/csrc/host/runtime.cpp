// runtime.cpp - specialisation cache, launches and graph-captured sweeps.
//
// jacc_specialize follows the paper's kernel cache and specialisation
// (§3.1: code compiled once is cached and reused; §3.2.2: runtime-invariant
// parameters are substituted by constants, non-conflicting pointers are
// restrict).  Descriptors are canonicalised into a byte key; identical keys
// share one Kernel object with a reference count.  Without JACC_SPEC_JIT the
// kernel is one of the precompiled instantiations (extents and coefficients
// as arguments); with it, NVRTC compiles the same template with them folded.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../kernels/tiles.h"
#include "jacc_internal.h"
#include "../kernels/jacobi_cluster.h"

extern "C" const void* const jacc_tab_5_64[JACC_NTILES];
extern "C" const void* const jacc_tab_5_32[JACC_NTILES];
extern "C" const void* const jacc_tab_7_64[JACC_NTILES];
extern "C" const void* const jacc_tab_7_32[JACC_NTILES];
extern "C" const void* const jacc_tab_27_64[JACC_NTILES];
extern "C" const void* const jacc_tab_27_32[JACC_NTILES];
extern "C" const void* const jacc_tab_5_64_out[JACC_NTILES];
extern "C" const void* const jacc_tab_5_32_out[JACC_NTILES];
extern "C" const void* const jacc_tab_7_64_out[JACC_NTILES];
extern "C" const void* const jacc_tab_7_32_out[JACC_NTILES];
extern "C" const void* const jacc_tab_27_64_out[JACC_NTILES];
extern "C" const void* const jacc_tab_27_32_out[JACC_NTILES];
extern "C" const void* const jacc_tab_tb[2];

namespace jacc {

static const TileCfg kTiles[JACC_NTILES] = {
#define JACC_TILE_ROW(id, BX, BY, VEC, ZC) {BX, BY, VEC, ZC},
    JACC_TILE_LIST(JACC_TILE_ROW)
#undef JACC_TILE_ROW
};

const TileCfg& tile_cfg(int id) { return kTiles[id]; }

static std::map<std::string, Kernel*>& cache() {
  static std::map<std::string, Kernel*> c;
  return c;
}

// d = m * 2^-k with m odd (d > 0 finite).  Returns false if d is not of
// that form with k in [0, 62].
static bool dyadic(double d, uint64_t* m, int* k) {
  if (!(d > 0.0) || !std::isfinite(d)) return false;
  int e = 0;
  double f = std::frexp(d, &e);  // d = f 2^e, f in [0.5, 1)
  uint64_t mm = static_cast<uint64_t>(std::ldexp(f, 53));
  int kk = 53 - e;
  while ((mm & 1u) == 0 && kk > 0) {
    mm >>= 1;
    --kk;
  }
  if ((mm & 1u) == 0 || kk > 62 || kk < 0) return false;
  *m = mm;
  *k = kk;
  return true;
}

static const void* table_entry(int stencil, int dtype, int tile, bool out) {
  const void* const* t = nullptr;
  if (stencil == 5) t = dtype == 64 ? (out ? jacc_tab_5_64_out : jacc_tab_5_64) : (out ? jacc_tab_5_32_out : jacc_tab_5_32);
  if (stencil == 7) t = dtype == 64 ? (out ? jacc_tab_7_64_out : jacc_tab_7_64) : (out ? jacc_tab_7_32_out : jacc_tab_7_32);
  if (stencil == 27)
    t = dtype == 64 ? (out ? jacc_tab_27_64_out : jacc_tab_27_64) : (out ? jacc_tab_27_32_out : jacc_tab_27_32);
  return t ? t[tile] : nullptr;
}

// Fills the fixed-point fields of p.  Returns the chosen path.
static int plan_fixed(const jacc_kernel_desc& d, JParams& p) {
  p.fpath = JACC_FP_NONE;
  if (d.dtype != JACC_F64 || d.arith != JACC_ARITH_AUTO) return p.fpath;
  if (d.stencil == JACC_STENCIL_5PT) {
    p.fpath = JACC_FP_JACOBI;
    p.fk = 2;
  } else if (d.stencil == JACC_STENCIL_7PT) {
    const double r = d.coeffs[0];
    if (r == 0.0) {
      p.fpath = JACC_FP_SMALL;
      p.fa = 1;
      p.fb = 0;
      p.fk = 0;
    } else if (r > 0.0 && r <= 1.0 / 6.0) {
      uint64_t m;
      int k;
      if (dyadic(r, &m, &k)) {
        if (k <= 5) {
          p.fpath = JACC_FP_SMALL;
          p.fb = static_cast<i64>(m);
          p.fa = (static_cast<i64>(1) << k) - 6 * static_cast<i64>(m);
          p.fk = k;
        } else {
          p.fpath = JACC_FP_WIDE;
          p.fw0 = static_cast<i64>(m);
          p.fk = k;
        }
      }
    }
  } else if (d.stencil == JACC_STENCIL_27PT) {
    const double* w = d.coeffs;
    for (int j = 0; j < 4; ++j)
      if (!(w[j] >= 0.0) || !std::isfinite(w[j])) return p.fpath;
    const double W = w[0] + 6.0 * w[1] + 12.0 * w[2] + 8.0 * w[3];
    if (!(W <= 1.0 + std::ldexp(1.0, -20))) return p.fpath;
    uint64_t m[4] = {0, 0, 0, 0};
    int k[4] = {0, 0, 0, 0};
    int K = 0;
    for (int j = 0; j < 4; ++j) {
      if (w[j] == 0.0) continue;
      if (!dyadic(w[j], &m[j], &k[j])) return p.fpath;
      K = k[j] > K ? k[j] : K;
    }
    if (K > 62) return p.fpath;
    i64 f[4];
    for (int j = 0; j < 4; ++j) {
      if (w[j] == 0.0) {
        f[j] = 0;
        continue;
      }
      const int sh = K - k[j];
      if (sh >= 64 || (m[j] >> (63 - sh)) != 0) return p.fpath;  // factor must stay below 2^63
      f[j] = static_cast<i64>(m[j] << sh);
    }
    p.fpath = JACC_FP_WIDE;
    p.fw0 = f[0];
    p.fw1 = f[1];
    p.fw2 = f[2];
    p.fw3 = f[3];
    p.fk = K;
  }
  return p.fpath;
}

static jacc_status validate(const jacc_kernel_desc& d) {
  if (d.stencil != 5 && d.stencil != 7 && d.stencil != 27 && d.stencil != 19)
    return fail(JACC_ERR_INVALID_ARG, "unknown stencil");
  if (d.stencil == 19) {
    if (d.dtype != JACC_F32) return fail(JACC_ERR_UNSUPPORTED, "19-point variable-coefficient stencil: FP32 only");
    if (d.boundary != JACC_DIRICHLET) return fail(JACC_ERR_UNSUPPORTED, "19-point: Dirichlet only");
    if (d.nx % 4) return fail(JACC_ERR_UNSUPPORTED, "19-point: nx must be a multiple of 4 (16-byte rows)");
    if (d.flags) return fail(JACC_ERR_UNSUPPORTED, "19-point: no JIT or cluster variant");
    if (d.tblock > 1) return fail(JACC_ERR_UNSUPPORTED, "19-point: no temporal blocking");
    if (d.tile_id != -1) return fail(JACC_ERR_INVALID_ARG, "19-point: one fixed tile (tile_id must be -1)");
  }
  if (d.dtype != JACC_F32 && d.dtype != JACC_F64) return fail(JACC_ERR_INVALID_ARG, "dtype must be 32 or 64");
  if (d.tile_id < -1 || d.tile_id >= JACC_NTILES) return fail(JACC_ERR_INVALID_ARG, "tile_id out of range");
  if (d.arith != JACC_ARITH_AUTO && d.arith != JACC_ARITH_NATIVE) return fail(JACC_ERR_INVALID_ARG, "bad arith");
  if (d.flags & ~(JACC_SPEC_JIT | JACC_SPEC_CLUSTER)) return fail(JACC_ERR_INVALID_ARG, "unknown specialisation flags");
  if ((d.flags & JACC_SPEC_CLUSTER) && (d.stencil != 5 || d.dtype != JACC_F64))
    return fail(JACC_ERR_UNSUPPORTED, "JACC_SPEC_CLUSTER: 5-point FP64 only");
  if (d.nx < 3 || d.ny < 3 || d.nz < 1) return fail(JACC_ERR_INVALID_ARG, "extents must be >= 3");
  if (d.stencil == 5) {
    if (d.nz != 1) return fail(JACC_ERR_INVALID_ARG, "5-point stencil is 2D: nz must be 1");
    if (d.boundary != JACC_DIRICHLET) return fail(JACC_ERR_UNSUPPORTED, "5-point stencil supports Dirichlet only");
  } else {
    if (d.nz < 3) return fail(JACC_ERR_INVALID_ARG, "3D stencil: nz must be >= 3");
  }
  if (d.stencil == 7 && d.boundary != JACC_DIRICHLET) return fail(JACC_ERR_UNSUPPORTED, "7-point: Dirichlet only");
  if (d.stencil == 27 && d.boundary != JACC_PERIODIC) return fail(JACC_ERR_UNSUPPORTED, "27-point: periodic only");
  if (d.tblock < 0) return fail(JACC_ERR_INVALID_ARG, "tblock < 0");
  if (d.tblock > 1) {
    if (d.stencil != 27 || d.dtype != JACC_F32 || d.tblock > 3)
      return fail(JACC_ERR_UNSUPPORTED, "temporal blocking: 27-point FP32 with depth 2 or 3 only");
    if (d.nx % 4) return fail(JACC_ERR_UNSUPPORTED, "temporal blocking needs nx divisible by 4");
    if (d.flags & JACC_SPEC_JIT) return fail(JACC_ERR_UNSUPPORTED, "temporal blocking has no folded variant");
  }
  for (int j = 0; j < 4; ++j)
    if (!std::isfinite(d.coeffs[j])) return fail(JACC_ERR_INVALID_ARG, "non-finite coefficient");
  const double n = static_cast<double>(d.nx) * static_cast<double>(d.ny) * static_cast<double>(d.nz);
  if (n > 9.0e18) return fail(JACC_ERR_OVERFLOW, "element count overflows int64");
  return ok();
}

// The default tile, from the autotuner's timing tables on GB300 (5/7/27-point,
// FP32 and FP64, sides 256-1024), by size class.  3D: 32 x 4 threads with
// 16-byte columns; a 64-plane march (tile 3) when it still yields at least
// 1024 CTAs, else a 16-plane march (tile 1) for more CTAs on small grids.
// 2D: 128 x 2 threads, 16-byte columns, 16-row march (tile 17) from 2^19
// points; 64 x 4 threads, scalar columns, 4-row march (tile 8) below, where
// the grid lives in L2 and more, shorter CTAs hide latency better.  Scalar
// 3D variants (2, 0) when nx is not a multiple of the vector width.
int default_tile(const jacc_kernel_desc& d) {
  const int V = d.dtype == 64 ? 2 : 4;
  const bool vec_ok = (d.nx % V) == 0;
  if (d.stencil == 5) {
    if (d.nx * d.ny < (int64_t(1) << 19)) return 8;
    return vec_ok ? 17 : 16;
  }
  const int64_t w = 32 * (vec_ok ? V : 1);  // columns of a 32 x 4 tile
  const int64_t ctas_long = ((d.nx + w - 1) / w) * ((d.ny + 7) / 8) * ((d.nz + 63) / 64);
  if (ctas_long >= 1024) return vec_ok ? 3 : 2;
  return vec_ok ? 1 : 0;
}

bool staged_tile(const jacc_kernel_desc& d, int t) {
  return kTiles[t].vec16 && (d.stencil == 7 || (d.stencil == 27 && d.dtype == 32));
}

bool tile_valid(const jacc_kernel_desc& d, int t) {
  const TileCfg& c = kTiles[t];
  const int V = c.vec16 ? (d.dtype == 64 ? 2 : 4) : 1;
  if (d.nx % V) return false;
  // grid-dimension limits
  const int64_t gy = d.stencil == 5 ? (d.ny + c.by * (c.zc / 4) - 1) / (c.by * (c.zc / 4)) : (d.ny + c.by - 1) / c.by;
  const int64_t gz = d.stencil == 5 ? 1 : (d.nz + c.zc - 1) / c.zc;
  const int64_t gx = (d.nx + c.bx * V - 1) / (c.bx * V);
  return gx < (1ll << 31) && gy <= 65535 && gz <= 65535;
}

static std::string key_of(const jacc_kernel_desc& d, int tile) {
  jacc_kernel_desc c = d;
  c.tile_id = tile;
  c.reserved = 0;
  if (c.tblock == 0) c.tblock = 1;
  return std::string(reinterpret_cast<const char*>(&c), sizeof(c));
}

// Planes per CTA of a 3D kernel.  The constant-folded variants of the staged
// tiles with the long march take fewer planes than the table's 64: with the
// extents folded their kernels need fewer registers and more CTAs fit, and
// shallower chunks then balance better.  Measured with tile 3: heat 512^3
// FP64 best at 40 planes (396.8 against 392.1 GLUP/s at 64), 27-point 1024^3
// FP32 best at 24-32 (128.6 ms for 100 sweeps at 32 against 144.7 at 64).
// The precompiled kernels stay at 64.
static int plane_chunk(const jacc_kernel_desc& d, int tile) {
  const TileCfg& c = kTiles[tile];
  if ((d.flags & JACC_SPEC_JIT) && d.stencil != 5 && staged_tile(d, tile) && c.zc == 64)
    return d.stencil == 27 ? 32 : 40;
  return c.zc;
}

// The NVRTC source of a folded variant: the device text plus a struct whose
// static constexpr members replace JParams.
static std::string jit_source(const Kernel& k) {
  const JParams& p = k.params;
  const TileCfg& c = kTiles[k.tile];
  char buf[4096];
  const char* T = k.desc.dtype == 64 ? "double" : "float";
  const char* entry = k.desc.stencil == 5 ? "jacobi2d_entry" : (k.desc.stencil == 7 ? "heat3d_entry" : "box27_entry");
  const int zc = k.desc.stencil == 5 ? c.zc / 4 : plane_chunk(k.desc, k.tile);
  const char* edge = k.desc.dtype == 64 ? "true" : "false";  // the converting sweeps' instantiation
  std::snprintf(buf, sizeof(buf),
                "\nstruct JFold {\n"
                "  static constexpr i64 nx = %lldll, ny = %lldll, nz = %lldll;\n"
                "  static constexpr double c0 = %a, c1 = %a, c2 = %a, c3 = %a;\n"
                "  static constexpr i64 fa = %lldll, fb = %lldll;\n"
                "  static constexpr i64 fw0 = %lldll, fw1 = %lldll, fw2 = %lldll, fw3 = %lldll;\n"
                "  static constexpr int fk = %d, fpath = %d;\n"
                "};\n"
                "template <> struct JacobiPrefetch<JFold> { static constexpr bool value = %s; };\n"
                "extern \"C\" __global__ void __launch_bounds__(%d, (SweepMinBlocks<%d, %s, %d, %d, %d, false, true>::value))\n"
                "jacc_jit(const %s* __restrict__ u, "
                "%s* __restrict__ v, JParams rt, double* resid, const u64* maxword, int flags) {\n"
                "  const JFold f{};\n"
                "  %s<%s, %d, %d, %d, %d, false>(u, v, f, rt, resid, maxword, flags);\n"
                "}\n"
                "extern \"C\" __global__ void __launch_bounds__(%d, (SweepMinBlocks<%d, %s, %d, %d, %d, %s, true>::value))\n"
                "jacc_jit_out(const %s* __restrict__ u, "
                "%s* __restrict__ v, JParams rt, double* resid, const u64* maxword, int flags) {\n"
                "  const JFold f{};\n"
                "  %s<%s, %d, %d, %d, %d, %s>(u, v, f, rt, resid, maxword, flags);\n"
                "}\n"
                "extern \"C\" __global__ void __launch_bounds__(%d, (SweepMinBlocksLast<%d, %s, %d, %d, %d>::value))\n"
                "jacc_jit_last(const %s* __restrict__ u, "
                "%s* __restrict__ v, JParams rt, double* resid, const u64* maxword, int flags) {\n"
                "  const JFold f{};\n"
                "  %s<%s, %d, %d, %d, %d, %s>(u, v, f, rt, resid, maxword, JFX_OUT_F64);\n"
                "}\n",
                (long long)p.nx, (long long)p.ny, (long long)p.nz, p.c0, p.c1, p.c2, p.c3, (long long)p.fa,
                (long long)p.fb, (long long)p.fw0, (long long)p.fw1, (long long)p.fw2, (long long)p.fw3, p.fk, p.fpath,
                // small (L2-resident) 2D grids: the prefetching march
                (k.desc.stencil == 5 && k.desc.nx * k.desc.ny <= (int64_t(1) << 17)) ? "true" : "false",
                c.bx * c.by, k.desc.stencil, T, c.bx, c.by, k.vec, T, T, entry, T, c.bx, c.by, k.vec, zc, c.bx * c.by,
                k.desc.stencil, T, c.bx, c.by, k.vec, edge, T, T, entry, T, c.bx, c.by, k.vec, zc, edge, c.bx * c.by,
                k.desc.stencil, T, c.bx, c.by, k.vec, T, T, entry, T, c.bx, c.by, k.vec, zc, edge);
  return std::string(device_source()) + buf;
}

static void free_kernel(Kernel* k) {
  for (auto& g : k->graphs) {
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (g.second.graph) cudaGraphDestroy(g.second.graph);
    if (g.second.scratch) cudaFree(g.second.scratch);
  }
  k->graphs.clear();
  for (auto& g : k->coeff_graphs) {
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (g.second.graph) cudaGraphDestroy(g.second.graph);
  }
  k->coeff_graphs.clear();
  free_until_graphs(*k);
  if (k->scratch) cudaFree(k->scratch);
  if (k->lib) cudaLibraryUnload(k->lib);
  delete k;
}

}  // namespace jacc

using namespace jacc;

extern "C" jacc_status jacc_tile_info(int32_t tile_id, jacc_tile* out) {
  if (tile_id < 0 || tile_id >= JACC_NTILES || !out) return fail(JACC_ERR_INVALID_ARG, "bad tile_id or NULL out");
  const TileCfg& c = kTiles[tile_id];
  out->bx = c.bx;
  out->by = c.by;
  out->vec16 = c.vec16;
  out->zc = c.zc;
  return ok();
}

extern "C" jacc_status jacc_specialize(const jacc_kernel_desc* desc, jacc_kernel* out) {
  if (!desc || !out) return fail(JACC_ERR_INVALID_ARG, "NULL descriptor or output");
  jacc_status st = validate(*desc);
  if (st) return st;
  int tile = desc->tile_id;
  if (desc->stencil == 19) {
    tile = 3;  // the kernel's one configuration: 32 x 4 threads, 16-byte columns, 40-plane march
  } else if (tile < 0) {
    tile = tuned_tile(*desc);
    if (tile < 0 || !tile_valid(*desc, tile)) tile = default_tile(*desc);
  }
  if (!tile_valid(*desc, tile))
    return fail(JACC_ERR_INVALID_ARG, "tile " + std::to_string(tile) + " does not fit this shape (x vector width)");
  const std::string key = key_of(*desc, tile);
  std::lock_guard<std::mutex> lock(global_mutex());
  auto it = cache().find(key);
  if (it != cache().end()) {
    it->second->refcount++;
    *out = reinterpret_cast<jacc_kernel>(it->second);
    return ok();
  }
  std::unique_ptr<Kernel> k(new Kernel());
  k->desc = *desc;
  k->desc.tile_id = tile;
  k->key = key;
  k->tile = tile;
  k->elem = desc->dtype / 8;
  const TileCfg& c = kTiles[tile];
  k->vec = c.vec16 ? 16 / k->elem : 1;
  JParams& p = k->params;
  p.nx = desc->nx;
  p.ny = desc->ny;
  p.nz = desc->nz;
  p.c0 = desc->coeffs[0];
  p.c1 = desc->coeffs[1];
  p.c2 = desc->coeffs[2];
  p.c3 = desc->coeffs[3];
  plan_fixed(*desc, p);
  k->block = dim3(c.bx, c.by, 1);
  const int64_t tx = static_cast<int64_t>(c.bx) * k->vec;
  if (desc->stencil == 5) {
    const int64_t ty = static_cast<int64_t>(c.by) * (c.zc / 4);
    k->grid = dim3(static_cast<unsigned>((desc->nx + tx - 1) / tx), static_cast<unsigned>((desc->ny + ty - 1) / ty), 1);
  } else {
    // the staged kernels (16-byte columns: 7-point, and 27-point FP32) give each thread 2 rows
    const int64_t ty = static_cast<int64_t>(c.by) * (staged_tile(*desc, tile) ? 2 : 1);
    const int64_t zc = plane_chunk(*desc, tile);
    k->grid = dim3(static_cast<unsigned>((desc->nx + tx - 1) / tx), static_cast<unsigned>((desc->ny + ty - 1) / ty),
                   static_cast<unsigned>((desc->nz + zc - 1) / zc));
  }
  if (desc->stencil == 19) {
    var19_geometry(desc->nx, desc->ny, desc->nz, &k->grid, &k->block);
    k->func = k->func_out = nullptr;  // launched by jacc_sweep_coeffs only
  } else if (desc->tblock == 2) {
    // two sweeps per launch, staged: 320 threads over a 128 x 16 output tile,
    // 64-plane chunks (box27_tb2.cu)
    k->tblock = 2;
    st = cuda_check(box27_tb2_setup(), "cudaFuncSetAttribute(two-sweep 27-point kernel)");
    if (st) return st;
    k->func = k->func_out = box27_tb2_kernel();
    k->block = box27_tb2_block();
    k->grid = box27_tb2_grid(desc->nx, desc->ny, desc->nz);
    k->smem = box27_tb2_smem();
  } else if (desc->tblock > 1) {
    // temporally blocked 27-point kernel: 32 x 16 threads over a 128 x 16 region,
    // output tile 120 x (16 - 2T), 64-plane chunks
    const int T = desc->tblock;
    k->tblock = T;
    k->func = jacc_tab_tb[T - 2];
    k->block = dim3(32, 16, 1);
    const int64_t oy = 16 - 2 * T;
    k->grid = dim3(static_cast<unsigned>((desc->nx + 119) / 120), static_cast<unsigned>((desc->ny + oy - 1) / oy),
                   static_cast<unsigned>((desc->nz + 63) / 64));
    k->func_out = k->func;
  } else if (desc->flags & JACC_SPEC_JIT) {
    static const char* const names[3] = {"jacc_jit", "jacc_jit_out", "jacc_jit_last"};
    const void* f[3] = {nullptr, nullptr, nullptr};
    st = jit_compile(jit_source(*k), names, 3, &k->lib, f, &k->compile_ms);
    if (st) return st;
    k->func = f[0];
    k->func_out = f[1];
    // the store-only converting kernel: FP64 fixed-point sequences only
    if (desc->dtype == 64) k->func_last = f[2];
    k->jit = true;
  } else {
    k->func = table_entry(desc->stencil, desc->dtype, tile, false);
    k->func_out = table_entry(desc->stencil, desc->dtype, tile, true);
    if (!k->func || !k->func_out) return fail(JACC_ERR_UNSUPPORTED, "no precompiled kernel for this descriptor");
  }
  if (desc->flags & JACC_SPEC_CLUSTER) {
    int nc = 0;
    if (!jacobi_cluster_plan(desc->nx, desc->ny, &nc)) {
      if (k->lib) cudaLibraryUnload(k->lib);
      return fail(JACC_ERR_UNSUPPORTED, "JACC_SPEC_CLUSTER: the grid does not fit one cluster's shared memory");
    }
    k->cluster_nc = nc;
  }
  // scratch words: [0] max|u| bits of direct FP64 fixed-point launches, [1] the
  // device status word of bounded waits (JACC_DEV_TIMEOUT)
  st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&k->scratch), 256), "cudaMalloc(scratch)");
  if (!st) st = cuda_check(cudaMemset(k->scratch, 0, 256), "cudaMemset(scratch)");
  if (st) {
    if (k->scratch) cudaFree(k->scratch);
    if (k->lib) cudaLibraryUnload(k->lib);
    return st;
  }
  p.status = reinterpret_cast<int*>(k->scratch + 1);
  p.timeout_ns = kDefaultTimeoutNs;
  p.stall_plane = -1;
  k->refcount = 1;
  Kernel* raw = k.release();
  cache()[key] = raw;
  *out = reinterpret_cast<jacc_kernel>(raw);
  return ok();
}

extern "C" jacc_status jacc_kernel_status(jacc_kernel h, int32_t* status) {
  if (!h || !status) return fail(JACC_ERR_INVALID_ARG, "NULL handle or output");
  const Kernel& k = *reinterpret_cast<Kernel*>(h);
  jacc_status st = cuda_check(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if (st) return st;
  int v = 0;
  st = cuda_check(cudaMemcpy(&v, k.params.status, sizeof(int), cudaMemcpyDeviceToHost), "read status word");
  if (!st) st = cuda_check(cudaMemset(k.params.status, 0, sizeof(int)), "clear status word");
  if (st) return st;
  *status = v;
  return ok();
}

extern "C" jacc_status jacc_kernel_set_wait(jacc_kernel h, int32_t timeout_ms, int32_t stall_plane) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  if (timeout_ms < 0 || stall_plane < -1) return fail(JACC_ERR_INVALID_ARG, "timeout_ms < 0 or stall_plane < -1");
  std::lock_guard<std::mutex> lock(global_mutex());
  Kernel& k = *reinterpret_cast<Kernel*>(h);
  k.params.timeout_ns = timeout_ms == 0 ? kDefaultTimeoutNs : static_cast<int64_t>(timeout_ms) * 1000000;
  k.params.stall_plane = stall_plane;
  // cached graphs hold the old parameters: drop them
  for (auto& g : k.graphs) {
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    if (g.second.graph) cudaGraphDestroy(g.second.graph);
    if (g.second.scratch) cudaFree(g.second.scratch);
  }
  k.graphs.clear();
  free_until_graphs(k);
  return ok();
}

extern "C" jacc_status jacc_kernel_info(jacc_kernel h, jacc_kernel_info_t* out) {
  if (!h || !out) return fail(JACC_ERR_INVALID_ARG, "NULL handle or output");
  const Kernel& k = *reinterpret_cast<Kernel*>(h);
  out->tile_id = k.tile;
  out->jit = k.jit ? 1 : 0;
  out->fixed_point = k.params.fpath != JACC_FP_NONE ? 1 : 0;
  out->tblock = k.tblock;
  out->block[0] = static_cast<int32_t>(k.block.x);
  out->block[1] = static_cast<int32_t>(k.block.y);
  out->block[2] = static_cast<int32_t>(k.block.z);
  out->grid[0] = static_cast<int32_t>(k.grid.x);
  out->grid[1] = static_cast<int32_t>(k.grid.y);
  out->grid[2] = static_cast<int32_t>(k.grid.z);
  out->compile_ms = k.compile_ms;
  return ok();
}

extern "C" jacc_status jacc_release(jacc_kernel h) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  std::lock_guard<std::mutex> lock(global_mutex());
  Kernel* k = reinterpret_cast<Kernel*>(h);
  auto it = cache().find(k->key);
  if (it == cache().end() || it->second != k) return fail(JACC_ERR_INVALID_ARG, "unknown or released handle");
  if (--k->refcount > 0) return ok();
  cache().erase(it);
  free_kernel(k);
  return ok();
}

extern "C" jacc_status jacc_shutdown(void) {
  std::lock_guard<std::mutex> lock(global_mutex());
  for (auto& e : cache()) free_kernel(e.second);
  cache().clear();
  static_scratch_forget();
  return ok();
}

// ---------------------------------------------------------------- launches

namespace jacc {

cudaError_t launch_sweep_kernel(const Kernel& k, const void* u, void* v, double* resid, const u64* maxword, int flags,
                                cudaStream_t s) {
  JParams p = k.params;
  const void* args[] = {&u, &v, &p, &resid, &maxword, &flags};
  // programmatic dependent launch: the kernel may start while the previous
  // sweep finishes; every sweep kernel waits (griddepcontrol.wait) for the
  // previous grid before it touches a field
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = k.grid;
  cfg.blockDim = k.block;
  cfg.dynamicSmemBytes = static_cast<size_t>(k.smem);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const void* f = flags == kFxOut && k.func_last ? k.func_last : ((flags & (kFxIn | kFxOut)) ? k.func_out : k.func);
  return cudaLaunchKernelExC(&cfg, f, const_cast<void**>(args));
}

jacc_status check_buffers(const Kernel& k, const void* a, const void* b) {
  if (!a || !b) return fail(JACC_ERR_INVALID_ARG, "NULL field pointer");
  if ((reinterpret_cast<uintptr_t>(a) % 16) || (reinterpret_cast<uintptr_t>(b) % 16))
    return fail(JACC_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
  const uintptr_t bytes = static_cast<uintptr_t>(k.desc.nx * k.desc.ny * k.desc.nz) * k.elem;
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  if (pa < pb + bytes && pb < pa + bytes) return fail(JACC_ERR_INVALID_ARG, "input and output fields overlap");
  return ok();
}

}  // namespace jacc

// Enqueue one sweep with its pre-pass (fixed point) and residual zeroing.
static jacc_status enqueue_one(const Kernel& k, const void* u, void* v, double* resid, u64* scratch, cudaStream_t s) {
  const u64* mw = nullptr;
  if (k.params.fpath != JACC_FP_NONE && k.desc.dtype == 64) {
    jacc_status st = cuda_check(launch_maxabs(static_cast<const double*>(u), k.desc.nx * k.desc.ny * k.desc.nz,
                                              scratch, s),
                                "max-abs pre-pass");
    if (st) return st;
    mw = scratch;
  }
  if (resid) {
    jacc_status st = cuda_check(cudaMemsetAsync(resid, 0, sizeof(double), s), "cudaMemsetAsync(resid)");
    if (st) return st;
  }
  return cuda_check(launch_sweep_kernel(k, u, v, resid, mw, kFxIn | kFxOut, s), "stencil launch");
}

extern "C" jacc_status jacc_launch(jacc_kernel h, const void* u_in, void* u_out, double* resid_dev, uintptr_t stream) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  const Kernel& k = *reinterpret_cast<Kernel*>(h);
  if (k.desc.stencil == 19) return fail(JACC_ERR_INVALID_ARG, "19-point stencil: use jacc_sweep_coeffs");
  jacc_status st = check_buffers(k, u_in, u_out);
  if (st) return st;
  return enqueue_one(k, u_in, u_out, resid_dev, k.scratch, reinterpret_cast<cudaStream_t>(stream));
}

// The full sweep sequence on stream s.  A temporally blocked kernel performs
// tblock sweeps per launch; only every tblock-th sweep is materialised and the
// residual slots of the others are set to NaN.
static jacc_status enqueue_sweeps(const Kernel& k, void* u0, void* u1, int32_t n, double* resid, u64* scratch,
                                  cudaStream_t s) {
  const u64* mw = nullptr;
  if (k.params.fpath != JACC_FP_NONE && k.desc.dtype == 64) {
    jacc_status st = cuda_check(
        launch_maxabs(static_cast<const double*>(u0), k.desc.nx * k.desc.ny * k.desc.nz, scratch, s), "max-abs pre-pass");
    if (st) return st;
    mw = scratch;
  }
  const int T = k.tblock > 1 ? k.tblock : 1;
  if (resid) {
    jacc_status st = cuda_check(cudaMemsetAsync(resid, 0, sizeof(double) * static_cast<size_t>(n), s), "memset resid");
    if (!st && T > 1) st = cuda_check(launch_fill_skipped(resid, n, T, s), "resid NaN fill");
    if (st) return st;
  }
  const int32_t launches = n / T;
  // A large FP64 fixed-point field is converted in place first, so that its
  // first sweep runs the intermediate kernel: the converting kernel holds
  // fewer CTAs per SM and converts each staged value where it is used (512^3:
  // 1.11 ms against 0.34 + 0.17 ms for the conversion).  u0 is overwritten by
  // the second sweep anyway, and the values are those the first sweep would
  // convert on load, so results do not change.  Small fields keep one launch.
  const int64_t npts = k.desc.nx * k.desc.ny * k.desc.nz;
  const bool pre = mw && launches >= 2 && npts >= (int64_t(1) << 22);
  if (pre) {
    jacc_status st = cuda_check(launch_to_fixed(static_cast<double*>(u0), npts, mw, s), "fixed-point conversion");
    if (st) return st;
  }
  for (int32_t i = 0; i < launches; ++i) {
    const void* src = (i % 2 == 0) ? u0 : u1;
    void* dst = (i % 2 == 0) ? u1 : u0;
    const int fl = (i == 0 && !pre ? kFxIn : 0) | (i == launches - 1 ? kFxOut : 0);
    double* r = resid ? resid + static_cast<int64_t>(i) * T + (T - 1) : nullptr;
    jacc_status st = cuda_check(launch_sweep_kernel(k, src, dst, r, mw, fl, s), "stencil launch");
    if (st) return st;
  }
  return ok();
}

extern "C" jacc_status jacc_sweep(jacc_kernel h, void* u0, void* u1, int32_t nsweeps, double* resid_dev, uint32_t flags,
                                  uintptr_t stream, int32_t* final_buf) {
  if (!h) return fail(JACC_ERR_INVALID_ARG, "NULL handle");
  if (nsweeps < 1) return fail(JACC_ERR_INVALID_ARG, "nsweeps must be >= 1");
  if (flags & ~JACC_SWEEP_GRAPH) return fail(JACC_ERR_INVALID_ARG, "unknown sweep flags");
  Kernel& k = *reinterpret_cast<Kernel*>(h);
  if (k.desc.stencil == 19) return fail(JACC_ERR_INVALID_ARG, "19-point stencil: use jacc_sweep_coeffs");
  jacc_status st = check_buffers(k, u0, u1);
  if (st) return st;
  if (k.tblock > 1 && nsweeps % k.tblock)
    return fail(JACC_ERR_INVALID_ARG, "nsweeps must be a multiple of the temporal-blocking depth");
  if (k.desc.stencil == 27 && k.params.fpath != JACC_FP_NONE) {
    // the fixed-point scale is taken once from u0; values may grow by W per sweep
    const double W = k.desc.coeffs[0] + 6 * k.desc.coeffs[1] + 12 * k.desc.coeffs[2] + 8 * k.desc.coeffs[3];
    if (std::pow(W, static_cast<double>(nsweeps)) > 4.0)
      return fail(JACC_ERR_UNSUPPORTED, "weight sum too far above 1 for this many fixed-point sweeps");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (final_buf) *final_buf = (nsweeps / (k.tblock > 1 ? k.tblock : 1)) % 2;
  if (k.cluster_nc > 0) {  // the whole sequence in one cluster launch (it writes every residual slot)
    JClusterArgs a = {};
    a.u = static_cast<const double*>(u0);
    a.res = static_cast<double*>((nsweeps & 1) ? u1 : u0);
    a.oth = static_cast<double*>((nsweeps & 1) ? u0 : u1);
    a.resid = resid_dev;
    a.nx = k.desc.nx;
    a.ny = k.desc.ny;
    a.nsweeps = nsweeps;
    a.native = k.params.fpath == JACC_FP_NONE ? 1 : 0;
    st = cuda_check(launch_jacobi_cluster(a, k.cluster_nc, s), "cluster sweep launch");
    if (st) return st;
    if (final_buf) *final_buf = (nsweeps & 1) ? 1 : 0;
    return ok();
  }
  if (!(flags & JACC_SWEEP_GRAPH)) return enqueue_sweeps(k, u0, u1, nsweeps, resid_dev, k.scratch, s);

  std::lock_guard<std::mutex> lock(global_mutex());
  const GraphKey gk{u0, u1, nsweeps, resid_dev};
  auto it = k.graphs.find(gk);
  if (it == k.graphs.end()) {
    SweepGraph g;
    if (k.params.fpath != JACC_FP_NONE && k.desc.dtype == 64) {
      st = cuda_check(cudaMalloc(reinterpret_cast<void**>(&g.scratch), 256), "cudaMalloc(graph scratch)");
      if (st) return st;
    }
    cudaStream_t cap = nullptr;
    st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (!st) {
      jacc_status est = enqueue_sweeps(k, u0, u1, nsweeps, resid_dev, g.scratch, cap);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(cap, &graph);
      if (est) st = est;
      else st = cuda_check(ce, "cudaStreamEndCapture");
      g.graph = graph;
      if (!st) st = cuda_check(cudaGraphInstantiate(&g.exec, g.graph, 0), "cudaGraphInstantiate");
    }
    if (cap) cudaStreamDestroy(cap);
    if (st) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      if (g.scratch) cudaFree(g.scratch);
      return st;
    }
    it = k.graphs.emplace(gk, g).first;
  }
  return cuda_check(cudaGraphLaunch(it->second.exec, s), "cudaGraphLaunch");
}
