// nvrtc.cpp - runtime compilation of constant-folded kernel variants.
//
// The paper's runtime generates function code for a kernel, hands it to a
// compiler at run time and links the result dynamically (§3.1); the first
// compilation costs about two seconds per kernel and later launches reuse it
// (§4.4).  Here NVRTC compiles the variant straight to an sm_103a cubin,
// which is loaded with the CUDA library-management API.  Cubins are cached on
// disk under $JACC_CACHE_DIR (if set), keyed by a hash of the full source,
// the options and the NVRTC version.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "jacc_internal.h"

namespace jacc {

static uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

static bool read_file(const std::string& path, std::string* out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  *out = ss.str();
  return !out->empty();
}

jacc_status jit_compile(const std::string& src, const char* const* names, int nnames, cudaLibrary_t* lib,
                        const void** funcs, double* ms) {
  const auto t0 = std::chrono::steady_clock::now();
  static const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-DJACC_NVRTC=1"};
  const int nopts = 4;
  int major = 0, minor = 0;
  nvrtcVersion(&major, &minor);
  std::string keytext = src + "|" + params_source();
  for (int i = 0; i < nopts; ++i) keytext += std::string("|") + opts[i];
  keytext += "|" + std::to_string(major) + "." + std::to_string(minor);
  char hex[32];
  std::snprintf(hex, sizeof(hex), "%016llx", static_cast<unsigned long long>(fnv1a(keytext)));
  const char* dir = std::getenv("JACC_CACHE_DIR");
  std::string path = dir ? std::string(dir) + "/jacc_" + hex + ".cubin" : std::string();

  std::string cubin;
  if (path.empty() || !read_file(path, &cubin)) {
    nvrtcProgram prog;
    const char* hdr_src[] = {params_source()};
    const char* hdr_name[] = {"jacc_params.h"};
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "jacc_jit.cu", 1, hdr_src, hdr_name);
    if (r != NVRTC_SUCCESS) return fail(JACC_ERR_COMPILE, std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r));
    r = nvrtcCompileProgram(prog, nopts, opts);
    if (r != NVRTC_SUCCESS) {
      size_t n = 0;
      nvrtcGetProgramLogSize(prog, &n);
      std::string log(n, '\0');
      if (n) nvrtcGetProgramLog(prog, &log[0]);
      nvrtcDestroyProgram(&prog);
      if (log.size() > 4000) log.resize(4000);
      return fail(JACC_ERR_COMPILE, std::string("NVRTC compile failed: ") + log);
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin.assign(n, '\0');
    nvrtcGetCUBIN(prog, &cubin[0]);
    nvrtcDestroyProgram(&prog);
    if (!path.empty()) {
      std::string tmp = path + ".tmp" + std::to_string(reinterpret_cast<uintptr_t>(&cubin));
      std::ofstream f(tmp, std::ios::binary);
      if (f) {
        f.write(cubin.data(), static_cast<std::streamsize>(cubin.size()));
        f.close();
        std::rename(tmp.c_str(), path.c_str());
      }
    }
  }
  cudaError_t e = cudaLibraryLoadData(lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return fail(JACC_ERR_COMPILE, std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e));
  for (int i = 0; i < nnames; ++i) {
    cudaKernel_t kern = nullptr;
    e = cudaLibraryGetKernel(&kern, *lib, names[i]);
    if (e != cudaSuccess) {
      cudaLibraryUnload(*lib);
      *lib = nullptr;
      return fail(JACC_ERR_COMPILE, std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e));
    }
    funcs[i] = reinterpret_cast<const void*>(kern);
  }
  *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ok();
}

}  // namespace jacc
