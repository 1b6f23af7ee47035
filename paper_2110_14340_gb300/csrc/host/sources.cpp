// sources.cpp - the device-code text that NVRTC compiles, embedded at build time.
#include "jacc_internal.h"

namespace jacc {
#include "jacc_embedded_src.inc"  // generated by build.py from kernels/*.h, *.cuh
const char* device_source() { return kDeviceSource; }
const char* params_source() { return kParamsSource; }
}  // namespace jacc
