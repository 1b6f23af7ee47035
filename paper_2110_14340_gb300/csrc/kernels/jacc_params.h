// jacc_params.h - the kernel parameter block, shared by the host runtime, the
// precompiled kernels and the NVRTC-compiled variants.
#pragma once

typedef unsigned long long u64;
typedef long long i64;
typedef unsigned int u32;

// Fixed-point path selector (JParams::fpath).
#define JACC_FP_NONE 0   // native arithmetic only
#define JACC_FP_SMALL 1  // 7pt, r = fb 2^-k with k <= 5: v 2^(F+k) = fa u + fb S in int64
#define JACC_FP_WIDE 2   // 7pt / 27pt: exact 128-bit products
#define JACC_FP_JACOBI 3 // 5pt: v 2^(F+2) = S

struct JParams {
  i64 nx, ny, nz;
  double c0, c1, c2, c3;   // coefficients for the native path: 7pt r; 27pt w0, wf, we, wc
  i64 fa, fb;              // JACC_FP_SMALL factors
  i64 fw0, fw1, fw2, fw3;  // JACC_FP_WIDE factors (7pt: fw0 = odd mantissa of r)
  int fk;                  // extra fraction bits of the fixed-point result
  int fpath;               // JACC_FP_*
  // Bounded waits of the bulk-copy staged kernels: each wait on an mbarrier
  // gives up after timeout_ns, writes JACC_DEV_TIMEOUT to *status (device,
  // nullable) and the CTA returns.  stall_plane >= 0 is a test hook: CTA
  // (0,0,0) never requests that staged plane, so its waits run out.
  int* status;
  i64 timeout_ns;
  int stall_plane;
  int reserved;
  // The twelve coefficient fields of the variable-coefficient 19-point
  // stencil (a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 wrk1 bnd; FP32, device), set per
  // call; unused by the other stencils.
  const float* cf[12];
};

#define JACC_DEV_TIMEOUT (-6)  // the value of JACC_ERR_TIMEOUT
