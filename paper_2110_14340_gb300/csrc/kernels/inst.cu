// inst.cu - precompiled (generic) kernel instantiations.  Compiled once per
// (stencil, dtype) with -DJACC_INST_STENCIL={5,7,27} -DJACC_INST_DTYPE={32,64};
// each object exports one table of 24 kernel entry points.
#include "jacc_device.cuh"
#include "tiles.h"

#if JACC_INST_DTYPE == 64
typedef double JT;
#define JVEC 2
#else
typedef float JT;
#define JVEC 4
#endif

#if JACC_INST_STENCIL == 5
#define JKERN(BX, BY, V, ZC, O) jacc_k_jacobi2d<JT, BX, BY, V, (ZC) / 4, O>
#elif JACC_INST_STENCIL == 7
#define JKERN(BX, BY, V, ZC, O) jacc_k_heat3d<JT, BX, BY, V, ZC, O>
#else
#define JKERN(BX, BY, V, ZC, O) jacc_k_box27<JT, BX, BY, V, ZC, O>
#endif

#define JCAT3(a, b, c) a##b##_##c
#define JCAT4(a, b, c, d) a##b##_##c##d
#define JTABNAME(s, d) JCAT3(jacc_tab_, s, d)
#define JTABOUT(s, d) JCAT4(jacc_tab_, s, d, _out)
#define JENTRY(id, BX, BY, VEC, ZC) (const void*)JKERN(BX, BY, ((VEC) ? JVEC : 1), ZC, false),
#define JENTRY_OUT(id, BX, BY, VEC, ZC) (const void*)JKERN(BX, BY, ((VEC) ? JVEC : 1), ZC, (JACC_INST_DTYPE == 64)),

// Table 1: the intermediate sweeps of a fixed-point sequence (and every FP32
// or native sweep).  Table 2 ("_out"): the first and last sweeps of a
// fixed-point sequence and single launches, which convert FP64 on load and/or
// store; identical to table 1 for FP32.
extern "C" const void* const JTABNAME(JACC_INST_STENCIL, JACC_INST_DTYPE)[JACC_NTILES] = {JACC_TILE_LIST(JENTRY)};
extern "C" const void* const JTABOUT(JACC_INST_STENCIL, JACC_INST_DTYPE)[JACC_NTILES] = {JACC_TILE_LIST(JENTRY_OUT)};
