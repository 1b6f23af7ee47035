"""GB300 (sm_103a) runtime-specialised affine stencil path.

The compute lives in libjacc.so (CUDA kernels + C ABI, include/jacc.h);
`jacc` is its ctypes binding, `build` compiles it in-tree and `inputs` draws
the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
