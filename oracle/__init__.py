"""CPU oracle for the runtime-specialised affine stencil path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2110_14340_gb300``) never does, and shares no code with it.

``oracle.c`` holds the definitions (plain C, FP64 unless the stencil is
defined in FP32, no FMA contraction); this module only marshals numpy arrays
into it through ctypes.
"""
from .oracle import *  # noqa: F401,F403
from .build import build  # noqa: F401
