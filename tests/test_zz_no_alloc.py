"""jacc_launch_static, the allocation-free launch, against jacc_launch.

Some callers cannot allocate device memory when they launch (a memory pool
that must own every device byte, a path that must not synchronise on
cudaMalloc).  jacc_launch_static keeps its scratch in a static device array
instead; its output must equal jacc_launch's, call after call, since the
array keeps the previous call's contents, and match the oracle's sweep.  This file sorts last so that a run
stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL64, assert_resid, nerr

pytestmark = pytest.mark.gpu


def test_static_scratch_launch_matches_jacc_launch(orc):
    from paper_2110_14340_gb300 import build
    build.build()
    L = jacc.lib()
    n = 66
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, n, n + 2, n - 2, coeffs=(0.125,))
    assert k.info()["fixed_point"]
    s = torch.cuda.current_stream().cuda_stream
    fields = [inputs.heat3d_field(n, seed=2, ny=n + 2, nz=n - 2),
              inputs.heat3d_field(n, seed=3, ny=n + 2, nz=n - 2) * 1e3]  # a different scale on the second call
    for u in fields:
        a = torch.from_numpy(u).cuda()
        want = torch.empty_like(a)
        got = torch.full_like(a, float("nan"))
        r_want = torch.zeros(1, dtype=torch.float64, device="cuda")
        r_got = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert L.jacc_launch(k.handle, C.c_void_p(a.data_ptr()), C.c_void_p(want.data_ptr()),
                             C.c_void_p(r_want.data_ptr()), s) == 0
        assert L.jacc_launch_static(k.handle, C.c_void_p(a.data_ptr()), C.c_void_p(got.data_ptr()),
                                    C.c_void_p(r_got.data_ptr()), s) == 0
        torch.cuda.synchronize()
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert np.max(np.abs(g - w)) <= TOL64 * np.max(np.abs(w))
        assert abs(r_got.item() - r_want.item()) <= TOL64 * np.max(np.abs(w))
        o, orr = orc.heat3d_sweep(u, 0.125)
        assert nerr(g, o) <= TOL64
        assert_resid([r_got.item()], [orr], np.max(np.abs(u)))
    # errors are those of jacc_launch
    assert L.jacc_launch_static(k.handle, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), None, s) == \
        jacc.ERR_INVALID_ARG
    k.release()
