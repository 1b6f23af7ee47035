"""GPU: the pointwise error bound of the FP64 fixed-point path, on fields whose
values span 1e-12 to 1.

For convex stencils an FP64 sweep sequence computes in 64-bit fixed point
with 2^-F resolution, F = 57 - E where max|u_0| = m 2^E (0.5 <= m < 1), so
2^-F <= 2^-56 max|u_0|.  The input is truncated toward zero onto that grid
(error < 2^-F), every intermediate sweep rounds to nearest on it (error
<= 2^-(F+1)), and the last sweep rounds the exact stencil value once to FP64
(<= half an ulp of the result).  The 5- and 7-point updates are
non-expansive in the max norm, so after k sweeps every point satisfies

    |g - exact| <= 2^-F + (k - 1) 2^-(F+1) + ulp(g) / 2,

an absolute bound in units of max|u_0|, not a relative one per point: where
the field is locally far below its maximum, the relative error of a point
can reach 2^-56 max|u_0| / |u|, while FP64 evaluated in place keeps about
1e-16 relative there.  The normwise error stays within the 1e-12 tolerance.

"exact" is the same sweep sequence evaluated in numpy's long double (at
least 64 significand bits; its own rounding, at most 4 k 2^-(p) max|u_0|, is
added to the bound).
"""
import math

import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL64, nerr

pytestmark = pytest.mark.gpu

LD = np.longdouble
LD_BITS = np.finfo(LD).nmant + 1


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def frac_bits(M):
    _, E = math.frexp(M)
    return 57 - E


def ulp(x):
    return np.spacing(np.abs(x).astype(np.float64))


def jacobi_ld(u, k):
    a = u.astype(LD)
    for _ in range(k):
        b = a.copy()
        b[1:-1, 1:-1] = LD(0.25) * ((a[:-2, 1:-1] + a[2:, 1:-1]) + (a[1:-1, :-2] + a[1:-1, 2:]))
        a = b
    return a


def heat_ld(u, r, k):
    a = u.astype(LD)
    r = LD(r)
    for _ in range(k):
        b = a.copy()
        c = a[1:-1, 1:-1, 1:-1]
        s = ((a[1:-1, 1:-1, :-2] + a[1:-1, 1:-1, 2:]) + (a[1:-1, :-2, 1:-1] + a[1:-1, 2:, 1:-1])
             + (a[:-2, 1:-1, 1:-1] + a[2:, 1:-1, 1:-1]))
        b[1:-1, 1:-1, 1:-1] = c + r * (s - LD(6) * c)
        a = b
    return a


def check(g, exact, o, M, k):
    if LD_BITS < 64:
        pytest.skip("long double has fewer than 64 significand bits here")
    F = frac_bits(M)
    bound = (2.0 ** -F + (k - 1) * 2.0 ** -(F + 1) + 0.5 * ulp(g)
             + 4 * k * 2.0 ** -(LD_BITS - 1) * M)
    err = np.abs(g.astype(LD) - exact).astype(np.float64)
    worst = np.max(err / bound)
    small = np.abs(exact.astype(np.float64)) < 1e-9 * M
    rel_g = np.max(err[small] / np.abs(exact[small]).astype(np.float64)) if small.any() else 0.0
    rel_o = (np.max(np.abs(o[small].astype(LD) - exact[small]).astype(np.float64)
                    / np.abs(exact[small]).astype(np.float64)) if small.any() else 0.0)
    print(f"F={F}: worst error / bound {worst:.3f}; points below 1e-9 max|u0|: {int(small.sum())}, "
          f"largest relative error there {rel_g:.2e} (fixed point) vs {rel_o:.2e} (FP64 oracle)")
    assert worst <= 1.0
    assert nerr(g, o) <= TOL64


@pytest.mark.parametrize("tile", [0, 17])
def test_jacobi_fixed_point_pointwise_bound_on_1e12_range(orc, tile):
    ny, nx, k = 70, 98, 10
    x = np.arange(nx) / (nx - 1)
    u = np.repeat((10.0 ** (-12.0 * x))[None, :], ny, axis=0)  # smooth: 1 at x = 0 down to 1e-12
    u *= 1.0 + 0.25 * inputs.uniform64(51, nx * ny).reshape(ny, nx)
    kk = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, tile_id=tile)
    assert kk.info()["fixed_point"]
    a = torch.from_numpy(u).cuda()
    b = torch.empty_like(a)
    fb = jacc.sweep(kk, a, b, k)
    torch.cuda.synchronize()
    g = (a if fb == 0 else b).cpu().numpy()
    o, _ = orc.jacobi2d_run(u, k)
    check(g, jacobi_ld(u, k), o, float(np.max(np.abs(u))), k)


@pytest.mark.parametrize("tile", [1, 3])
def test_heat_fixed_point_pointwise_bound_on_1e12_range(orc, tile):
    nz, ny, nx, k = 20, 22, 68, 8
    mag = 10.0 ** (-12.0 * inputs.uniform64(52, nx * ny * nz))
    sgn = np.where(inputs.uniform64(53, nx * ny * nz) < 0.5, -1.0, 1.0)
    u = (mag * sgn).reshape(nz, ny, nx)
    kk = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,), tile_id=tile)
    assert kk.info()["fixed_point"]
    a = torch.from_numpy(u).cuda()
    b = torch.empty_like(a)
    fb = jacc.sweep(kk, a, b, k)
    torch.cuda.synchronize()
    g = (a if fb == 0 else b).cpu().numpy()
    o, _ = orc.heat3d_run(u, 0.125, k)
    check(g, heat_ld(u, 0.125, k), o, float(np.max(np.abs(u))), k)
