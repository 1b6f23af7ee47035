"""GPU: jacc_sweep_until, the device-side loop that stops at a residual tolerance.

The loop must stop at the first sweep whose residual is <= tol (or at
max_sweeps): the stop count expected is the oracle's, from its own residuals,
with tolerances placed between two consecutive oracle residuals.  The result
field and residuals must match the oracle run of that many sweeps, and both
buffers and the residuals must be bit-identical to jacc_sweep run for that
many sweeps.
"""
import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL32, TOL64, assert_resid, nerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def fixed_count(k, u, n):
    a = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    b = torch.zeros_like(a)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    fb = jacc.sweep(k, a, b, n, r)
    torch.cuda.synchronize()
    return fb, a.cpu().numpy(), b.cpu().numpy(), r.cpu().numpy()


def until(k, u, max_sweeps, tol):
    a = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    b = torch.zeros_like(a)
    r = torch.full((max_sweeps,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    jacc.sweep_until(k, a, b, max_sweeps, tol, r, st)
    torch.cuda.synchronize()
    n, fb = st.cpu().tolist()
    return n, fb, a.cpu().numpy(), b.cpu().numpy(), r.cpu().numpy()


def field(stencil, dtype):
    if stencil == jacc.STENCIL_5PT:
        u = inputs.jacobi2d_field(70, 48, seed=31)
        shape = dict(nx=70, ny=48)
    else:
        u = inputs.heat3d_field(40, ny=26, nz=21, seed=32)
        shape = dict(nx=40, ny=26, nz=21)
    return (u.astype(np.float32) if dtype == jacc.F32 else u), shape


CASES = [(jacc.STENCIL_5PT, jacc.F64, jacc.ARITH_AUTO), (jacc.STENCIL_5PT, jacc.F64, jacc.ARITH_NATIVE),
         (jacc.STENCIL_5PT, jacc.F32, jacc.ARITH_AUTO), (jacc.STENCIL_7PT, jacc.F64, jacc.ARITH_AUTO),
         (jacc.STENCIL_7PT, jacc.F32, jacc.ARITH_AUTO)]


def oracle_run(orc, stencil, u, n):
    u64 = u.astype(np.float64)
    if stencil == jacc.STENCIL_5PT:
        return orc.jacobi2d_run(u64, n)
    return orc.heat3d_run(u64, 0.125, n)


@pytest.mark.parametrize("stencil,dtype,arith", CASES)
@pytest.mark.parametrize("stop", ["tol", "first", "max"])
def test_until_stops_where_the_residual_says_and_matches_fixed_count(orc, stencil, dtype, arith, stop):
    u, shape = field(stencil, dtype)
    coeffs = (0.125,) if stencil == jacc.STENCIL_7PT else (0.0,)
    k = jacc.Kernel(stencil, dtype, coeffs=coeffs, arith=arith, **shape)
    max_sweeps = 60
    _, orr = oracle_run(orc, stencil, u, max_sweeps)
    assert np.all(np.diff(orr) < 0)  # strictly decreasing residuals on these fields
    # a tolerance strictly between two consecutive oracle residuals (their
    # geometric mean), far from either compared with the rounding of a sweep
    tol = {"tol": float(np.sqrt(orr[22] * orr[23])), "first": float(orr[0]) * 2.0, "max": 0.0}[stop]
    n_expected = {"tol": 24, "first": 1, "max": max_sweeps}[stop]
    n, fb, a, b, r = until(k, u, max_sweeps, tol)
    assert n == n_expected and fb == n % 2
    o, orn = oracle_run(orc, stencil, u, n)
    fp64 = dtype == jacc.F64
    assert nerr(b if fb else a, o) <= (TOL64 if fp64 else TOL32)
    assert_resid(r[:n], orn, np.max(np.abs(u)), fp64=fp64)
    fb2, a2, b2, r2 = fixed_count(k, u, n)
    assert fb2 == fb
    view = np.int64 if dtype == jacc.F64 else np.int32
    assert np.array_equal(a.view(view), a2.view(view))
    assert np.array_equal(b.view(view), b2.view(view))
    assert np.array_equal(r[:n], r2)
    assert np.all(r[n:] == -1.0)  # slots after the last sweep are untouched


def test_until_graph_is_cached_and_replays(orc):
    u, shape = field(jacc.STENCIL_5PT, jacc.F64)
    k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, **shape)
    a = torch.from_numpy(u).cuda()
    b = torch.zeros_like(a)
    r = torch.zeros(40, dtype=torch.float64, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    _, orr = orc.jacobi2d_run(u, 40)
    tol = float(np.sqrt(orr[14] * orr[15]))  # between the oracle's 15th and 16th residuals
    n_expected = 16
    outs = []
    for _ in range(3):
        a.copy_(torch.from_numpy(u))
        jacc.sweep_until(k, a, b, 40, tol, r, st)
        torch.cuda.synchronize()
        n, fb = st.cpu().tolist()
        outs.append((n, (b if fb else a).cpu().numpy().copy()))
    assert all(o[0] == n_expected for o in outs)
    assert all(np.array_equal(o[1], outs[0][1]) for o in outs)
    o, _ = orc.jacobi2d_run(u, n_expected)
    assert nerr(outs[0][1], o) <= TOL64


def test_until_rejects_27_point_and_bad_arguments():
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, 16, 16, 16, coeffs=(0.5, 0.05, 0.01, 0.005))
    a = torch.zeros(16, 16, 16, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    r = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        jacc.sweep_until(k, a, b, 4, 0.0, r, st)
    k5 = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, 8, 8)
    a5 = torch.zeros(8, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep_until(k5, a5, torch.zeros_like(a5), 0, 0.0, r, st)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep_until(k5, a5, torch.zeros_like(a5), 4, -1.0, r, st)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep_until(k5, a5, a5, 4, 0.0, r, st)


def test_large_field_sequence_with_input_conversion_matches_until(orc):
    # a field of at least 2^22 points: jacc_sweep converts u0 in place before
    # its first sweep; jacc_sweep_until converts on load in its first sweep.
    # Both must leave the same bits in both buffers and the same residuals,
    # and match the oracle.
    side = 162  # 162^3 = 4.25 M points
    u = inputs.heat3d_field(side, seed=33)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    n = 6
    fb, a, b, r = fixed_count(k, u, n)
    n2, fb2, a2, b2, r2 = until(k, u, n, 0.0)
    assert n2 == n and fb2 == fb
    assert np.array_equal(a.view(np.int64), a2.view(np.int64))
    assert np.array_equal(b.view(np.int64), b2.view(np.int64))
    assert np.array_equal(r, r2[:n])
    with orc.threads():
        o, orr = orc.heat3d_run(u, 0.125, n)
    assert nerr(b2 if fb2 else a2, o) <= TOL64
    assert_resid(r2[:n], orr, np.max(np.abs(u)))
