"""GPU parity: every stencil kernel through the C ABI against the CPU oracle.

Sizes span several tiles in every axis with ragged tails; every one of the 24
tile configurations is exercised.  Tolerances (tests/tolerances.py): fields
normwise (max |g - o| / max |o|) within 1e-12 for FP64 and 1e-5 for FP32;
residuals within 1e-12 (1e-5) of the residual vector's own scale, or within
the rounding that k FP64 (FP32) sweeps can leave in a difference of two
fields, whichever is larger.
"""
import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL32, TOL64, assert_resid, nerr

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()
    yield
    torch.cuda.synchronize()


def run(k, u, nsweeps, graph=True):
    t = torch.float64 if k.desc.dtype == 64 else torch.float32
    a = torch.from_numpy(np.ascontiguousarray(u)).to(DEV, t)
    b = torch.zeros_like(a)
    res = torch.full((nsweeps,), -1.0, dtype=torch.float64, device=DEV)
    fb = jacc.sweep(k, a, b, nsweeps, res, graph=graph)
    torch.cuda.synchronize()
    return (a if fb == 0 else b).cpu().numpy(), res.cpu().numpy()


# ----------------------------------------------------------------------------- 5-point Jacobi

@pytest.mark.parametrize("tile", range(24))
def test_jacobi2d_f64_all_tiles(orc, tile):
    ny, nx = 150, 266  # ragged against every tile in both axes
    u = inputs.jacobi2d_field(nx, ny, seed=1)
    k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, tile_id=tile)
    assert k.info()["fixed_point"]
    g, gr = run(k, u, 7)
    o, orr = orc.jacobi2d_run(u, 7)
    assert nerr(g, o) <= TOL64
    assert_resid(gr, orr, np.max(np.abs(u)))


@pytest.mark.parametrize("tile", [0, 4, 8, 16, 22])
def test_jacobi2d_f64_odd_width_native_and_fixed(orc, tile):
    ny, nx = 37, 101
    u = inputs.jacobi2d_field(nx, ny, seed=7)
    o, orr = orc.jacobi2d_run(u, 5)
    for arith in (jacc.ARITH_AUTO, jacc.ARITH_NATIVE):
        k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, tile_id=tile, arith=arith)
        g, gr = run(k, u, 5)
        assert nerr(g, o) <= TOL64
        assert_resid(gr, orr, np.max(np.abs(u)))


@pytest.mark.parametrize("tile", [1, 5, 13, 23])
def test_jacobi2d_f32(orc, tile):
    ny, nx = 90, 300
    u = inputs.jacobi2d_field(nx, ny, seed=11)
    k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F32, nx, ny, 1, tile_id=tile)
    g, gr = run(k, u.astype(np.float32), 6)
    o, orr = orc.jacobi2d_run(u.astype(np.float32).astype(np.float64), 6)
    assert nerr(g, o) <= TOL32
    assert_resid(gr, orr, np.max(np.abs(u)), fp64=False)


def test_jacobi2d_affine_fixed_point_bit_exact():
    ny, nx = 45, 130
    y, x = np.mgrid[0:ny, 0:nx]
    u = 3.0 * x - 2.0 * y + 7.0
    k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1)
    g, gr = run(k, u, 9)
    assert np.array_equal(g, u) and np.all(gr == 0.0)


def test_jacobi2d_full_size_256_100_sweeps(orc):
    # the 256 x 256, 100-sweep configuration, element by element
    u = inputs.jacobi2d_field(256, 256, seed=1)
    k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, 256, 256, 1)
    g, gr = run(k, u, 100)
    o, orr = orc.jacobi2d_run(u, 100)
    assert nerr(g, o) <= TOL64
    assert_resid(gr, orr, np.max(np.abs(u)))
    assert np.all(gr[1:] <= gr[:-1] + 1e-15)


def run_both(k, u, nsweeps):
    """Both buffers and the residuals after a sweep sequence."""
    a = torch.from_numpy(np.ascontiguousarray(u)).to(DEV)
    b = torch.zeros_like(a)
    res = torch.full((nsweeps,), -1.0, dtype=torch.float64, device=DEV)
    fb = jacc.sweep(k, a, b, nsweeps, res)
    torch.cuda.synchronize()
    return fb, a.cpu().numpy(), b.cpu().numpy(), res.cpu().numpy()


@pytest.mark.parametrize("shape,nsweeps,arith", [
    ((256, 256), 100, jacc.ARITH_AUTO), ((130, 37), 7, jacc.ARITH_AUTO), ((3, 3), 1, jacc.ARITH_AUTO),
    ((17, 255), 2, jacc.ARITH_AUTO), ((64, 41), 1, jacc.ARITH_AUTO), ((101, 37), 5, jacc.ARITH_NATIVE),
    ((320, 300), 3, jacc.ARITH_AUTO), ((64, 41), 1100, jacc.ARITH_AUTO), ((40, 52), 513, jacc.ARITH_NATIVE),
    ((256, 256), 1025, jacc.ARITH_AUTO)])
def test_jacobi2d_cluster_resident_bit_identical_to_per_sweep(orc, shape, nsweeps, arith):
    # the whole sequence in one cluster launch: result buffer, the other
    # buffer (sweep n-1 in the internal form) and residuals equal the
    # launch-per-sweep sequence bit for bit
    ny, nx = shape
    u = inputs.jacobi2d_field(nx, ny, seed=21)
    kc = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, arith=arith, cluster=True)
    kp = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, arith=arith)
    fc, ac, bc, rc = run_both(kc, u, nsweeps)
    fp, ap, bp, rp = run_both(kp, u, nsweeps)
    assert fc == fp == nsweeps % 2
    assert np.array_equal(ac.view(np.int64), ap.view(np.int64))
    assert np.array_equal(bc.view(np.int64), bp.view(np.int64))
    assert np.array_equal(rc, rp)
    o, orr = orc.jacobi2d_run(u, nsweeps)
    assert nerr(bc if fc else ac, o) <= TOL64
    assert_resid(rc, orr, np.max(np.abs(u)))


def test_jacobi2d_cluster_nonfinite_input_and_limits(orc):
    ny, nx = 40, 52
    u = inputs.jacobi2d_field(nx, ny, seed=22)
    u[10, 11] = np.inf  # routes the sequence to native FP64, as in the per-sweep path
    kc = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, cluster=True)
    kp = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1)
    fc, ac, bc, rc = run_both(kc, u, 4)
    fp, ap, bp, rp = run_both(kp, u, 4)
    assert np.array_equal(ac.view(np.int64), ap.view(np.int64)) and np.array_equal(rc.view(np.int64), rp.view(np.int64))
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        jacc.Kernel(jacc.STENCIL_5PT, jacc.F32, nx, ny, 1, cluster=True)
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, 4096, 4096, 1, cluster=True)
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, 16, 16, 16, coeffs=(0.1,), cluster=True)


# ----------------------------------------------------------------------------- 7-point heat

@pytest.mark.parametrize("tile", range(24))
def test_heat3d_f64_all_tiles(orc, tile):
    nz, ny, nx = 37, 21, 134
    u = inputs.heat3d_field(nx, seed=2, ny=ny, nz=nz)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,), tile_id=tile)
    assert k.info()["fixed_point"]
    g, gr = run(k, u, 5)
    o, orr = orc.heat3d_run(u, 0.125, 5)
    assert nerr(g, o) <= TOL64
    assert_resid(gr, orr, np.max(np.abs(u)))


@pytest.mark.parametrize("r,fixed", [(0.1, True), (1.0 / 16, True), (1.0 / 6, True), (0.2, False), (0.0, True)])
def test_heat3d_coefficient_paths(orc, r, fixed):
    nz, ny, nx = 19, 23, 66
    rng = np.random.default_rng(3)
    u = rng.uniform(-2.0, 3.0, (nz, ny, nx))
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(r,))
    assert k.info()["fixed_point"] == fixed
    g, gr = run(k, u, 4)
    o, orr = orc.heat3d_run(u, r, 4)
    assert nerr(g, o) <= TOL64
    assert_resid(gr, orr, np.max(np.abs(u)))


def test_heat3d_native_path_and_nonfinite_input(orc):
    nz, ny, nx = 12, 14, 40
    u = inputs.heat3d_field(nx, ny=ny, nz=nz, seed=5)
    o, orr = orc.heat3d_run(u, 0.125, 3)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,), arith=jacc.ARITH_NATIVE)
    g, gr = run(k, u, 3)
    assert nerr(g, o) <= TOL64
    assert_resid(gr, orr, np.max(np.abs(u)))
    # a NaN in the input routes the sweep to the native path: NaN propagates like IEEE FP64
    u2 = u.copy()
    u2[5, 6, 7] = np.nan
    k2 = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,))
    g2, _ = run(k2, u2, 1)
    o2, _ = orc.heat3d_sweep(u2, 0.125)
    assert np.array_equal(np.isnan(g2), np.isnan(o2))
    m = ~np.isnan(o2)
    assert nerr(g2[m], o2[m]) <= TOL64


@pytest.mark.parametrize("tile", [3, 9, 15, 21])
def test_heat3d_f32(orc, tile):
    nz, ny, nx = 20, 18, 136
    u = inputs.heat3d_field(nx, ny=ny, nz=nz, seed=2).astype(np.float32)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F32, nx, ny, nz, coeffs=(0.125,), tile_id=tile)
    g, gr = run(k, u, 4)
    o, orr = orc.heat3d_run(u.astype(np.float64), 0.125, 4)
    assert nerr(g, o) <= TOL32
    assert_resid(gr, orr, np.max(np.abs(u)), fp64=False)


@pytest.mark.parametrize("dtype", [jacc.F64, jacc.F32])
@pytest.mark.parametrize("tile", [1, 3, 7, 13, 19, 23])
@pytest.mark.parametrize("shape", [(3, 3, 4), (4, 17, 8), (33, 5, 12), (18, 9, 264)])
def test_heat3d_staged_small_and_ragged(orc, dtype, tile, shape):
    # 16-byte-column tiles stage planes with bulk copies: one-point interiors,
    # widths below one tile, z chunks holding only a boundary plane
    nz, ny, nx = shape
    u = inputs.heat3d_field(nx, ny=ny, nz=nz, seed=7)
    if dtype == jacc.F32:
        u = u.astype(np.float32)
    k = jacc.Kernel(jacc.STENCIL_7PT, dtype, nx, ny, nz, coeffs=(0.125,), tile_id=tile)
    g, gr = run(k, u, 3)
    o, orr = orc.heat3d_run(u.astype(np.float64), 0.125, 3)
    tol = TOL64 if dtype == jacc.F64 else TOL32
    assert nerr(g, o) <= tol
    assert_resid(gr, orr, np.max(np.abs(u)), fp64=dtype == jacc.F64)
    assert k.status() == 0


@pytest.mark.parametrize("dtype", [jacc.F64, jacc.F32])
def test_heat3d_staged_wait_timeout_is_reported_and_recoverable(orc, dtype):
    nz, ny, nx = 30, 20, 128
    u = inputs.heat3d_field(nx, ny=ny, nz=nz, seed=8)
    if dtype == jacc.F32:
        u = u.astype(np.float32)
    k = jacc.Kernel(jacc.STENCIL_7PT, dtype, nx, ny, nz, coeffs=(0.125,), tile_id=3)
    k.set_wait(timeout_ms=20, stall_plane=2)
    run(k, u, 3, graph=False)
    assert k.status() == jacc.ERR_TIMEOUT
    k.set_wait()
    g, _ = run(k, u, 3)
    o, _ = orc.heat3d_run(u.astype(np.float64), 0.125, 3)
    assert nerr(g, o) <= (TOL64 if dtype == jacc.F64 else TOL32)
    assert k.status() == 0


# ----------------------------------------------------------------------------- 27-point periodic box

W = inputs.box27_weights()


@pytest.mark.parametrize("tile", range(24))
def test_box27_f32_all_tiles(orc, tile):
    nz, ny, nx = 35, 11, 140
    u = inputs.box27_field(nx, ny, nz, seed=6)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tile_id=tile)
    g, gs = run(k, u, 4)
    o, osum = orc.box27_run(u, W, 4)
    assert nerr(g, o) <= TOL32
    A = float(np.sum(np.abs(o.astype(np.float64))))
    assert np.max(np.abs(gs - osum)) <= 1e-6 * A


@pytest.mark.parametrize("tile", [0, 7, 13, 23])
def test_box27_f64(orc, tile):
    nz, ny, nx = 18, 13, 70
    u = inputs.box27_field(nx, ny, nz, seed=9).astype(np.float64)
    w64 = W.astype(np.float64)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F64, nx, ny, nz, coeffs=tuple(w64), tile_id=tile)
    assert k.info()["fixed_point"]
    g, gs = run(k, u, 3)
    o, sums = orc.box27_run_f64(u, w64, 3)
    assert nerr(g, o) <= TOL64
    assert np.max(np.abs(gs - np.array(sums))) <= 1e-12 * float(np.sum(np.abs(o)))


def test_box27_f64_large_field_with_input_conversion(orc):
    # at least 2^22 points: the sequence converts u0 in place before its first
    # sweep, which then runs the intermediate kernel (plain and folded)
    nz, ny, nx = 64, 256, 258  # 4.23 M points
    u = inputs.box27_field(nx, ny, nz, seed=19).astype(np.float64)
    w64 = W.astype(np.float64)
    o, sums = orc.box27_run_f64(u, w64, 3)
    for jit in (False, True):
        k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F64, nx, ny, nz, coeffs=tuple(w64), jit=jit)
        assert k.info()["fixed_point"]
        g, gs = run(k, u, 3)
        assert nerr(g, o) <= TOL64
        assert np.max(np.abs(gs - np.array(sums))) <= 1e-12 * float(np.sum(np.abs(o)))


def test_box27_impulse_response_exact():
    nz, ny, nx = 6, 7, 8
    u = np.zeros((nz, ny, nx), dtype=np.float32)
    u[0, 0, 0] = 1.0
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tile_id=0)
    g, _ = run(k, u, 1)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                assert g[dz % nz, dy % ny, dx % nx] == W[(dz != 0) + (dy != 0) + (dx != 0)]
    assert np.count_nonzero(g) == 27


@pytest.mark.parametrize("tile", [1, 3, 11, 23])
@pytest.mark.parametrize("shape", [(3, 3, 4), (5, 17, 8), (4, 3, 524), (70, 9, 12)])
def test_box27_f32_staged_small_and_ragged(orc, tile, shape):
    # 16-byte-column tiles stage planes with bulk copies: widths below one
    # tile, rows and planes that wrap several times, a 4-wide halo at nx = 4
    nz, ny, nx = shape
    u = inputs.box27_field(nx, ny, nz, seed=12)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tile_id=tile)
    g, gs = run(k, u, 3)
    o, osum = orc.box27_run(u, W, 3)
    assert nerr(g, o) <= TOL32
    assert np.max(np.abs(gs - osum)) <= 1e-6 * float(np.sum(np.abs(o.astype(np.float64))))
    assert k.status() == 0


@pytest.mark.parametrize("tile", [1, 3])
def test_box27_staged_impulse_response_exact(tile):
    nz, ny, nx = 6, 7, 8
    u = np.zeros((nz, ny, nx), dtype=np.float32)
    u[0, 0, 0] = 1.0
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tile_id=tile)
    g, _ = run(k, u, 1)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                assert g[dz % nz, dy % ny, dx % nx] == W[(dz != 0) + (dy != 0) + (dx != 0)]
    assert np.count_nonzero(g) == 27


def test_box27_staged_wait_timeout_is_reported_and_recoverable(orc):
    # CTA (0,0,0) never requests staged plane 3: its mbarrier waits run out
    # after 20 ms, the status word says TIMEOUT, and the context stays usable
    nz, ny, nx = 40, 20, 256
    u = inputs.box27_field(nx, ny, nz, seed=13)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tile_id=3)
    assert k.status() == 0
    k.set_wait(timeout_ms=20, stall_plane=3)
    run(k, u, 1, graph=False)
    assert k.status() == jacc.ERR_TIMEOUT
    assert k.status() == 0  # reading clears it
    k.set_wait()
    g, _ = run(k, u, 2)
    o, _ = orc.box27_run(u, W, 2)
    assert nerr(g, o) <= TOL32
    assert k.status() == 0


# ----------------------------------------------------------------------------- specialisation and graphs

@pytest.mark.parametrize("stencil,dtype,shape,coeffs", [
    (5, 64, (1, 70, 134), ()), (7, 64, (21, 22, 70), (0.125,)), (7, 64, (21, 22, 70), (0.1,)),
    (27, 32, (12, 13, 64), tuple(float(w) for w in W)), (7, 32, (21, 22, 72), (0.125,))])
def test_jit_variant_matches_generic(stencil, dtype, shape, coeffs):
    nz, ny, nx = shape
    rng = np.random.default_rng(1)
    u = rng.uniform(0, 1, (ny, nx) if stencil == 5 else shape)
    if dtype == 32:
        u = u.astype(np.float32)
    kg = jacc.Kernel(stencil, dtype, nx, ny, nz, coeffs=coeffs)
    kj = jacc.Kernel(stencil, dtype, nx, ny, nz, coeffs=coeffs, jit=True)
    assert kj.info()["jit"] and not kg.info()["jit"]
    g1, r1 = run(kg, u, 3)
    g2, r2 = run(kj, u, 3)
    if dtype == 64:
        assert np.array_equal(g1, g2) and np.array_equal(r1, r2)  # integer arithmetic: bit-identical
    else:
        assert nerr(g2, g1) <= TOL32


@pytest.mark.parametrize("stencil,dtype,shape,coeffs", [
    (7, 64, (90, 22, 70), (0.125,)), (27, 32, (90, 13, 64), tuple(float(w) for w in W))])
def test_folded_long_march_takes_shallower_chunks_and_matches(stencil, dtype, shape, coeffs):
    # the folded variant of a staged long-march tile marches 40 planes per CTA
    # (27-point: 32; the precompiled one 64); both give the same field and
    # residuals
    nz, ny, nx = shape
    rng = np.random.default_rng(2)
    u = rng.uniform(0, 1, shape)
    if dtype == 32:
        u = u.astype(np.float32)
    kg = jacc.Kernel(stencil, dtype, nx, ny, nz, coeffs=coeffs, tile_id=3)
    kj = jacc.Kernel(stencil, dtype, nx, ny, nz, coeffs=coeffs, tile_id=3, jit=True)
    zc = 32 if stencil == 27 else 40
    assert kg.info()["grid"][2] == (nz + 63) // 64 and kj.info()["grid"][2] == (nz + zc - 1) // zc
    g1, r1 = run(kg, u, 4)
    g2, r2 = run(kj, u, 4)
    if dtype == 64:
        assert np.array_equal(g1, g2) and np.array_equal(r1, r2)
    else:
        assert nerr(g2, g1) <= TOL32


def test_graph_and_eager_sweeps_agree_and_cache():
    nz, ny, nx = 16, 16, 64
    u = inputs.heat3d_field(nx, ny=ny, nz=nz, seed=3)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,))
    k2 = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,))
    assert k.handle.value == k2.handle.value  # cache hit shares the compiled kernel
    g1, r1 = run(k, u, 6, graph=True)
    g2, r2 = run(k, u, 6, graph=False)
    assert np.array_equal(g1, g2) and np.array_equal(r1, r2)
    # replay of the cached graph on the same buffers
    a = torch.from_numpy(u).to(DEV)
    b = torch.zeros_like(a)
    res = torch.zeros(6, dtype=torch.float64, device=DEV)
    for _ in range(3):
        a.copy_(torch.from_numpy(u))
        fb = jacc.sweep(k, a, b, 6, res)
    torch.cuda.synchronize()
    assert np.array_equal((a if fb == 0 else b).cpu().numpy(), g1)


def test_launch_single_sweep_and_errors(orc):
    nz, ny, nx = 10, 12, 34
    u = inputs.heat3d_field(nx, ny=ny, nz=nz, seed=4)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, nx, ny, nz, coeffs=(0.125,))
    a = torch.from_numpy(u).to(DEV)
    b = torch.empty_like(a)
    r = torch.zeros(1, dtype=torch.float64, device=DEV)
    jacc.launch(k, a, b, r)
    torch.cuda.synchronize()
    o, orr = orc.heat3d_sweep(u, 0.125)
    assert nerr(b.cpu().numpy(), o) <= TOL64
    assert_resid([r.item()], [orr], np.max(np.abs(u)))
    with pytest.raises(jacc.JaccError) as e:
        jacc.launch(k, a, a, r)  # in-place is aliasing
    assert e.value.status == jacc.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        jacc.launch(k, a.float(), b)
    with pytest.raises(jacc.JaccError):
        jacc.sweep(k, a, b, 0)


# ----------------------------------------------------------------------------- temporal blocking (27-point FP32)

@pytest.mark.parametrize("T", [2, 3])
def test_box27_temporal_blocking_matches_single_sweeps(orc, T):
    nz, ny, nx = 70, 37, 248  # ragged against the 120 x (16 - 2T) output tiles and 64-plane chunks
    u = inputs.box27_field(nx, ny, nz, seed=6)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tblock=T)
    assert k.info()["tblock"] == T
    ns = 2 * T
    g, gs = run(k, u, ns)
    o, osum = orc.box27_run(u, W, ns)
    assert nerr(g, o) <= TOL32
    A = float(np.sum(np.abs(o.astype(np.float64))))
    for i in range(ns):
        if (i + 1) % T == 0:
            assert abs(gs[i] - osum[i]) <= 1e-6 * A
        else:
            assert np.isnan(gs[i])
    # the same field through the single-sweep kernel
    k1 = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W))
    g1, _ = run(k1, u, ns)
    assert nerr(g, g1) <= TOL32


def test_box27_temporal_blocking_small_periodic_and_errors(orc):
    nz, ny, nx = 5, 7, 12  # smaller than one tile in every axis: wrap inside the region
    u = inputs.box27_field(nx, ny, nz, seed=8)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tblock=2)
    g, _ = run(k, u, 4)
    o, _ = orc.box27_run(u, W, 4)
    assert nerr(g, o) <= TOL32
    a = torch.from_numpy(u).cuda()
    with pytest.raises(jacc.JaccError):
        jacc.sweep(k, a, torch.empty_like(a), 3)  # not a multiple of the depth
    with pytest.raises(jacc.JaccError) as e:
        jacc.Kernel(jacc.STENCIL_27PT, jacc.F64, 12, 7, 5, coeffs=(0.5, 0.05, 0.01, 0.005), tblock=2)
    assert e.value.status == jacc.ERR_UNSUPPORTED


@pytest.mark.parametrize("shape", [(70, 37, 248), (5, 7, 12), (33, 20, 520), (3, 3, 4)])
def test_box27_two_sweep_kernel_bit_identical_to_single_sweeps(orc, shape):
    # the staged two-sweep kernel (rows of a multiple of 4 floats) forms each
    # sweep with the single-sweep staged kernel's arithmetic in the same order:
    # after 2k sweeps its field equals 2k single staged sweeps bit for bit
    nz, ny, nx = shape
    u = inputs.box27_field(nx, ny, nz, seed=14)
    wt = tuple(float(w) for w in W)
    k2 = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=wt, tblock=2)
    k1 = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=wt, tile_id=3)
    g2, s2 = run(k2, u, 6)
    g1, s1 = run(k1, u, 6)
    assert np.array_equal(g2.view(np.int32), g1.view(np.int32))
    o, osum = orc.box27_run(u, W, 6)
    assert nerr(g2, o) <= TOL32
    A = float(np.sum(np.abs(o.astype(np.float64))))
    for i in range(6):
        if (i + 1) % 2:
            assert np.isnan(s2[i])
        else:
            assert abs(s2[i] - osum[i]) <= 1e-6 * A and abs(s2[i] - s1[i]) <= 1e-6 * A
    assert k2.status() == 0


def test_box27_two_sweep_kernel_wait_timeout_is_reported_and_recoverable(orc):
    nz, ny, nx = 40, 20, 256
    u = inputs.box27_field(nx, ny, nz, seed=15)
    k = jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(w) for w in W), tblock=2)
    k.set_wait(timeout_ms=20, stall_plane=3)
    run(k, u, 2, graph=False)
    assert k.status() == jacc.ERR_TIMEOUT
    k.set_wait()
    g, _ = run(k, u, 4)
    o, _ = orc.box27_run(u, W, 4)
    assert nerr(g, o) <= TOL32
    assert k.status() == 0
