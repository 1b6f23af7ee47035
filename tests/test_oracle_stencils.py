"""Pins for the oracle's stencils and reductions (CPU only).

Each pin is a fact the mathematics fixes independently of the oracle's loops:
fixed points, closed-form eigenvalues, impulse responses, conservation laws
and maximum principles.  Grids are anisotropic so that a transposed axis or
operand changes the answer.
"""
import math

import numpy as np
import pytest

from paper_2110_14340_gb300 import inputs


# ----------------------------------------------------------------------------- 5-point Jacobi

def test_jacobi_affine_field_is_exact_fixed_point(orc):
    ny, nx = 9, 13
    y, x = np.mgrid[0:ny, 0:nx]
    u = (3.0 * x - 2.0 * y + 7.0)
    v, res = orc.jacobi2d_run(u, 5)
    assert np.array_equal(v, u)
    assert np.all(res == 0.0)


def test_jacobi_sine_mode_decays_by_eigenvalue(orc):
    # u = sin(pi p x/(nx-1)) sin(pi q y/(ny-1)) with zero boundary is an
    # eigenvector of the 5-point average with eigenvalue (cos(pi p/(nx-1)) + cos(pi q/(ny-1)))/2.
    nx, ny, p, q = 21, 12, 2, 3
    x = np.arange(nx)
    y = np.arange(ny)
    u = np.outer(np.sin(np.pi * q * y / (ny - 1)), np.sin(np.pi * p * x / (nx - 1)))
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    mu = 0.5 * (math.cos(math.pi * p / (nx - 1)) + math.cos(math.pi * q / (ny - 1)))
    v, _ = orc.jacobi2d_run(u, 3)
    assert np.max(np.abs(v - mu ** 3 * u)) <= 1e-15
    # the transposed eigenvalue differs, so an axis swap would be caught
    mu_t = 0.5 * (math.cos(math.pi * p / (ny - 1)) + math.cos(math.pi * q / (nx - 1)))
    assert abs(mu - mu_t) > 1e-2


def test_jacobi_impulse_response(orc):
    u = np.zeros((7, 9))
    u[3, 4] = 1.0
    v, r = orc.jacobi2d_sweep(u)
    expect = np.zeros_like(u)
    expect[2, 4] = expect[4, 4] = expect[3, 3] = expect[3, 5] = 0.25
    assert np.array_equal(v, expect)
    assert r == 1.0


def test_jacobi_max_principle_and_monotone_residual(orc):
    u = inputs.jacobi2d_field(64, 48, seed=1)
    v, res = orc.jacobi2d_run(u, 60)
    assert v.min() >= 0.0 and v.max() <= 1.0
    assert np.all(res[1:] <= res[:-1] + 4e-16)
    # boundary is held
    assert np.all(v[0, :] == 1.0) and np.all(v[:, -1] == 1.0)


# ----------------------------------------------------------------------------- 7-point heat

def heat_mode(nx, ny, nz, p, q, s):
    fx = np.sin(np.pi * p * np.arange(nx) / (nx - 1))
    fy = np.sin(np.pi * q * np.arange(ny) / (ny - 1))
    fz = np.sin(np.pi * s * np.arange(nz) / (nz - 1))
    u = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    u[0] = u[-1] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    u[:, :, 0] = u[:, :, -1] = 0.0
    return u


def heat_lambda(r, nx, ny, nz, p, q, s):
    # Each axis contributes -4 sin^2(pi k / (2 (n - 1))) to the discrete Laplacian's eigenvalue.
    t = sum(math.sin(math.pi * k / (2 * (n - 1))) ** 2 for k, n in ((p, nx), (q, ny), (s, nz)))
    return 1.0 - 4.0 * r * t


def test_heat_eigenmode_decay(orc):
    nx, ny, nz, p, q, s = 12, 15, 18, 1, 2, 3
    r = 0.125
    u = heat_mode(nx, ny, nz, p, q, s)
    lam = heat_lambda(r, nx, ny, nz, p, q, s)
    v, _ = orc.heat3d_run(u, r, 10)
    assert np.max(np.abs(v - lam ** 10 * u)) <= 1e-14 * np.max(np.abs(u))


def test_heat_affine_fixed_point_and_max_principle(orc):
    z, y, x = np.mgrid[0:6, 0:7, 0:9]
    u = 2.0 * x - 3.0 * y + 5.0 * z + 1.0
    v, res = orc.heat3d_run(u, 0.125, 4)
    assert np.array_equal(v, u) and np.all(res == 0.0)
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, size=(10, 11, 12))
    prev = np.max(np.abs(u))
    a = u
    for _ in range(5):
        a, _ = orc.heat3d_sweep(a, 1.0 / 6.0)
        cur = np.max(np.abs(a))
        assert cur <= prev + 1e-15
        prev = cur


def test_heat_projection_on_noisy_field(orc):
    # The operator is symmetric, so the component along the eigenmode phi
    # decays by exactly lambda per step even with noise present.
    n = 17
    u = inputs.heat3d_field(n, seed=2)
    phi = heat_mode(n, n, n, 1, 1, 1)
    lam = heat_lambda(0.125, n, n, n, 1, 1, 1)
    c0 = np.sum(u * phi) / np.sum(phi * phi)
    v, _ = orc.heat3d_run(u, 0.125, 20)
    c20 = np.sum(v * phi) / np.sum(phi * phi)
    assert abs(c20 - lam ** 20 * c0) <= 1e-13


# ----------------------------------------------------------------------------- 27-point periodic box

W = inputs.box27_weights()


def test_box27_weights_sum_to_one():
    w = W.astype(np.float64)
    assert abs(w[0] + 6 * w[1] + 12 * w[2] + 8 * w[3] - 1.0) < 1e-7
    assert abs(W[0] - 6 / 11) < 1e-7 and abs(W[3] - 1 / 176) < 1e-9


@pytest.mark.parametrize("at", [(0, 0, 0), (2, 3, 4)])
def test_box27_impulse_response_is_class_weights(orc, at):
    nz, ny, nx = 5, 6, 7
    u = np.zeros((nz, ny, nx), dtype=np.float32)
    u[at] = 1.0
    v = orc.box27_sweep(u, W)
    expect = np.zeros_like(u)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                cls = (dz != 0) + (dy != 0) + (dx != 0)
                expect[(at[0] + dz) % nz, (at[1] + dy) % ny, (at[2] + dx) % nx] = W[cls]
    assert np.array_equal(v, expect)


def test_box27_constant_and_sum(orc):
    Wsum = float(W[0]) + 6 * float(W[1]) + 12 * float(W[2]) + 8 * float(W[3])
    u = np.full((4, 5, 6), 0.75, dtype=np.float32)
    v = orc.box27_sweep(u, W)
    assert np.max(np.abs(v.astype(np.float64) - 0.75 * Wsum)) <= 2e-7
    u = inputs.box27_field(10, 9, 8, seed=6)
    n = 12
    v, sums = orc.box27_run(u, W, n)
    S0 = orc.sum_f32(u)
    A = float(np.sum(np.abs(u.astype(np.float64))))
    for k in range(n):
        assert abs(sums[k] - Wsum ** (k + 1) * S0) <= 1e-6 * A
    assert sums[-1] == orc.sum_f32(v)


def test_box27_plane_wave_symbol(orc):
    nz, ny, nx = 10, 12, 16
    kz, ky, kx = 1, 2, 3
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    ph = 2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz)
    u = np.cos(ph).astype(np.float32)
    cx, cy, cz = (math.cos(2 * math.pi * k / n) for k, n in ((kx, nx), (ky, ny), (kz, nz)))
    w = W.astype(np.float64)
    sym = w[0] + 2 * w[1] * (cx + cy + cz) + 4 * w[2] * (cx * cy + cx * cz + cy * cz) + 8 * w[3] * cx * cy * cz
    v = orc.box27_sweep(u, W)
    assert np.max(np.abs(v - sym * np.cos(ph))) <= 2e-6
    # swapping edge and corner weights changes the symbol by more than the tolerance
    sym_bad = w[0] + 2 * w[1] * (cx + cy + cz) + 4 * w[3] * (cx * cy + cx * cz + cy * cz) + 8 * w[2] * cx * cy * cz
    assert abs(sym - sym_bad) > 1e-3


# ----------------------------------------------------------------------------- reductions

def test_sums_and_maxabs(orc):
    rng = np.random.default_rng(5)
    for n in (0, 1, 7, 9, 1000, 123457):
        a = rng.uniform(-1, 1, n)
        s = orc.sum_f64(a)
        exact = math.fsum(a)
        bound = (math.log2(max(n, 2)) + 8) * 2.0 ** -53 * float(np.sum(np.abs(a)))
        assert abs(s - exact) <= bound
        f = a.astype(np.float32)
        assert abs(orc.sum_f32(f) - math.fsum(f.astype(np.float64))) <= bound + 1e-300
        b = rng.uniform(-1, 1, n)
        assert orc.maxabs_diff(a, b) == (float(np.max(np.abs(a - b))) if n else 0.0)


def test_box27_f64_pins(orc):
    # FP64 variant: impulse response is the weights exactly; the plane-wave symbol holds to FP64 rounding.
    w = np.array([6 / 11, 1 / 22, 1 / 88, 1 / 176])
    nz, ny, nx = 10, 12, 16
    u = np.zeros((nz, ny, nx))
    u[1, 2, 3] = 1.0
    v, _ = orc.box27_run_f64(u, w, 1)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                assert v[1 + dz, 2 + dy, 3 + dx] == w[(dz != 0) + (dy != 0) + (dx != 0)]
    assert np.count_nonzero(v) == 27
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    ph = 2 * np.pi * (3 * x / nx + 2 * y / ny + 1 * z / nz)
    cx, cy, cz = (math.cos(2 * math.pi * k / n) for k, n in ((3, nx), (2, ny), (1, nz)))
    sym = w[0] + 2 * w[1] * (cx + cy + cz) + 4 * w[2] * (cx * cy + cx * cz + cy * cz) + 8 * w[3] * cx * cy * cz
    v, sums = orc.box27_run_f64(np.cos(ph), w, 2)
    assert np.max(np.abs(v - sym ** 2 * np.cos(ph))) <= 1e-14
