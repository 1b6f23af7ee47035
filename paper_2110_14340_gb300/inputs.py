"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the stencil method: it only draws numbers.
The generator is counter-based so any element can be produced independently
of the others (on the host with numpy, or on a device with torch):

    mix(z)    = the SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014):
                z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
    key(s, t) = mix(mix(s) + t * G)        G = 0x9E3779B97F4A7C15 (stream t)
    bits(i)   = mix(key + (i + 1) * G)     (all arithmetic mod 2^64)
    U64[0,1)  = (bits >> 11) * 2^-53
    U32[0,1)  = (bits >> 40) * 2^-24

Workload recipes (shapes, value ranges and seeds):
    jacobi2d_field   interior U64[0,1), boundary rows/columns = bval (1.0)
    heat3d_field     sin(pi x) sin(pi y) sin(pi z) + 1e-3 U64[0,1) on the
                     interior, x_i = i/(N-1); boundary exactly 0.0
    box27_field      U32[-1,1) = 2 U32 - 1 (exact in FP32)
    batched_shapes   nx, ny = round(exp(U64(ln 128, ln 2048))) per grid
"""
import math

import numpy as np

G = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix(z):
    z = z ^ (z >> np.uint64(30))
    z = z * M1
    z = z ^ (z >> np.uint64(27))
    z = z * M2
    return z ^ (z >> np.uint64(31))


def key(seed, stream=0):
    with np.errstate(over="ignore"):
        s = _mix(np.array([seed], dtype=np.uint64))
        return _mix(s + np.uint64(stream) * G)[0]


def bits(seed, n, stream=0, start=0):
    """uint64 words i = start .. start+n-1 of stream (seed, stream)."""
    k = key(seed, stream)
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for c0 in range(0, n, _CHUNK):
            c1 = min(n, c0 + _CHUNK)
            i = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
            out[c0:c1] = _mix(k + i * G)
    return out


def uniform64(seed, n, stream=0):
    return (bits(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform32(seed, n, stream=0):
    return ((bits(seed, n, stream) >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)


# ----------------------------------------------------------------------------- torch (device) variant

def uniform_torch(seed, n, device, dtype, stream=0):
    """Same numbers as uniform64 / uniform32, drawn with torch int64 ops on `device`.

    int64 multiply/add wrap mod 2^64 exactly like uint64; logical right shifts
    are emulated with a mask.
    """
    import torch
    k = int(key(seed, stream))
    k = k - (1 << 64) if k >= (1 << 63) else k
    g = int(G) - (1 << 64)
    m1 = int(M1) - (1 << 64)
    m2 = int(M2) - (1 << 64)

    def srl(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    out = torch.empty(n, dtype=dtype, device=device)
    chunk = 1 << 26
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        z = torch.arange(c0 + 1, c1 + 1, dtype=torch.int64, device=device)
        z = z * g + k
        z = z ^ srl(z, 30)
        z = z * m1
        z = z ^ srl(z, 27)
        z = z * m2
        z = z ^ srl(z, 31)
        if dtype == torch.float64:
            out[c0:c1] = srl(z, 11).to(torch.float64) * (2.0 ** -53)
        else:
            out[c0:c1] = srl(z, 40).to(torch.float32) * (2.0 ** -24)
    return out


# ----------------------------------------------------------------------------- workload fields

def jacobi2d_field(nx, ny, seed=1, bval=1.0, stream=0):
    u = uniform64(seed, nx * ny, stream).reshape(ny, nx)
    u[0, :] = bval
    u[-1, :] = bval
    u[:, 0] = bval
    u[:, -1] = bval
    return u


def heat3d_field(n, seed=2, noise=1e-3, ny=None, nz=None):
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    sx = np.sin(np.pi * np.arange(nx) / (nx - 1))
    sy = np.sin(np.pi * np.arange(ny) / (ny - 1))
    sz = np.sin(np.pi * np.arange(nz) / (nz - 1))
    u = np.empty((nz, ny, nx), dtype=np.float64)
    with np.errstate(over="ignore"):
        for z in range(nz):
            plane = np.outer(sy, sx) * sz[z]
            if noise:
                plane = plane + noise * (bits(seed, nx * ny, 0, z * nx * ny) >> np.uint64(11)).astype(
                    np.float64).reshape(ny, nx) * (2.0 ** -53)
            u[z] = plane
    u[0] = 0.0
    u[-1] = 0.0
    u[:, 0, :] = 0.0
    u[:, -1, :] = 0.0
    u[:, :, 0] = 0.0
    u[:, :, -1] = 0.0
    return u


def box27_field(nx, ny=None, nz=None, seed=6):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    u = uniform32(seed, nx * ny * nz)
    return (np.float32(2.0) * u - np.float32(1.0)).astype(np.float32).reshape(nz, ny, nx)


def var19_problem(nx, ny, nz, seed=7):
    """Synthetic input of the variable-coefficient 19-point stencil: the iterate
    p ~ U[0,1) and the twelve coefficient fields (a0 a1 a2 a3 b0 b1 b2 c0 c1 c2
    wrk1 bnd), all FP32 of shape (nz, ny, nx).  Face coefficients a_i, c_i =
    1 + 0.1 U[-1,1); cross coefficients b_i = 0.05 U[-1,1); a3 = 1 / (sum of
    the six face coefficients), so s0 a3 is close to a weighted average; source
    wrk1 = 0.01 U[-1,1); bnd = 1.  Stream k of the generator fills field k."""
    n = nx * ny * nz
    shape = (nz, ny, nx)

    def sym(stream, scale):
        return (np.float32(scale) * (np.float32(2.0) * uniform32(seed, n, stream) - np.float32(1.0))).reshape(shape)

    p = uniform32(seed, n, 0).reshape(shape)
    a = [(np.float32(1.0) + sym(1 + i, 0.1)).astype(np.float32) for i in range(3)]
    c = [(np.float32(1.0) + sym(4 + i, 0.1)).astype(np.float32) for i in range(3)]
    b = [sym(7 + i, 0.05).astype(np.float32) for i in range(3)]
    tot = a[0] + a[1] + a[2] + c[0] + c[1] + c[2]
    a3 = (np.float32(1.0) / tot).astype(np.float32)
    wrk1 = sym(10, 0.01).astype(np.float32)
    bnd = np.ones(shape, dtype=np.float32)
    return p.astype(np.float32), [a[0], a[1], a[2], a3, b[0], b[1], b[2], c[0], c[1], c[2], wrk1, bnd]


def var19_problem_torch(nx, ny, nz, device, seed=7):
    """var19_problem's fields generated on `device` with torch (same numbers)."""
    import torch
    n = nx * ny * nz
    shape = (nz, ny, nx)

    def sym(stream, scale):
        u = uniform_torch(seed, n, device, torch.float32, stream)
        return (scale * (2.0 * u - 1.0)).view(shape)

    p = uniform_torch(seed, n, device, torch.float32, 0).view(shape)
    a = [1.0 + sym(1 + i, 0.1) for i in range(3)]
    c = [1.0 + sym(4 + i, 0.1) for i in range(3)]
    b = [sym(7 + i, 0.05) for i in range(3)]
    a3 = 1.0 / (((((a[0] + a[1]) + a[2]) + c[0]) + c[1]) + c[2])
    wrk1 = sym(10, 0.01)
    bnd = torch.ones(shape, dtype=torch.float32, device=device)
    return p, [a[0], a[1], a[2], a3, b[0], b[1], b[2], c[0], c[1], c[2], wrk1, bnd]


def batched_shapes(ngrids=64, seed=3, lo=128, hi=2048):
    u = uniform64(seed, 2 * ngrids)
    a, b = math.log(lo), math.log(hi)
    sides = np.rint(np.exp(a + (b - a) * u)).astype(np.int64)
    return [(int(sides[2 * g]), int(sides[2 * g + 1])) for g in range(ngrids)]


def batched_fields(shapes, seed=4, bval=1.0):
    return [jacobi2d_field(nx, ny, seed=seed, bval=bval, stream=g + 1) for g, (nx, ny) in enumerate(shapes)]


def box27_weights():
    """Class weights (centre, face, edge, corner) = (1/2, 1/24, 1/96, 1/192) scaled to sum 1.

    Raw sum = 1/2 + 6/24 + 12/96 + 8/192 = 11/12, so the scaled weights are
    6/11, 1/22, 1/88, 1/176, rounded to FP32."""
    return np.array([6.0 / 11.0, 1.0 / 22.0, 1.0 / 88.0, 1.0 / 176.0], dtype=np.float32)


# ----------------------------------------------------------------------------- cost-model inputs

MLP_NPARAM = 8705


def mlp_init(seed=5):
    """Kaiming-uniform parameters (He et al. 2015) for the 4-64-64-64-1 ReLU MLP:
    weights U(-sqrt(6/fan_in), sqrt(6/fan_in)) drawn in layer order from stream 0
    of `seed`, biases 0; FP32.  Layout W1[64][4] b1 W2[64][64] b2 W3[64][64] b3 W4[64] b4."""
    fan = (4, 64, 64, 64)
    off = (0, 320, 4480, 8640)
    cnt = (256, 4096, 4096, 64)
    u = uniform64(seed, sum(cnt))
    p = np.zeros(MLP_NPARAM, dtype=np.float32)
    k = 0
    for f, o, c in zip(fan, off, cnt):
        b = math.sqrt(6.0 / f)
        p[o:o + c] = ((2.0 * u[k:k + c] - 1.0) * b).astype(np.float32)
        k += c
    return p


def mlp_dataset(seed, n):
    """Synthetic regression set: x ~ U[0,1)^4 (FP32), target a smooth function of x."""
    x = uniform64(seed, 4 * n).reshape(n, 4)
    y = np.sin(3.0 * x[:, 0]) + x[:, 1] ** 2 - x[:, 2] * x[:, 3] + 0.5 * x[:, 3]
    return x.astype(np.float32), y.astype(np.float32)
