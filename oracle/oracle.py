"""ctypes marshalling for liboracle.so (test infrastructure only).

Every function here converts numpy arrays to pointers and calls the C
definition in oracle.c; no arithmetic of the method lives in this file.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB, build

MAX_DIMS = 8
MAX_LOOPS = 8
NPARAM = 8705

OK, ERR_INVALID_ARG, ERR_OUT_OF_BOUNDS, ERR_OVERFLOW = 0, -1, -2, -3


class Loop(C.Structure):
    _fields_ = [("lo", C.c_int64), ("hi", C.c_int64), ("step", C.c_int64)]


class Ref(C.Structure):
    _fields_ = [("array_id", C.c_int32), ("ndim", C.c_int32), ("is_write", C.c_int32), ("pad_", C.c_int32),
                ("coef", (C.c_int64 * MAX_LOOPS) * MAX_DIMS), ("off", C.c_int64 * MAX_DIMS)]


class Array(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("pad_", C.c_int32), ("extent", C.c_int64 * MAX_DIMS)]


class LoopAffine(C.Structure):
    _fields_ = [("lo", C.c_int64), ("hi", C.c_int64), ("lo_coef", C.c_int64 * MAX_LOOPS),
                ("hi_coef", C.c_int64 * MAX_LOOPS)]


class Region(C.Structure):
    _fields_ = [("has_read", C.c_int32), ("has_write", C.c_int32),
                ("rlo", C.c_int64 * MAX_DIMS), ("rhi", C.c_int64 * MAX_DIMS),
                ("wlo", C.c_int64 * MAX_DIMS), ("whi", C.c_int64 * MAX_DIMS),
                ("rlin_lo", C.c_int64), ("rlin_hi", C.c_int64), ("wlin_lo", C.c_int64), ("wlin_hi", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = LIB if os.path.exists(LIB) else build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_region_analyze.restype = C.c_int
        L.orc_region_analyze.argtypes = [C.c_int32, P, C.c_int32, P, C.c_int32, P, P]
        L.orc_jacobi2d_sweep.restype = C.c_double
        L.orc_jacobi2d_sweep.argtypes = [C.c_int64, C.c_int64, P, P]
        L.orc_jacobi2d_run.restype = C.c_int
        L.orc_jacobi2d_run.argtypes = [C.c_int64, C.c_int64, P, P, C.c_int32, P]
        L.orc_heat3d_sweep.restype = C.c_double
        L.orc_heat3d_sweep.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double, P, P]
        L.orc_heat3d_run.restype = C.c_int
        L.orc_heat3d_run.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double, P, P, C.c_int32, P]
        L.orc_box27_sweep.restype = None
        L.orc_box27_sweep.argtypes = [C.c_int64, C.c_int64, C.c_int64, P, P, P]
        L.orc_box27_run.restype = C.c_int
        L.orc_box27_run.argtypes = [C.c_int64, C.c_int64, C.c_int64, P, P, P, C.c_int32, P]
        L.orc_box27_sweep_f64.restype = None
        L.orc_box27_sweep_f64.argtypes = [C.c_int64, C.c_int64, C.c_int64, P, P, P]
        L.orc_box27_run_f64.restype = C.c_int
        L.orc_box27_run_f64.argtypes = [C.c_int64, C.c_int64, C.c_int64, P, P, P, C.c_int32, P]
        L.orc_region_enumerate_affine.restype = C.c_int
        L.orc_region_enumerate_affine.argtypes = [C.c_int32, P, C.c_int32, P, C.c_int32, P, P]
        L.orc_var19_sweep.restype = C.c_double
        L.orc_var19_sweep.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_float, P, P, P]
        L.orc_var19_run.restype = C.c_int
        L.orc_var19_run.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_float, P, P, P, C.c_int32, P]
        L.orc_maxabs_diff.restype = C.c_double
        L.orc_maxabs_diff.argtypes = [P, P, C.c_int64]
        L.orc_sum_f64.restype = C.c_double
        L.orc_sum_f64.argtypes = [P, C.c_int64]
        L.orc_sum_f32.restype = C.c_double
        L.orc_sum_f32.argtypes = [P, C.c_int64]
        L.orc_mlp_forward.restype = None
        L.orc_mlp_forward.argtypes = [P, P, C.c_int64, P]
        L.orc_mlp_loss_grad.restype = C.c_double
        L.orc_mlp_loss_grad.argtypes = [P, P, P, C.c_int64, P]
        L.orc_adam_step.restype = None
        L.orc_adam_step.argtypes = [P, P, P, P, C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_double,
                                    C.c_double]
        L.orc_set_threads.restype = C.c_int32
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_get_threads.restype = C.c_int32
        L.orc_get_threads.argtypes = []
        L.orc_regret.restype = None
        L.orc_regret.argtypes = [P, C.c_int32, C.c_int32, P, P]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ----------------------------------------------------------------------------- region analysis

def make_nest(loops, refs, arrays):
    """Pack Python descriptions into ctypes arrays.

    loops:  [(lo, hi, step), ...]
    refs:   [dict(array=a, write=bool, coef=[[c_dk]*nloops]*ndim, off=[off_d]*ndim), ...]
    arrays: [[extent_0, ...], ...]
    """
    L = (Loop * max(1, len(loops)))()
    for k, (lo, hi, st) in enumerate(loops):
        L[k].lo, L[k].hi, L[k].step = lo, hi, st
    R = (Ref * max(1, len(refs)))()
    for r, ref in enumerate(refs):
        R[r].array_id = ref["array"]
        R[r].ndim = len(ref["off"])
        R[r].is_write = 1 if ref.get("write") else 0
        for d, row in enumerate(ref["coef"]):
            for k, c in enumerate(row):
                R[r].coef[d][k] = c
        for d, o in enumerate(ref["off"]):
            R[r].off[d] = o
    A = (Array * max(1, len(arrays)))()
    for a, ext in enumerate(arrays):
        A[a].ndim = len(ext)
        for d, e in enumerate(ext):
            A[a].extent[d] = e
    return L, R, A


def region_analyze(loops, refs, arrays):
    """Returns (status, [dict per array])."""
    L, R, A = make_nest(loops, refs, arrays)
    O = (Region * max(1, len(arrays)))()
    st = lib().orc_region_analyze(len(loops), C.cast(L, C.c_void_p), len(refs), C.cast(R, C.c_void_p),
                                  len(arrays), C.cast(A, C.c_void_p), C.cast(O, C.c_void_p))
    out = []
    for a, ext in enumerate(arrays):
        nd = len(ext)
        o = O[a]
        out.append(dict(has_read=bool(o.has_read), has_write=bool(o.has_write),
                        rlo=list(o.rlo[:nd]), rhi=list(o.rhi[:nd]), wlo=list(o.wlo[:nd]), whi=list(o.whi[:nd]),
                        rlin=(o.rlin_lo, o.rlin_hi), wlin=(o.wlin_lo, o.wlin_hi)))
    return st, out


def _regions(O, arrays):
    out = []
    for a, ext in enumerate(arrays):
        nd = len(ext)
        o = O[a]
        out.append(dict(has_read=bool(o.has_read), has_write=bool(o.has_write),
                        rlo=list(o.rlo[:nd]), rhi=list(o.rhi[:nd]), wlo=list(o.wlo[:nd]), whi=list(o.whi[:nd]),
                        rlin=(o.rlin_lo, o.rlin_hi), wlin=(o.wlin_lo, o.wlin_hi)))
    return out


def region_enumerate_affine(loops, refs, arrays):
    """Affine-bounded nest by enumeration.  loops: [(lo, hi, lo_coef[], hi_coef[])] (step 1)."""
    L = (LoopAffine * max(1, len(loops)))()
    for k, (lo, hi, lc, hc) in enumerate(loops):
        L[k].lo, L[k].hi = lo, hi
        for m, c in enumerate(lc):
            L[k].lo_coef[m] = c
        for m, c in enumerate(hc):
            L[k].hi_coef[m] = c
    _, R, A = make_nest([(0, 0, 1)] * len(loops), refs, arrays)
    O = (Region * max(1, len(arrays)))()
    st = lib().orc_region_enumerate_affine(len(loops), C.cast(L, C.c_void_p), len(refs), C.cast(R, C.c_void_p),
                                           len(arrays), C.cast(A, C.c_void_p), C.cast(O, C.c_void_p))
    return st, _regions(O, arrays)


# ----------------------------------------------------------------------------- threads

def set_threads(n):
    """Threads for the sweeps and large sums (bit-identical results for any count); returns the count set."""
    return int(lib().orc_set_threads(int(n)))


def get_threads():
    return int(lib().orc_get_threads())


class threads:
    """Context manager: run the oracle on n threads (default: every host core), then restore."""

    def __init__(self, n=None):
        self.n = n if n is not None else (os.cpu_count() or 1)

    def __enter__(self):
        self.old = get_threads()
        set_threads(self.n)
        return self

    def __exit__(self, *exc):
        set_threads(self.old)
        return False


# ----------------------------------------------------------------------------- stencils

def jacobi2d_sweep(u):
    u = _c(u, np.float64)
    ny, nx = u.shape
    v = np.empty_like(u)
    r = lib().orc_jacobi2d_sweep(nx, ny, _ptr(u), _ptr(v))
    return v, r


def jacobi2d_run(u, nsweeps):
    """Returns (final field, residuals[nsweeps])."""
    a = _c(u, np.float64).copy()
    b = a.copy()
    ny, nx = a.shape
    res = np.zeros(max(1, nsweeps), dtype=np.float64)
    par = lib().orc_jacobi2d_run(nx, ny, _ptr(a), _ptr(b), nsweeps, _ptr(res))
    return (a if par == 0 else b), res[:nsweeps]


def heat3d_sweep(u, r):
    u = _c(u, np.float64)
    nz, ny, nx = u.shape
    v = np.empty_like(u)
    res = lib().orc_heat3d_sweep(nx, ny, nz, r, _ptr(u), _ptr(v))
    return v, res


def heat3d_run(u, r, nsweeps):
    a = _c(u, np.float64).copy()
    b = a.copy()
    nz, ny, nx = a.shape
    res = np.zeros(max(1, nsweeps), dtype=np.float64)
    par = lib().orc_heat3d_run(nx, ny, nz, r, _ptr(a), _ptr(b), nsweeps, _ptr(res))
    return (a if par == 0 else b), res[:nsweeps]


def box27_sweep(u, w):
    u = _c(u, np.float32)
    w = _c(w, np.float32)
    nz, ny, nx = u.shape
    v = np.empty_like(u)
    lib().orc_box27_sweep(nx, ny, nz, _ptr(w), _ptr(u), _ptr(v))
    return v


def box27_run(u, w, nsweeps, with_sums=True):
    a = _c(u, np.float32).copy()
    b = np.empty_like(a)
    w = _c(w, np.float32)
    nz, ny, nx = a.shape
    sums = np.zeros(max(1, nsweeps), dtype=np.float64)
    par = lib().orc_box27_run(nx, ny, nz, _ptr(w), _ptr(a), _ptr(b), nsweeps,
                              _ptr(sums) if with_sums else None)
    return (a if par == 0 else b), sums[:nsweeps]


def box27_run_f64(u, w, nsweeps):
    a = _c(u, np.float64).copy()
    b = np.empty_like(a)
    w = _c(w, np.float64)
    nz, ny, nx = a.shape
    sums = np.zeros(max(1, nsweeps), dtype=np.float64)
    par = lib().orc_box27_run_f64(nx, ny, nz, _ptr(w), _ptr(a), _ptr(b), nsweeps, _ptr(sums))
    return (a if par == 0 else b), sums[:nsweeps]


def _coeff_ptrs(coeffs, shape):
    """12 coefficient fields (a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 wrk1 bnd) -> kept arrays + pointer table."""
    if len(coeffs) != 12:
        raise ValueError("12 coefficient fields")
    keep = [_c(f, np.float32) for f in coeffs]
    for f in keep:
        if f.shape != shape:
            raise ValueError("coefficient field shape mismatch")
    table = (C.c_void_p * 12)(*[f.ctypes.data for f in keep])
    return keep, table


def var19_sweep(p, coeffs, omega):
    """One variable-coefficient 19-point step (FP32); returns (v, sum of ss^2)."""
    a = _c(p, np.float32)
    v = np.empty_like(a)
    nz, ny, nx = a.shape
    keep, table = _coeff_ptrs(coeffs, a.shape)
    g = lib().orc_var19_sweep(nx, ny, nz, float(omega), table, _ptr(a), _ptr(v))
    return v, g


def var19_run(p, coeffs, omega, nsweeps):
    a = _c(p, np.float32).copy()
    b = np.empty_like(a)
    nz, ny, nx = a.shape
    keep, table = _coeff_ptrs(coeffs, a.shape)
    res = np.zeros(max(1, nsweeps), dtype=np.float64)
    par = lib().orc_var19_run(nx, ny, nz, float(omega), table, _ptr(a), _ptr(b), nsweeps, _ptr(res))
    return (a if par == 0 else b), res[:nsweeps]


# ----------------------------------------------------------------------------- reductions

def maxabs_diff(a, b):
    a = _c(a, np.float64).ravel()
    b = _c(b, np.float64).ravel()
    return lib().orc_maxabs_diff(_ptr(a), _ptr(b), a.size)


def sum_f64(a):
    a = _c(a, np.float64).ravel()
    return lib().orc_sum_f64(_ptr(a), a.size)


def sum_f32(a):
    a = _c(a, np.float32).ravel()
    return lib().orc_sum_f32(_ptr(a), a.size)


# ----------------------------------------------------------------------------- MLP

def mlp_forward(p, x):
    p = _c(p, np.float64)
    x = _c(x, np.float64)
    y = np.empty(x.shape[0], dtype=np.float64)
    lib().orc_mlp_forward(_ptr(p), _ptr(x), x.shape[0], _ptr(y))
    return y


def mlp_loss_grad(p, x, t):
    p = _c(p, np.float64)
    x = _c(x, np.float64)
    t = _c(t, np.float64)
    g = np.empty(NPARAM, dtype=np.float64)
    loss = lib().orc_mlp_loss_grad(_ptr(p), _ptr(x), _ptr(t), x.shape[0], _ptr(g))
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place on p, m, v (float64 arrays)."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    lib().orc_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.size, t, lr, beta1, beta2, eps)


def regret(times, pick):
    times = _c(times, np.float64)
    pick = _c(pick, np.int32)
    nq, nt = times.shape
    out = np.empty(nq, dtype=np.float64)
    lib().orc_regret(_ptr(times), nq, nt, _ptr(pick), _ptr(out))
    return out
