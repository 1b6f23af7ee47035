"""Tolerances of the parity tests, derived from the arithmetic.

Fields: normwise, ``max|g - o| / max|o|``, at most 1e-12 for FP64 and 1e-5
for FP32 after the stated sweep count (pointwise relative error is undefined
at zero crossings).

Residuals (``max|u_k - u_(k-1)|`` over the interior, one per sweep) are
differences of two fields of magnitude M = max|u_0|.  One FP64 sweep of the
5- or 7-point update (r <= 1/6) rounds each value by at most 4 eps M
(eps = 2^-53: the neighbour sums carry at most 22 eps M, scaled by r, plus
the final add), and both updates are non-expansive in the max norm, so two
correct evaluations differ by at most 4 k eps M per value after k sweeps and
their k-th residuals by at most 8 k eps M.  The residual tolerance of sweep k
is the larger of that bound and 1e-12 (FP64) or 1e-5 (FP32) of the residual
vector's own scale: a residual of order M is checked to 12 digits, and a
residual far below M to what its definition carries.
"""
import numpy as np

TOL64 = 1e-12
TOL32 = 1e-5
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def nerr(g, o):
    """Normwise relative error max|g - o| / max|o|."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    return float(np.max(np.abs(g - o)) / max(float(np.max(np.abs(o))), 1e-300))


def resid_tol(orr, M, fp64=True):
    """Per-sweep tolerance of residual k = 1..len(orr) (see the module text)."""
    orr = np.asarray(orr, dtype=np.float64)
    tol, eps = (TOL64, EPS64) if fp64 else (TOL32, EPS32)
    k = np.arange(1, orr.size + 1, dtype=np.float64)
    return np.maximum(tol * float(np.max(np.abs(orr))), 8.0 * k * eps * float(M))


def assert_resid(gr, orr, M, fp64=True):
    gr = np.asarray(gr, dtype=np.float64)
    orr = np.asarray(orr, dtype=np.float64)
    assert gr.shape == orr.shape
    err = np.abs(gr - orr)
    tol = resid_tol(orr, M, fp64)
    bad = np.nonzero(~(err <= tol))[0]
    assert bad.size == 0, (f"residual of sweep {bad[0] + 1}: |{gr[bad[0]]!r} - {orr[bad[0]]!r}| = {err[bad[0]]:.3e} "
                           f"> {tol[bad[0]]:.3e}")
