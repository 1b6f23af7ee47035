"""The oracle on several threads gives the bits it gives on one.

Threads only split the outermost loop of a sweep into slabs (each running
the single-thread loop body) or the top levels of a sum's pairwise
recursion, so every count must reproduce the single-thread result exactly:
fields, residual maxima and sums.  Counts above the outer extent, uneven
slabs and sums whose recursion reaches its 8-element runs above the thread
depth are included.
"""
import numpy as np
import pytest

from paper_2110_14340_gb300 import inputs

COUNTS = [2, 3, 7, 64]


def _bits(a):
    return a.view(np.int64 if a.dtype == np.float64 else np.int32)


def _single_and_threaded(orc, fn):
    with orc.threads(1):
        ref = fn()
    outs = []
    for n in COUNTS:
        with orc.threads(n):
            assert orc.get_threads() == n
            outs.append(fn())
    assert orc.get_threads() == 1
    return ref, outs


def test_jacobi2d_threads_bit_identical(orc):
    u = inputs.jacobi2d_field(37, 29, seed=41)
    ref, outs = _single_and_threaded(orc, lambda: orc.jacobi2d_run(u, 13))
    for g, r in outs:
        assert np.array_equal(_bits(g), _bits(ref[0]))
        assert np.array_equal(_bits(r), _bits(ref[1]))


def test_heat3d_threads_bit_identical(orc):
    u = inputs.heat3d_field(21, ny=18, nz=11, seed=42)
    ref, outs = _single_and_threaded(orc, lambda: orc.heat3d_run(u, 0.125, 9))
    for g, r in outs:
        assert np.array_equal(_bits(g), _bits(ref[0]))
        assert np.array_equal(_bits(r), _bits(ref[1]))


def test_box27_threads_bit_identical(orc):
    w = inputs.box27_weights()
    u = (2.0 * inputs.uniform32(43, 13 * 10 * 17) - 1.0).astype(np.float32).reshape(13, 10, 17)
    ref, outs = _single_and_threaded(orc, lambda: orc.box27_run(u, w, 5))
    for g, s in outs:
        assert np.array_equal(_bits(g), _bits(ref[0]))
        assert np.array_equal(_bits(s), _bits(ref[1]))
    u64 = u.astype(np.float64)
    ref, outs = _single_and_threaded(orc, lambda: orc.box27_run_f64(u64, w.astype(np.float64), 4))
    for g, s in outs:
        assert np.array_equal(_bits(g), _bits(ref[0]))
        assert np.array_equal(_bits(s), _bits(ref[1]))


@pytest.mark.parametrize("n", [1 << 16, (1 << 17) + 3, 1_000_003])
def test_pairwise_sums_threads_bit_identical(orc, n):
    a = (2.0 * inputs.uniform64(44, n) - 1.0) * np.exp(8.0 * inputs.uniform64(45, n))
    f = a.astype(np.float32)
    ref, outs = _single_and_threaded(orc, lambda: (orc.sum_f64(a), orc.sum_f32(f)))
    for s64, s32 in outs:
        assert s64 == ref[0] and s32 == ref[1]


def test_threads_are_clamped(orc):
    with orc.threads(1):
        assert orc.set_threads(0) == 1
        assert orc.set_threads(100000) == 256
