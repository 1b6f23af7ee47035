"""Pins of the oracle's variable-coefficient 19-point step (FP32).

Each term of the definition is isolated by a coefficient choice whose result
the mathematics fixes exactly (small integers stay exact in FP32): a wrong
sign, a swapped direction or a cross term in the wrong plane changes one of
these results.
"""
import numpy as np
import pytest

NZ, NY, NX = 5, 6, 7


def grid():
    z, y, x = np.mgrid[0:NZ, 0:NY, 0:NX]
    return x.astype(np.float32), y.astype(np.float32), z.astype(np.float32)


def coeffs(**kw):
    """a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 wrk1 bnd, zero unless given (bnd defaults to 1)."""
    names = ["a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "wrk1", "bnd"]
    out = []
    for n in names:
        v = kw.get(n, 1.0 if n == "bnd" else 0.0)
        out.append(np.broadcast_to(np.float32(v) if np.isscalar(v) else v.astype(np.float32), (NZ, NY, NX)).copy())
    return out


def interior():
    m = np.zeros((NZ, NY, NX), dtype=bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def expect(p, ss, omega):
    """v = p + omega ss on the interior (two FP32 roundings), p elsewhere."""
    m = interior()
    v = p.copy()
    v[m] = (p[m] + np.float32(omega) * ss[m]).astype(np.float32)
    return v


def test_affine_field_is_a_fixed_point(orc):
    # a = (1, 1, 2), c = (1, 1, 2), a3 = 1/8: s0 a3 is the weighted average of
    # the six faces, exactly p for an affine p with integer coefficients
    x, y, z = grid()
    p = (3 * x - 2 * y + z + 5).astype(np.float32)
    c = coeffs(a0=1, a1=1, a2=2, c0=1, c1=1, c2=2, a3=0.125)
    v, g = orc.var19_sweep(p, c, 1.7)
    assert np.array_equal(v, p) and g == 0.0


@pytest.mark.parametrize("term,field,zero_field", [
    ("b0", lambda x, y, z: x * y, lambda x, y, z: y * z),   # xy plane
    ("b1", lambda x, y, z: y * z, lambda x, y, z: x * z),   # yz plane
    ("b2", lambda x, y, z: x * z, lambda x, y, z: x * y)])  # xz plane
def test_cross_terms_signs_and_planes(orc, term, field, zero_field):
    # for p = u v in the term's plane the four diagonal neighbours combine to
    # exactly 4; for a bilinear field in another plane they cancel to 0
    x, y, z = grid()
    omega = 0.75
    c = coeffs(a3=1.0, **{term: 1.0})
    p = field(x, y, z).astype(np.float32)
    v, g = orc.var19_sweep(p, c, omega)
    ss = (np.float32(4.0) - p).astype(np.float32)
    assert np.array_equal(v, expect(p, ss, omega))
    m = interior()
    assert g == pytest.approx(float(np.sum(ss[m].astype(np.float64) ** 2)), rel=0, abs=0)
    q = zero_field(x, y, z).astype(np.float32)
    v2, _ = orc.var19_sweep(q, c, omega)
    assert np.array_equal(v2, expect(q, (-q).astype(np.float32), omega))


@pytest.mark.parametrize("name,axis,sign", [("a0", 0, 1), ("c0", 0, -1), ("a1", 1, 1), ("c1", 1, -1),
                                            ("a2", 2, 1), ("c2", 2, -1)])
def test_face_coefficients_pick_their_neighbour(orc, name, axis, sign):
    # with p = the coordinate along the axis, the face term reads p +- 1
    x, y, z = grid()
    p = (x, y, z)[axis]
    c = coeffs(a3=1.0, **{name: 1.0})
    v, g = orc.var19_sweep(p, c, 0.5)
    ss = np.full(p.shape, np.float32(sign), dtype=np.float32)
    assert np.array_equal(v, expect(p, ss, 0.5))
    assert g == float(interior().sum())


def test_source_term_and_mask(orc):
    x, y, z = grid()
    p = (x + 2 * y).astype(np.float32)
    w = (z - x).astype(np.float32)
    c = coeffs(a3=1.0, wrk1=w)
    v, _ = orc.var19_sweep(p, c, 1.0)
    assert np.array_equal(v, expect(p, (w - p).astype(np.float32), 1.0))
    # bnd = 0 freezes a point (ss = 0), and only the interior is ever updated
    rng = np.random.default_rng(0)
    bnd = (rng.uniform(size=p.shape) < 0.5).astype(np.float32)
    c2 = coeffs(a3=1.0, wrk1=w, bnd=bnd)
    v2, g2 = orc.var19_sweep(p, c2, 1.0)
    assert np.array_equal(v2[bnd == 0], p[bnd == 0])
    m = interior() & (bnd == 1)
    assert np.array_equal(v2[m], w[m])
    assert g2 == float(np.sum((w[m] - p[m]).astype(np.float64) ** 2))


def test_run_ping_pong_and_residuals(orc):
    rng = np.random.default_rng(1)
    p = rng.uniform(0, 1, (NZ, NY, NX)).astype(np.float32)
    c = coeffs(a0=1, a1=1, a2=2, c0=1, c1=1, c2=2, a3=0.125, b0=0.01, b1=-0.02, b2=0.015)
    a = p
    gs = []
    for _ in range(3):
        a, g = orc.var19_sweep(a, c, 0.8)
        gs.append(g)
    b, res = orc.var19_run(p, c, 0.8, 3)
    assert np.array_equal(a, b) and np.array_equal(res, np.array(gs))
