"""Pins for the oracle's region analysis (CPU only).

The oracle computes exact hulls with a closed form (per-loop endpoint choice);
these tests check it against a different method - enumerating every
iteration - and against hulls derived by hand from the paper's own loops.
"""
import itertools
import random

import numpy as np
import pytest

INT64_MAX = (1 << 63) - 1


def brute_force(loops, refs, arrays):
    """Enumerate every iteration point; per array, per dim, min/max of each subscript."""
    ranges = []
    for lo, hi, st in loops:
        if st > 0:
            ranges.append(list(range(lo, hi + 1, st)))
        else:
            ranges.append(list(range(lo, hi - 1, st)))
    res = [dict(has_read=False, has_write=False, rlo=None, rhi=None, wlo=None, whi=None, rlin=None, wlin=None)
           for _ in arrays]
    pts = list(itertools.product(*ranges)) if loops else [()]
    if any(len(r) == 0 for r in ranges):
        pts = []
    for ref in refs:
        a = ref["array"]
        ext = arrays[a]
        nd = len(ext)
        strides = [1] * nd
        for d in range(nd - 2, -1, -1):
            strides[d] = strides[d + 1] * ext[d + 1]
        w = "w" if ref.get("write") else "r"
        for p in pts:
            e = [ref["off"][d] + sum(ref["coef"][d][k] * p[k] for k in range(len(loops))) for d in range(nd)]
            lin = sum(strides[d] * e[d] for d in range(nd))
            R = res[a]
            if not R["has_write" if w == "w" else "has_read"]:
                R["has_write" if w == "w" else "has_read"] = True
                R[w + "lo"] = list(e)
                R[w + "hi"] = list(e)
                R[w + "lin"] = (lin, lin)
            else:
                R[w + "lo"] = [min(x, y) for x, y in zip(R[w + "lo"], e)]
                R[w + "hi"] = [max(x, y) for x, y in zip(R[w + "hi"], e)]
                R[w + "lin"] = (min(R[w + "lin"][0], lin), max(R[w + "lin"][1], lin))
    inb = True
    for a, ext in enumerate(arrays):
        R = res[a]
        for w in "rw":
            if R["has_write" if w == "w" else "has_read"]:
                if any(l < 0 or h > e - 1 for l, h, e in zip(R[w + "lo"], R[w + "hi"], ext)):
                    inb = False
    return inb, res


def compare(orc_out, bf_out, arrays):
    for a, ext in enumerate(arrays):
        o, b = orc_out[a], bf_out[a]
        assert o["has_read"] == b["has_read"]
        assert o["has_write"] == b["has_write"]
        if b["has_read"]:
            assert o["rlo"] == b["rlo"] and o["rhi"] == b["rhi"] and tuple(o["rlin"]) == tuple(b["rlin"])
        if b["has_write"]:
            assert o["wlo"] == b["wlo"] and o["whi"] == b["whi"] and tuple(o["wlin"]) == tuple(b["wlin"])


def random_nest(rng):
    nl = rng.randint(0, 3)
    loops = []
    for _ in range(nl):
        st = rng.choice([-3, -2, -1, 1, 2, 3])
        lo = rng.randint(-4, 6)
        hi = rng.randint(-4, 6)
        loops.append((lo, hi, st))
    narr = rng.randint(1, 3)
    arrays = [[rng.randint(1, 7) for _ in range(rng.randint(1, 3))] for _ in range(narr)]
    refs = []
    for _ in range(rng.randint(1, 5)):
        a = rng.randrange(narr)
        nd = len(arrays[a])
        refs.append(dict(array=a, write=rng.random() < 0.4,
                         coef=[[rng.randint(-3, 3) for _ in range(nl)] for _ in range(nd)],
                         off=[rng.randint(-3, 8) for _ in range(nd)]))
    return loops, refs, arrays


def test_random_nests_match_enumeration(orc):
    rng = random.Random(2110)
    n_oob = n_ok = 0
    for _ in range(1500):
        loops, refs, arrays = random_nest(rng)
        st, out = orc.region_analyze(loops, refs, arrays)
        inb, bf = brute_force(loops, refs, arrays)
        assert st in (orc.OK, orc.ERR_OUT_OF_BOUNDS)
        assert (st == orc.OK) == inb
        n_ok += st == orc.OK
        n_oob += st != orc.OK
        compare(out, bf, arrays)
    assert n_ok > 100 and n_oob > 100


def five_point_nest(N):
    """The interior loop [1, N-2]^2 of the 5-point Jacobi sweep: four neighbour
    reads and the centre read of u (the centre feeds the residual), one write of v."""
    loops = [(1, N - 2, 1), (1, N - 2, 1)]
    I = [[1, 0], [0, 1]]
    refs = [dict(array=0, coef=I, off=[-1, 0]), dict(array=0, coef=I, off=[1, 0]),
            dict(array=0, coef=I, off=[0, -1]), dict(array=0, coef=I, off=[0, 1]),
            dict(array=0, coef=I, off=[0, 0]), dict(array=1, write=True, coef=I, off=[0, 0])]
    return loops, refs, [[N, N], [N, N]]


def test_five_point_interior_worked_values(orc):
    # Derivation for N = 256: writes v[i][j], i, j in [1, 254]: flattened
    # 256*i + j spans [257, 254*256 + 254 = 65278].  Reads u[i+-1][j], u[i][j+-1]
    # and u[i][j]: per-dimension hull [0, 255]; flattened extremes are
    # u[0][1] -> 1 and u[255][254] -> 65534 (the hull's corners are never read).
    st, out = orc.region_analyze(*five_point_nest(256))
    assert st == orc.OK
    u, v = out
    assert u["has_read"] and not u["has_write"]
    assert u["rlo"] == [0, 0] and u["rhi"] == [255, 255] and u["rlin"] == (1, 65534)
    assert v["has_write"] and not v["has_read"]
    assert v["wlo"] == [1, 1] and v["whi"] == [254, 254] and v["wlin"] == (257, 65278)


def test_listing1_elementwise(orc):
    # Listing 1 (§2.2): for (i = 0; i < N; i++) x[i] = y[i] * y[i];  N = 1000.
    N = 1000
    loops = [(0, N - 1, 1)]
    refs = [dict(array=0, write=True, coef=[[1]], off=[0]), dict(array=1, coef=[[1]], off=[0]),
            dict(array=1, coef=[[1]], off=[0])]
    st, (x, y) = orc.region_analyze(loops, refs, [[N], [N]])
    assert st == orc.OK
    assert x["wlo"] == [0] and x["whi"] == [N - 1] and x["wlin"] == (0, N - 1) and not x["has_read"]
    assert y["rlo"] == [0] and y["rhi"] == [N - 1] and not y["has_write"]


def listing5_nest(gp02=160, gp22=160, jsize=161, ext=(5, 5, 3, 163, 162, 162)):
    """Listing 5 (§4.2, NPB-BT kernel): loops i = 1..gp02, k = 1..gp22, m = 0..4,
    n = 0..4 (loop order i, k, m, n);
        lhsY[n][m][BB][jsize][i][k] = lhsY[n][m][BB][jsize][i][k]
            - sum_{t=0..4} lhsY[n][t][AA][jsize][i][k] * lhsY[t][m][CC][jsize-1][i][k]
    with the t-sum unrolled as in the listing; AA = 0, BB = 1, CC = 2."""
    AA, BB, CC = 0, 1, 2
    loops = [(1, gp02, 1), (1, gp22, 1), (0, 4, 1), (0, 4, 1)]
    # subscript coefficient rows over (i, k, m, n)
    n_ = [0, 0, 0, 1]
    m_ = [0, 0, 1, 0]
    i_ = [1, 0, 0, 0]
    k_ = [0, 1, 0, 0]
    z = [0, 0, 0, 0]
    refs = [dict(array=0, write=True, coef=[n_, m_, z, z, i_, k_], off=[0, 0, BB, jsize, 0, 0]),
            dict(array=0, coef=[n_, m_, z, z, i_, k_], off=[0, 0, BB, jsize, 0, 0])]
    for t in range(5):
        refs.append(dict(array=0, coef=[n_, z, z, z, i_, k_], off=[0, t, AA, jsize, 0, 0]))
        refs.append(dict(array=0, coef=[z, m_, z, z, i_, k_], off=[t, 0, CC, jsize - 1, 0, 0]))
    return loops, refs, [list(ext)]


def test_listing5_multidimensional(orc):
    loops, refs, arrays = listing5_nest()
    st, (a,) = orc.region_analyze(loops, refs, arrays)
    assert st == orc.OK
    # By hand: the write touches [0,4][0,4][BB][jsize][1,160][1,160]; the reads
    # add the AA and CC planes and the jsize-1 slab.
    assert a["wlo"] == [0, 0, 1, 161, 1, 1] and a["whi"] == [4, 4, 1, 161, 160, 160]
    assert a["rlo"] == [0, 0, 0, 160, 1, 1] and a["rhi"] == [4, 4, 2, 161, 160, 160]
    # Flattened offsets against enumeration of every iteration, vectorised.
    ext = arrays[0]
    strides = np.array([int(np.prod(ext[d + 1:])) for d in range(6)], dtype=np.int64)
    i, k, m, n = np.meshgrid(np.arange(1, 161), np.arange(1, 161), np.arange(5), np.arange(5), indexing="ij")
    pts = {"i": i.ravel(), "k": k.ravel(), "m": m.ravel(), "n": n.ravel()}
    lin_r, lin_w = [], []
    for ref in refs:
        e = [ref["off"][d] + ref["coef"][d][0] * pts["i"] + ref["coef"][d][1] * pts["k"]
             + ref["coef"][d][2] * pts["m"] + ref["coef"][d][3] * pts["n"] for d in range(6)]
        lin = sum(strides[d] * e[d] for d in range(6))
        (lin_w if ref.get("write") else lin_r).append((int(lin.min()), int(lin.max())))
    assert a["wlin"] == (min(x[0] for x in lin_w), max(x[1] for x in lin_w))
    assert a["rlin"] == (min(x[0] for x in lin_r), max(x[1] for x in lin_r))


def test_steps_and_last_iterate(orc):
    # i = 10, 7, 4 (stops before 2): hull [4, 10], not [2, 10].
    st, (x,) = orc.region_analyze([(10, 2, -3)], [dict(array=0, coef=[[1]], off=[0])], [[11]])
    assert st == orc.OK and x["rlo"] == [4] and x["rhi"] == [10]
    # i = 0, 4, 8 (hi = 10 is not reached): hull [0, 8].
    st, (x,) = orc.region_analyze([(0, 10, 4)], [dict(array=0, coef=[[1]], off=[0])], [[11]])
    assert st == orc.OK and x["rlo"] == [0] and x["rhi"] == [8]
    # Negative coefficient: x[20 - 2 i], i = 0..9 -> [2, 20].
    st, (x,) = orc.region_analyze([(0, 9, 1)], [dict(array=0, coef=[[-2]], off=[20])], [[21]])
    assert st == orc.OK and x["rlo"] == [2] and x["rhi"] == [20]


def test_empty_nest_touches_nothing(orc):
    st, (x,) = orc.region_analyze([(0, 9, 1), (5, 4, 1)], [dict(array=0, write=True, coef=[[1, 0]], off=[0])],
                                  [[10]])
    assert st == orc.OK and not x["has_read"] and not x["has_write"]


def test_errors(orc):
    ref = [dict(array=0, coef=[[1]], off=[0])]
    assert orc.region_analyze([(0, 3, 0)], ref, [[4]])[0] == orc.ERR_INVALID_ARG
    assert orc.region_analyze([(0, 3, 1)], [dict(array=1, coef=[[1]], off=[0])], [[4]])[0] == orc.ERR_INVALID_ARG
    # ndim mismatch between reference and array
    assert orc.region_analyze([(0, 3, 1)], [dict(array=0, coef=[[1], [0]], off=[0, 0])], [[4]])[0] == \
        orc.ERR_INVALID_ARG
    st, (x,) = orc.region_analyze([(0, 4, 1)], [dict(array=0, coef=[[1]], off=[1])], [[5]])
    assert st == orc.ERR_OUT_OF_BOUNDS and x["rlo"] == [1] and x["rhi"] == [5]
    # coefficient x endpoint outside int64
    assert orc.region_analyze([(0, 4, 1)], [dict(array=0, coef=[[1 << 62]], off=[0])], [[4]])[0] == \
        orc.ERR_OVERFLOW
    # exact sum outside int64 although each term fits
    assert orc.region_analyze([(0, 1, 1), (0, 1, 1)],
                              [dict(array=0, coef=[[INT64_MAX, INT64_MAX]], off=[0])], [[4]])[0] == orc.ERR_OVERFLOW
    # stride overflow: extents whose product exceeds int64
    assert orc.region_analyze([(0, 0, 1)], [dict(array=0, coef=[[0], [0], [0]], off=[0, 0, 0])],
                              [[2, 1 << 40, 1 << 40]])[0] == orc.ERR_OVERFLOW
