"""Region analysis beyond rectangular hulls, against brute force (no GPU).

Triangular nests: the library's elimination must equal the oracle's
enumeration of every iteration, bit for bit.  Box unions: every touched
index lies in some box, and when every box is flagged exact the union is
exactly the touched set.
"""
import itertools

import numpy as np
import pytest

from paper_2110_14340_gb300 import jacc


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def random_affine_nest(rng, nloops):
    """Loops whose bounds follow outer indices; inner loops never empty."""
    loops = []
    for k in range(nloops):
        while True:
            lo = int(rng.integers(-3, 4))
            hi = lo + int(rng.integers(0, 5))
            lc = [int(rng.integers(-1, 2)) if m < k else 0 for m in range(k)]
            hc = [int(rng.integers(-1, 2)) if m < k else 0 for m in range(k)]
            # keep hi_k - lo_k >= 0 over the outer ranges: equal slopes
            if any(h != l for h, l in zip(hc, lc)):
                hc = list(lc)
            loops.append((lo, hi, lc, hc))
            break
    return loops


def random_refs(rng, nloops, nd, narr):
    refs = []
    for r in range(int(rng.integers(1, 5))):
        a = int(rng.integers(0, narr))
        refs.append(dict(array=a, write=bool(rng.integers(0, 2)),
                         coef=[[int(rng.integers(-2, 3)) for _ in range(nloops)] for _ in range(nd)],
                         off=[int(rng.integers(-3, 4)) for _ in range(nd)]))
    return refs


def test_triangular_nests_match_enumeration(orc):
    rng = np.random.default_rng(0)
    checked = 0
    for trial in range(300):
        nloops = int(rng.integers(1, 4))
        nd = int(rng.integers(1, 3))
        narr = 2
        loops = random_affine_nest(rng, nloops)
        refs = random_refs(rng, nloops, nd, narr)
        arrays = [[10 ** 6] * nd] * narr  # large: the bounds check never fires
        # shift offsets so subscripts are non-negative
        for r in refs:
            r["off"] = [o + 500 for o in r["off"]]
        st, got = jacc.region_analyze_affine(loops, refs, arrays)
        ost, want = orc.region_enumerate_affine(loops, refs, arrays)
        assert ost == 0
        assert st == 0, (trial, loops)
        assert got == want, (trial, loops, refs)
        checked += 1
    assert checked == 300


def test_triangle_and_empty_cases(orc):
    # j = i .. 9 over i = 0 .. 9 on a 10 x 10 array: the upper triangle
    loops = [(0, 9, [], []), (0, 9, [1], [0])]
    refs = [dict(array=0, write=True, coef=[[1, 0], [0, 1]], off=[0, 0])]
    st, got = jacc.region_analyze_affine(loops, refs, [[10, 10]])
    assert st == 0 and got[0]["wlo"] == [0, 0] and got[0]["whi"] == [9, 9]
    assert got[0]["wlin"] == (0, 99)
    # the anti-diagonal reference i + j over that triangle: 0 + 0 .. 9 + 9
    refs2 = [dict(array=0, coef=[[1, 1]], off=[0])]
    st, got = jacc.region_analyze_affine(loops, refs2, [[19]])
    assert st == 0 and (got[0]["rlo"], got[0]["rhi"]) == ([0], [18])
    # an outer loop that never runs touches nothing
    st, got = jacc.region_analyze_affine([(3, 2, [], []), (0, 1, [0], [0])], refs, [[10, 10]])
    assert st == 0 and not got[0]["has_write"]
    # an inner loop empty for some outer iterations: j = i .. 5 with i up to 9
    # runs the body only for i <= 5; the outer bound is tightened to that
    loops3 = [(0, 9, [], []), (0, 5, [1], [0])]
    st, got = jacc.region_analyze_affine(loops3, refs, [[10, 10]])
    ost, want = orc.region_enumerate_affine(loops3, refs, [[10, 10]])
    assert st == 0 and ost == 0 and got == want and got[0]["whi"] == [5, 5]
    # an inner loop that never runs: nothing is touched
    st, got = jacc.region_analyze_affine([(2, 8, [], []), (9, 0, [0], [1])], refs, [[10, 10]])
    assert st == 0 and not got[0]["has_write"]
    # emptiness that couples two indices (k = i .. j - 1 over j = 0 .. 3):
    # still unsupported
    st, _ = jacc.region_analyze_affine([(0, 3, [], []), (0, 3, [0], [0]), (0, -1, [1, 0], [0, 1])],
                                       [dict(array=0, coef=[[0, 0, 1]], off=[0])], [[10]])
    assert st == jacc.ERR_UNSUPPORTED
    # bounds may only depend on outer loops
    st, _ = jacc.region_analyze_affine([(0, 9, [0, 1], [0, 0])], [], [])
    assert st == jacc.ERR_INVALID_ARG


def touched(loops, refs, arrays):
    """Brute force: set of (array, write, index tuple) over every iteration."""
    ranges = []
    for lo, hi, st in loops:
        ranges.append(list(range(lo, hi + (1 if st > 0 else -1), st)))
    out = set()
    for it in itertools.product(*ranges):
        for r in refs:
            idx = tuple(r["off"][d] + sum(c * i for c, i in zip(r["coef"][d], it)) for d in range(len(r["off"])))
            out.add((r["array"], bool(r.get("write")), idx))
    return out


def box_points(b):
    return {(b["array"], b["write"], idx) for idx in itertools.product(*[range(l, h + 1)
                                                                        for l, h in zip(b["lo"], b["hi"])])}


def test_five_point_read_set_is_a_cross():
    ident = [[1, 0], [0, 1]]
    refs = [dict(array=0, coef=ident, off=o) for o in ([-1, 0], [1, 0], [0, -1], [0, 1], [0, 0])]
    loops = [(1, 6, 1), (1, 6, 1)]
    st, boxes = jacc.region_boxes(loops, refs, [[8, 8]])
    assert st == 0 and all(b["exact"] for b in boxes) and len(boxes) == 5
    union = set().union(*[box_points(b) for b in boxes])
    assert union == touched(loops, refs, [[8, 8]])
    assert (0, False, (0, 0)) not in union  # the hull's corner is not read


def test_box_unions_cover_and_are_exact_when_flagged():
    rng = np.random.default_rng(1)
    for trial in range(200):
        nloops = int(rng.integers(1, 3))
        nd = int(rng.integers(1, 3))
        loops = []
        for _ in range(nloops):
            lo = int(rng.integers(0, 3))
            n = int(rng.integers(1, 4))
            st = int(rng.choice([1, 2, -1]))
            loops.append((lo, lo + (n - 1) * abs(st), st) if st > 0 else (lo + n - 1, lo, st))
        refs = []
        for _ in range(int(rng.integers(1, 5))):
            coef = [[int(rng.choice([0, 1, -1, 2])) for _ in range(nloops)] for _ in range(nd)]
            refs.append(dict(array=0, write=bool(rng.integers(0, 2)), coef=coef,
                             off=[int(rng.integers(8, 12)) for _ in range(nd)]))
        arrays = [[32] * nd]
        st, boxes = jacc.region_boxes(loops, refs, arrays)
        assert st == 0, trial
        t = touched(loops, refs, arrays)
        union = set().union(*[box_points(b) for b in boxes]) if boxes else set()
        assert t <= union, trial
        for kind in (False, True):
            bk = [b for b in boxes if b["write"] == kind]
            if bk and all(b["exact"] for b in bk):
                assert {p for p in union if p[1] == kind} == {p for p in t if p[1] == kind}, trial


def test_widening_and_narrowing_triangles_match_enumeration(orc):
    # inner widths that follow the outer index (j = 0 .. i, k = i .. i + j + 2, ...)
    rng = np.random.default_rng(2)
    shapes = [
        [(0, 6, [], []), (0, 0, [0], [1])],                      # j = 0 .. i
        [(1, 5, [], []), (0, 2, [1], [1])],                      # j = i .. i + 2
        [(0, 4, [], []), (0, 0, [0], [1]), (0, 2, [1, 0], [1, 1])],  # k = i .. i + j + 2
        [(0, 5, [], []), (0, 5, [1], [0])],                      # j = i .. 5 (never empty: i <= 5)
    ]
    for loops in shapes:
        n = len(loops)
        for _ in range(20):
            refs = random_refs(rng, n, 2, 1)
            for r in refs:
                r["off"] = [o + 100 for o in r["off"]]
            st, got = jacc.region_analyze_affine(loops, refs, [[1000, 1000]])
            ost, want = orc.region_enumerate_affine(loops, refs, [[1000, 1000]])
            assert st == 0 and ost == 0 and got == want, (loops, refs)


def test_inner_loops_empty_for_some_outer_iterations_match_enumeration(orc):
    # inner bounds whose extent depends on one outer index with constant
    # bounds (j = i .. c, j = c .. d - i, ...): the outer range is tightened to
    # where the inner loop runs; the result must equal enumeration
    rng = np.random.default_rng(4)
    checked = 0
    for trial in range(300):
        n = int(rng.integers(2, 4))
        loops = [(int(rng.integers(-3, 3)), int(rng.integers(3, 9)), [], [])]
        for k in range(1, n):
            m = int(rng.integers(0, k))  # the one outer index the extent follows
            lc = [0] * k
            hc = [0] * k
            lc[m] = int(rng.integers(-2, 3))
            hc[m] = int(rng.integers(-2, 3))
            for q in range(k):  # other outer indices: same slope on both bounds
                if q != m and rng.integers(0, 2):
                    lc[q] = hc[q] = int(rng.integers(-1, 2))
            lo = int(rng.integers(-4, 5))
            loops.append((lo, lo + int(rng.integers(-3, 6)), lc, hc))
        # the one-index rule needs that index's own bounds constant
        if any(any(loops[m][2]) or any(loops[m][3]) for k in range(1, n) for m in range(k)
               if (loops[k][3][m] - loops[k][2][m]) != 0):
            continue
        refs = random_refs(rng, n, 2, 1)
        for r in refs:
            r["off"] = [o + 200 for o in r["off"]]
        st, got = jacc.region_analyze_affine(loops, refs, [[1000, 1000]])
        ost, want = orc.region_enumerate_affine(loops, refs, [[1000, 1000]])
        assert ost == 0
        if st == jacc.ERR_UNSUPPORTED:
            continue
        assert st == 0, (trial, loops)
        assert got == want, (trial, loops, refs)
        checked += 1
    assert checked >= 100


def touched_affine(loops, refs):
    """Brute force over an affine nest (step 1): set of (array, write, index tuple)."""
    out = set()

    def walk(k, idx):
        if k == len(loops):
            for r in refs:
                t = tuple(r["off"][d] + sum(c * i for c, i in zip(r["coef"][d], idx)) for d in range(len(r["off"])))
                out.add((r["array"], bool(r.get("write")), t))
            return
        lo, hi, lc, hc = loops[k]
        a = lo + sum(c * i for c, i in zip(lc, idx))
        b = hi + sum(c * i for c, i in zip(hc, idx))
        for v in range(a, b + 1):
            walk(k + 1, idx + [v])

    walk(0, [])
    return out


def test_affine_box_unions_cover_and_are_exact_when_flagged():
    rng = np.random.default_rng(5)
    exact_seen = inexact_seen = 0
    for trial in range(200):
        n = int(rng.integers(1, 4))
        loops = random_affine_nest(rng, n)
        nd = int(rng.integers(1, 3))
        refs = []
        for _ in range(int(rng.integers(1, 4))):
            coef = [[int(rng.choice([0, 1, -1, 2])) if rng.integers(0, 2) else 0 for _ in range(n)] for _ in range(nd)]
            refs.append(dict(array=0, write=bool(rng.integers(0, 2)), coef=coef, off=[int(rng.integers(20, 24)) for _ in range(nd)]))
        arrays = [[64] * nd]
        st, boxes = jacc.region_boxes_affine(loops, refs, arrays)
        assert st == 0, trial
        t = touched_affine(loops, refs)
        union = set().union(*[box_points(b) for b in boxes]) if boxes else set()
        assert t <= union, trial
        for kind in (False, True):
            bk = [b for b in boxes if b["write"] == kind]
            if bk and all(b["exact"] for b in bk):
                exact_seen += 1
                assert {p for p in union if p[1] == kind} == {p for p in t if p[1] == kind}, (trial, loops, refs)
            elif bk:
                inexact_seen += 1
    assert exact_seen > 20 and inexact_seen > 20


def test_triangle_box_is_not_exact_but_constant_loops_are():
    tri = [(0, 9, [], []), (0, 0, [0], [1])]            # j = 0 .. i
    st, b = jacc.region_boxes_affine(tri, [dict(array=0, coef=[[1, 0], [0, 1]], off=[0, 0])], [[10, 10]])
    assert st == 0 and len(b) == 1 and not b[0]["exact"] and b[0]["hi"] == [9, 9]
    st, b = jacc.region_boxes_affine(tri, [dict(array=0, coef=[[1, 0]], off=[0])], [[10]])
    assert st == 0 and b[0]["exact"]                     # A[i]: every i occurs
    nest = [(0, 9, [], []), (0, 0, [0], [1]), (0, 3, [0, 0], [0, 0])]   # k = 0 .. 3 inside the triangle
    st, b = jacc.region_boxes_affine(nest, [dict(array=0, coef=[[1, 0, 0], [0, 0, 1]], off=[0, 0])], [[10, 4]])
    assert st == 0 and b[0]["exact"] and b[0]["lo"] == [0, 0] and b[0]["hi"] == [9, 3]
