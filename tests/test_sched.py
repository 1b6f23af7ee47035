"""The region-driven scheduler's dependency logic, in dry-run mode (no GPU).

A task must wait for exactly the earlier tasks whose byte ranges conflict
with its own (read after write, write after read, write after write on
overlapping bytes) - checked against brute force - and nest tasks take
their ranges from region analysis of their loop nests.
"""
import numpy as np
import pytest

from paper_2110_14340_gb300 import jacc


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def overlaps(a, b):
    return a[0] < b[1] and b[0] < a[1]


def test_copy_dependencies_match_brute_force():
    rng = np.random.default_rng(0)
    base = [0x100000 + k * 0x10000 for k in range(5)]
    s = jacc.Sched(nstreams=4, dry_run=True)
    tasks = []
    for i in range(120):
        a, b = rng.choice(5, 2, replace=False)
        n = int(rng.integers(1, 64)) * 16
        so = int(rng.integers(0, 0x10000 - n) // 16 * 16)
        do = int(rng.integers(0, 0x10000 - n) // 16 * 16)
        src = (base[a] + so, base[a] + so + n)
        dst = (base[b] + do, base[b] + do + n)
        t = s.copy(dst[0], src[0], n)
        assert t == i
        want = [j for j, (ps, pd) in enumerate(tasks)
                if overlaps(dst, pd) or overlaps(dst, ps) or overlaps(src, pd)]
        deps, stream = s.info(t)
        assert deps == want, (i, deps, want)
        assert 0 <= stream < 4
        tasks.append((src, dst))
    s.release()


def test_nest_tasks_take_their_ranges_from_region_analysis():
    # one 128 x 64 FP64 array at B; nests over row ranges
    B = 0x7000000
    arr = [[128, 64]]
    ident = [[1, 0], [0, 1]]

    def rows(lo, hi, write):
        return [(lo, hi, 1), (0, 63, 1)], [dict(array=0, coef=ident, off=[0, 0], write=write)]

    s = jacc.Sched(nstreams=4, dry_run=True)
    t0, _ = s.nest_begin(*rows(0, 63, True), arr, [B], [8])      # writes rows 0..63
    s.nest_end(t0)
    t1, _ = s.nest_begin(*rows(64, 127, False), arr, [B], [8])   # reads rows 64..127
    s.nest_end(t1)
    t2, _ = s.nest_begin(*rows(60, 70, False), arr, [B], [8])    # reads rows 60..70
    s.nest_end(t2)
    t3, _ = s.nest_begin(*rows(100, 110, True), arr, [B], [8])   # writes rows 100..110
    s.nest_end(t3)
    # a 5-point update of rows 1..62 reads rows 0..63 and writes rows 1..62
    five = [dict(array=0, coef=ident, off=o) for o in ([-1, 0], [1, 0], [0, -1], [0, 1])]
    five.append(dict(array=0, coef=ident, off=[0, 0], write=True))
    t4, _ = s.nest_begin([(1, 62, 1), (1, 62, 1)], five, arr, [B], [8])
    s.nest_end(t4)
    assert s.info(t0)[0] == []
    assert s.info(t1)[0] == []            # disjoint rows: runs concurrently with t0
    assert s.info(t2)[0] == [t0]          # overlaps t0's write
    assert s.info(t3)[0] == [t1]          # write after t1's read, disjoint from t0 and t2
    assert s.info(t4)[0] == [t0, t2]      # rewrites rows t0 wrote and t2 read
    # independent tasks spread over the streams; a dependent one continues its chain
    assert s.info(t0)[1] != s.info(t1)[1]
    assert s.info(t2)[1] == s.info(t0)[1]
    s.release()


def test_scheduler_errors():
    s = jacc.Sched(nstreams=2, dry_run=True)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        s.copy(0x1000, 0x1008, 64)        # overlapping copy
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        s.nest_end(0)                     # no such nest task
    # region analysis errors come back unchanged
    with pytest.raises(RuntimeError, match="OUT_OF_BOUNDS"):
        s.nest_begin([(0, 10, 1)], [dict(array=0, coef=[[1]], off=[0])], [[5]], [0x1000], [8])
    s.release()
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.Sched(nstreams=0, dry_run=True)
