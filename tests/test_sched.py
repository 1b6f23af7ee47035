"""The region-driven scheduler's dependency logic, in dry-run mode (no GPU).

For every byte a task touches, it must wait for the last earlier task that
wrote the byte and, if it writes the byte, for the tasks that read it since
that write - exactly those, checked against a byte-by-byte brute force; every
other earlier conflicting task is ordered before one of them.  Nest tasks
take their ranges from region analysis of their loop nests.
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


class ByteState:
    """Brute force over 16-byte units: last writer and readers since, per unit."""

    def __init__(self):
        self.writer = {}
        self.readers = {}

    def deps(self, reads, writes):
        out = set()
        for lo, hi in reads + writes:
            for u in range(lo // 16, hi // 16):
                if u in self.writer:
                    out.add(self.writer[u])
        for lo, hi in writes:
            for u in range(lo // 16, hi // 16):
                out.update(self.readers.get(u, ()))
        return sorted(out)

    def apply(self, t, reads, writes):
        for lo, hi in reads:
            for u in range(lo // 16, hi // 16):
                self.readers.setdefault(u, set()).add(t)
        for lo, hi in writes:
            for u in range(lo // 16, hi // 16):
                self.writer[u] = t
                self.readers[u] = set()


def test_copy_dependencies_match_brute_force():
    rng = np.random.default_rng(0)
    base = [0x100000 + k * 0x10000 for k in range(5)]
    s = jacc.Sched(nstreams=4, dry_run=True)
    bs = ByteState()
    conflicting = 0
    tasks = []
    for i in range(300):
        a, b = rng.choice(5, 2, replace=False)
        n = int(rng.integers(1, 64)) * 16
        so = int(rng.integers(0, 0x10000 - n) // 16 * 16)
        do = int(rng.integers(0, 0x10000 - n) // 16 * 16)
        src = (base[a] + so, base[a] + so + n)
        dst = (base[b] + do, base[b] + do + n)
        t = s.copy(dst[0], src[0], n)
        assert t == i
        want = bs.deps([src], [dst])
        deps, stream = s.info(t)
        assert deps == want, (i, deps, want)
        assert 0 <= stream < 4
        # every earlier conflicting task is a dependency or ordered before one
        conflicting += sum(1 for ps, pd in tasks if overlaps(dst, pd) or overlaps(dst, ps) or overlaps(src, pd))
        bs.apply(t, [src], [dst])
        tasks.append((src, dst))
    assert conflicting > 300  # the random copies do conflict
    s.release()


def test_dependencies_are_sufficient_transitively():
    # three writers of one range, then a reader: the reader waits for the last
    # writer only, which waited for the one before, and so on
    s = jacc.Sched(nstreams=4, dry_run=True)
    A, B, C = 0x10000, 0x20000, 0x30000
    t0 = s.copy(A, B, 256)      # writes A
    t1 = s.copy(A, C, 256)      # writes A again
    t2 = s.copy(A + 64, B, 64)  # writes part of A
    t3 = s.copy(C, A, 256)      # reads A: last writers of its parts
    assert s.info(t1)[0] == [t0]
    assert s.info(t2)[0] == [t1]
    assert s.info(t3)[0] == [t1, t2]
    t4 = s.copy(A, B, 256)      # writes A: after its last writers and its reader
    assert s.info(t4)[0] == [t1, t2, t3]
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


def test_many_tasks_stay_cheap():
    # 20000 copies among 200 buffers: the interval map keeps a submission at
    # O(log n) plus the segments it overlaps (a scan over all earlier tasks
    # would make this quadratic)
    import time
    rng = np.random.default_rng(3)
    base = [0x1000000 + k * 0x100000 for k in range(200)]
    s = jacc.Sched(nstreams=16, dry_run=True)
    t0 = time.perf_counter()
    for i in range(20000):
        a, b = rng.choice(200, 2, replace=False)
        n = int(rng.integers(1, 256)) * 64
        s.copy(base[b] + int(rng.integers(0, 1024)) * 64, base[a] + int(rng.integers(0, 1024)) * 64, n)
    dt = time.perf_counter() - t0
    deps, _ = s.info(19999)
    assert all(0 <= d < 19999 for d in deps)
    print(f"20000 dry-run submissions: {dt:.2f} s")
    assert dt < 20.0
    s.release()


def test_affine_nest_task_waits_only_for_its_triangle():
    # A[10 + j - i] over the triangle j = 0 .. i, i = 0 .. 9 touches A[1..10];
    # the rectangle i, j = 0 .. 9 would give A[1..19]
    B = 0x5000000
    ref = [dict(array=0, coef=[[-1, 1]], off=[10], write=True)]
    s = jacc.Sched(nstreams=4, dry_run=True)
    t0, _ = s.nest_begin_affine([(0, 9, [], []), (0, 0, [0], [1])], ref, [[32]], [B], [8])
    s.nest_end(t0)
    t1 = s.copy(B + 400, B + 120, 8 * 5)   # reads A[15..19], writes A[50..54]: disjoint from the triangle
    assert s.info(t1)[0] == []
    t2 = s.copy(B + 400, B + 8 * 8, 8 * 4)  # reads A[8..11]: after the triangle's writes of A[8..10]
    assert s.info(t2)[0] == [t0, t1]        # (and after t1, which wrote the same destination)
    s2 = jacc.Sched(nstreams=4, dry_run=True)
    r0, _ = s2.nest_begin([(0, 9, 1), (0, 9, 1)], ref, [[32]], [B], [8])  # the rectangle's hull
    s2.nest_end(r0)
    r1 = s2.copy(B + 400, B + 120, 8 * 5)
    assert s2.info(r1)[0] == [r0]
    s.release()
    s2.release()
