"""GPU: the region-driven scheduler runs independent sweeps concurrently and
orders dependent work.  Every task's final field is checked against the
oracle run of the same task sequence, and equals sequential execution bit
for bit; completed tasks release their events in long runs."""
import time

import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL64, nerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def grids(n, side, seed):
    return [inputs.heat3d_field(side, seed=seed + g) for g in range(n)]


def test_independent_and_dependent_tasks_match_sequential_execution(orc):
    side, ns, G = 40, 12, 16
    hosts = grids(G, side, 50)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    # sequential reference: every grid swept on the current stream; then grid 1
    # restarts from grid 0's result (a copy) and is swept again
    ref = []
    for h in hosts:
        a = torch.from_numpy(h).cuda()
        b = torch.empty_like(a)
        fb = jacc.sweep(k, a, b, ns)
        ref.append((b if fb else a).clone())
    a1 = ref[0].clone()
    b1 = torch.empty_like(a1)
    fb = jacc.sweep(k, a1, b1, ns)
    chained = (b1 if fb else a1).clone()
    torch.cuda.synchronize()

    s = jacc.Sched(nstreams=8)
    bufs = [(torch.from_numpy(h).cuda(), torch.empty(h.shape, dtype=torch.float64, device="cuda")) for h in hosts]
    torch.cuda.synchronize()
    ids = [s.sweep(k, u0, u1, ns) for u0, u1 in bufs]       # ns even: results land in u0
    assert ns % 2 == 0
    for t in ids:
        assert s.info(t)[0] == []                          # no conflicts between the grids
    assert len({s.info(t)[1] for t in ids}) == 8           # spread over the whole pool
    # (tasks already finished on the device are retired and need no wait, so
    # the recorded dependencies are a subset of the conflicting tasks)
    c = s.copy(bufs[1][0], bufs[0][0], bufs[0][0].numel() * 8)
    assert set(s.info(c)[0]) <= {ids[0], ids[1]}           # reads grid 0's result, overwrites grid 1's
    t = s.sweep(k, bufs[1][0], bufs[1][1], ns)
    assert set(s.info(t)[0]) <= {ids[1], c}
    s.join()
    torch.cuda.synchronize()
    for g, (u0, _) in enumerate(bufs):
        want = chained if g == 1 else ref[g]
        assert torch.equal(u0, want), g
    # the oracle runs the same task sequence: every grid ns sweeps, then grid
    # 1 restarts from grid 0's result and runs ns more
    o = [orc.heat3d_run(h, 0.125, ns)[0] for h in hosts]
    o[1] = orc.heat3d_run(o[0], 0.125, ns)[0]
    for g, (u0, _) in enumerate(bufs):
        assert nerr(u0.cpu().numpy(), o[g]) <= TOL64, g
    s.release()


def test_nest_task_orders_the_callers_own_work(orc):
    side = 32
    h = inputs.heat3d_field(side, seed=7)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    u0 = torch.from_numpy(h).cuda()
    u1 = torch.empty_like(u0)
    torch.cuda.synchronize()
    s = jacc.Sched(nstreams=4)
    n = side ** 3
    # the caller's work: scale the whole field by 0.5 on the task's stream
    t0, st = s.nest_begin([(0, n - 1, 1)], [dict(array=0, coef=[[1]], off=[0], write=True),
                                            dict(array=0, coef=[[1]], off=[0])],
                          [[n]], [u0.data_ptr()], [8])
    with torch.cuda.stream(torch.cuda.ExternalStream(st)):
        u0.mul_(0.5)
    s.nest_end(t0)
    t1 = s.sweep(k, u0, u1, 2)
    assert set(s.info(t1)[0]) <= {t0}
    s.join()
    torch.cuda.synchronize()
    a = torch.from_numpy(h * 0.5).cuda()
    b = torch.empty_like(a)
    jacc.sweep(k, a, b, 2)
    torch.cuda.synchronize()
    assert torch.equal(u0, a)
    o, _ = orc.heat3d_run(h * 0.5, 0.125, 2)
    assert nerr(u0.cpu().numpy(), o) <= TOL64
    s.release()


def test_concurrency_pays_for_small_independent_sweeps(orc):
    # 32 small grids: one stream runs their sweep sequences back to back, the
    # scheduler spreads them over 8 streams
    side, ns, G = 32, 40, 32
    hosts = grids(G, side, 90)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    bufs = [(torch.from_numpy(h).cuda(), torch.empty(h.shape, dtype=torch.float64, device="cuda")) for h in hosts]
    # one scheduled pass from the inputs, against the oracle
    sc = jacc.Sched(nstreams=8)
    for u0, u1 in bufs:
        sc.sweep(k, u0, u1, ns)
    sc.join()
    torch.cuda.synchronize()
    sc.release()
    for (u0, _), h in zip(bufs, hosts):
        o, _ = orc.heat3d_run(h, 0.125, ns)
        assert nerr(u0.cpu().numpy(), o) <= TOL64
    for u0, u1 in bufs:  # warm the graph cache
        jacc.sweep(k, u0, u1, ns)
    torch.cuda.synchronize()

    def seq():
        for u0, u1 in bufs:
            jacc.sweep(k, u0, u1, ns)

    def sched():
        s = jacc.Sched(nstreams=8)
        for u0, u1 in bufs:
            s.sweep(k, u0, u1, ns)
        s.join()
        s.release()

    times = {}
    for name, fn in (("seq", seq), ("sched", sched)):
        fn()
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        times[name] = best
    print("small independent sweeps: sequential %.2f ms, scheduled %.2f ms" % (times["seq"] * 1e3,
                                                                             times["sched"] * 1e3))
    assert times["sched"] < times["seq"]


@pytest.mark.parametrize("nstreams", [1, 4])
def test_completed_tasks_release_their_events(nstreams):
    # thousands of small independent sweeps: once the device has finished
    # them, only each stream's last task keeps its event
    side, ntasks = 16, 3000
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    bufs = [(torch.from_numpy(inputs.heat3d_field(side, seed=200 + g)).cuda(),
             torch.empty((side,) * 3, dtype=torch.float64, device="cuda")) for g in range(8)]
    torch.cuda.synchronize()
    s = jacc.Sched(nstreams=nstreams)
    peak = 0
    for i in range(ntasks):
        u0, u1 = bufs[i % len(bufs)]
        s.sweep(k, u0, u1, 2)
        if i % 500 == 499:
            s.join()
            torch.cuda.synchronize()
            live, n = s.live_events()
            assert n == i + 1
            assert live <= nstreams, (i, live)
            peak = max(peak, live)
    s.join()
    torch.cuda.synchronize()
    live, n = s.live_events()
    assert n == ntasks and live <= nstreams
    # a nest task that is still open keeps its event until it is ended
    t, st = s.nest_begin([(0, 15, 1)], [dict(array=0, coef=[[1]], off=[0], write=True)], [[16]],
                         [bufs[0][0].data_ptr()], [8])
    s.nest_end(t)
    s.join()
    torch.cuda.synchronize()
    s.sweep(k, bufs[1][0], bufs[1][1], 2)
    s.join()
    torch.cuda.synchronize()
    live, _ = s.live_events()
    assert live <= nstreams
    s.release()
