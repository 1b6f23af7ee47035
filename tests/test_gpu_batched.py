"""GPU parity of the batched persistent launch (many uneven 5-point FP64 grids).

Each grid must match its own single-grid oracle run; every schedule (load
path, item size, per-grid tiles, group budget, order, CTAs per SM) gives the
same bits (the fixed-point arithmetic is exact per point, and the native
path evaluates each point the same way); a stalled ticket, or a staged row
that is never fetched, makes the bounded waits time out with
JACC_ERR_TIMEOUT and leaves the context usable.
Widths below one 64-column strip, odd widths (rows that start off a 16-byte
boundary) and fields with an odd number of points (whose last element is
staged through a register) are included.
"""
import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL64, assert_resid, nerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


SHAPES = [(37, 19), (300, 130), (64, 64), (129, 7), (5, 411), (256, 3), (1000, 23), (3, 3), (513, 66)]  # (nx, ny)


def make(shapes, seed=4):
    hosts = inputs.batched_fields(shapes, seed=seed)
    fields = [(torch.from_numpy(h).cuda(), torch.zeros(h.shape, dtype=torch.float64, device="cuda")) for h in hosts]
    return hosts, fields


def results(fields, fb):
    return [(a if fb == 0 else b).cpu().numpy() for a, b in fields]


def reset(fields, hosts):
    for (a, c), h in zip(fields, hosts):
        a.copy_(torch.from_numpy(h))
        c.zero_()


@pytest.mark.parametrize("march", [0, 1])
def test_batched_matches_oracle_per_grid(orc, march):
    hosts, fields = make(SHAPES)
    b = jacc.Batch(fields, item_points=2048, march=march)
    ns = 9
    res = torch.full((len(SHAPES) * ns,), -1.0, dtype=torch.float64, device="cuda")
    fb = b.sweep(ns, res)
    b.status()
    got = results(fields, fb)
    r = res.cpu().numpy().reshape(len(SHAPES), ns)
    for g, h in enumerate(hosts):
        o, orr = orc.jacobi2d_run(h, ns)
        assert nerr(got[g], o) <= TOL64, g
        assert_resid(r[g], orr, np.max(np.abs(h)))


SCHEDULES = [dict(item_points=512, order=1, ctas_per_sm=1), dict(item_points=65536, order=0),
             dict(item_points=4096, order=1, ctas_per_sm=2, march=1), dict(item_points=1024, group_bytes=1),
             dict(item_points=8192, group_bytes=-1, march=1), dict(item_points=2048, group_bytes=200000, order=1)]


@pytest.mark.parametrize("cfg", SCHEDULES)
def test_schedules_give_identical_bits(cfg):
    hosts, fields = make(SHAPES, seed=8)
    b = jacc.Batch(fields)
    res = torch.zeros(len(SHAPES) * 6, dtype=torch.float64, device="cuda")
    fb = b.sweep(6, res, graph=False)
    b.status()
    ref, rref = results(fields, fb), res.cpu().numpy().copy()
    reset(fields, hosts)
    b.configure(**cfg)
    fb = b.sweep(6, res)
    b.status()
    for x, y in zip(results(fields, fb), ref):
        assert np.array_equal(x.view(np.int64), y.view(np.int64))
    assert np.array_equal(res.cpu().numpy(), rref)


def test_per_grid_tiles_report_and_override():
    hosts, fields = make(SHAPES, seed=9)
    b = jacc.Batch(fields, item_points=4096)
    t = b.tiles()
    for (nx, ny), x in zip(SHAPES, t):
        assert x["cols"] in (64, 128, 256, 512) and 1 <= x["rows"] <= ny
        assert x["nitems"] == -(-ny // x["rows"]) * -(-nx // x["cols"])
    fb = b.sweep(5)
    b.status()
    ref = results(fields, fb)
    reset(fields, hosts)
    tiles = [(3, 64), (1, 512), (64, 128), (2, 256), (50, 64), (1, 64), (7, 512), (1, 64), (5, 128)]
    b.set_tiles(tiles)
    got_t = b.tiles()
    for (r, c), (nx, ny), x in zip(tiles, SHAPES, got_t):
        assert x["cols"] == c and x["rows"] == min(r, ny)
    fb = b.sweep(5)
    b.status()
    for x, y in zip(results(fields, fb), ref):
        assert np.array_equal(x.view(np.int64), y.view(np.int64))
    with pytest.raises(jacc.JaccError):
        b.set_tiles([(1, 96)] * len(SHAPES))
    assert b.tiles() == got_t  # a rejected override leaves the plan as it was


def test_native_path_grid_matches_plain_path():
    # a grid holding an infinity runs the native FP64 path for the whole
    # sequence, in the batch as in the single-grid kernels
    shapes = [(70, 40), (33, 21)]
    hosts = inputs.batched_fields(shapes, seed=12)
    hosts[0][10, 11] = np.inf
    fields = [(torch.from_numpy(h).cuda(), torch.zeros(h.shape, dtype=torch.float64, device="cuda")) for h in hosts]
    for march in (0, 1):
        reset(fields, hosts)
        b = jacc.Batch(fields, item_points=1024, march=march)
        res = torch.zeros(2 * 4, dtype=torch.float64, device="cuda")
        fb = b.sweep(4, res)
        b.status()
        got = results(fields, fb)
        r = res.cpu().numpy().reshape(2, 4)
        for g, (nx, ny) in enumerate(shapes):
            k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1)
            a = torch.from_numpy(hosts[g]).cuda()
            c = torch.zeros_like(a)
            rr = torch.zeros(4, dtype=torch.float64, device="cuda")
            f2 = jacc.sweep(k, a, c, 4, rr)
            assert np.array_equal(got[g].view(np.int64), (a if f2 == 0 else c).cpu().numpy().view(np.int64)), g
            assert np.array_equal(r[g].view(np.int64), rr.cpu().numpy().view(np.int64)), g
            k.release()
        b.release()


def test_batched_equals_plain_sweeps_on_the_64_grid_workload(orc):
    # the 64-grid workload (sides log-uniform in [128, 2048]) at a reduced
    # sweep count: batched bits equal the single-grid kernel's, and every grid
    # matches the oracle
    shapes = inputs.batched_shapes(64, seed=3)
    hosts, fields = make(shapes, seed=4)
    ns = 20
    b = jacc.Batch(fields)
    res = torch.zeros(64 * ns, dtype=torch.float64, device="cuda")
    fb = b.sweep(ns, res)
    b.status()
    got = results(fields, fb)
    r = res.cpu().numpy().reshape(64, ns)
    for g in range(64):
        nx, ny = shapes[g]
        k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1, tile_id=0)
        a = torch.from_numpy(hosts[g]).cuda()
        c = torch.zeros_like(a)
        rr = torch.zeros(ns, dtype=torch.float64, device="cuda")
        f2 = jacc.sweep(k, a, c, ns, rr)
        plain = (a if f2 == 0 else c).cpu().numpy()
        assert np.array_equal(got[g], plain), g
        assert np.array_equal(r[g], rr.cpu().numpy()), g
        k.release()
    with orc.threads():
        for g in range(64):
            o, orr = orc.jacobi2d_run(hosts[g], ns)
            assert nerr(got[g], o) <= TOL64, g
            assert_resid(r[g], orr, np.max(np.abs(hosts[g])))


@pytest.mark.parametrize("march", [0, 1])
def test_stalled_ticket_times_out_and_context_survives(march):
    hosts, fields = make(SHAPES[:3], seed=5)
    b = jacc.Batch(fields, item_points=1024, timeout_ms=20, test_stall_ticket=0, march=march)
    b.sweep(4, graph=False)
    with pytest.raises(jacc.JaccError) as e:
        b.status()
    assert e.value.status == jacc.ERR_TIMEOUT
    # the same batch without the stall runs to completion
    b.configure(item_points=1024, timeout_ms=2000, test_stall_ticket=-1, march=march)
    b.sweep(4)
    b.status()
    x = torch.ones(4, device="cuda") * 2
    assert float(x.sum().item()) == 8.0


def test_stalled_row_copy_times_out_and_context_survives(orc):
    # warp 0 of the CTA running the first ticket never fetches its 3rd staged row: its
    # bounded wait for that row's barrier runs out, the launch ends early
    # with JACC_ERR_TIMEOUT, and the next launch is correct
    hosts, fields = make(SHAPES[:3], seed=7)
    b = jacc.Batch(fields, item_points=1024, timeout_ms=20, test_stall_row=3, march=0)
    b.sweep(4, graph=False)
    with pytest.raises(jacc.JaccError) as e:
        b.status()
    assert e.value.status == jacc.ERR_TIMEOUT
    b.configure(item_points=1024, timeout_ms=2000, test_stall_row=0, march=0)
    reset(fields, hosts)
    fb = b.sweep(6)
    b.status()
    got = results(fields, fb)
    for g in range(3):
        o, _ = orc.jacobi2d_run(hosts[g], 6)
        assert nerr(got[g], o) <= TOL64, g


def test_tuner_returns_a_valid_schedule():
    hosts, fields = make(SHAPES, seed=6)
    b = jacc.Batch(fields)
    cfg, ms = b.tune(probe_sweeps=4)
    assert ms > 0 and cfg["item_points"] in (8192, 16384, 32768) and cfg["order"] in (0, 1)
    assert cfg["march"] in (0, 1) and cfg["ctas_per_sm"] >= 1
    assert b.config() == cfg
    # the tuned schedule (with its per-grid tiles) still gives the untuned bits
    reset(fields, hosts)
    fb = b.sweep(5)
    b.status()
    got = results(fields, fb)
    b2 = jacc.Batch(fields)
    reset(fields, hosts)
    fb2 = b2.sweep(5)
    b2.status()
    for x, y in zip(got, results(fields, fb2)):
        assert np.array_equal(x.view(np.int64), y.view(np.int64))
