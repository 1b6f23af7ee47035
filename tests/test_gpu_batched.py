"""GPU parity of the batched persistent launch (many uneven 5-point FP64 grids).

Each grid must match its own single-grid oracle run; every schedule gives the
same bits (the fixed-point arithmetic is exact per point); a stalled ticket
makes the bounded waits time out with JACC_ERR_TIMEOUT and leaves the
context usable.
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


SHAPES = [(37, 19), (300, 130), (64, 64), (129, 7), (5, 411), (256, 3), (1000, 23)]  # (nx, ny), odd and even nx


def make(shapes, seed=4):
    hosts = inputs.batched_fields(shapes, seed=seed)
    fields = [(torch.from_numpy(h).cuda(), torch.zeros(h.shape, dtype=torch.float64, device="cuda")) for h in hosts]
    return hosts, fields


def results(fields, fb):
    return [(a if fb == 0 else b).cpu().numpy() for a, b in fields]


def test_batched_matches_oracle_per_grid(orc):
    hosts, fields = make(SHAPES)
    b = jacc.Batch(fields, item_points=2048)
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


@pytest.mark.parametrize("cfg", [dict(item_points=512, order=1, ctas_per_sm=1), dict(item_points=65536, order=0),
                                 dict(item_points=4096, order=1, ctas_per_sm=2)])
def test_schedules_give_identical_bits(cfg):
    hosts, fields = make(SHAPES, seed=8)
    b = jacc.Batch(fields)
    fb = b.sweep(6, graph=False)
    b.status()
    ref = results(fields, fb)
    for (a, c), h in zip(fields, hosts):
        a.copy_(torch.from_numpy(h))
    b.configure(**cfg)
    fb = b.sweep(6)
    b.status()
    for x, y in zip(results(fields, fb), ref):
        assert np.array_equal(x, y)


def test_batched_equals_plain_sweeps_on_the_64_grid_workload(orc):
    # the 64-grid workload (sides log-uniform in [128, 2048]) at reduced sweep
    # count: batched bits equal the single-grid kernel's; the smallest grids
    # also against the oracle.
    shapes = inputs.batched_shapes(64, seed=3)
    hosts, fields = make(shapes, seed=4)
    ns = 20
    b = jacc.Batch(fields)
    res = torch.zeros(64 * ns, dtype=torch.float64, device="cuda")
    fb = b.sweep(ns, res)
    b.status()
    got = results(fields, fb)
    r = res.cpu().numpy().reshape(64, ns)
    order = np.argsort([nx * ny for nx, ny in shapes])
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
    for g in order[:3]:
        o, orr = orc.jacobi2d_run(hosts[g], ns)
        assert nerr(got[g], o) <= TOL64
        assert_resid(r[g], orr, np.max(np.abs(hosts[g])))


def test_stalled_ticket_times_out_and_context_survives():
    hosts, fields = make(SHAPES[:3], seed=5)
    b = jacc.Batch(fields, item_points=1024, timeout_ms=20, test_stall_ticket=0)
    b.sweep(4, graph=False)
    with pytest.raises(jacc.JaccError) as e:
        b.status()
    assert e.value.status == jacc.ERR_TIMEOUT
    # the same batch without the stall runs to completion
    b.configure(item_points=1024, timeout_ms=2000, test_stall_ticket=-1)
    b.sweep(4)
    b.status()
    x = torch.ones(4, device="cuda") * 2
    assert float(x.sum().item()) == 8.0


def test_tuner_returns_a_valid_schedule():
    hosts, fields = make(SHAPES, seed=6)
    b = jacc.Batch(fields)
    cfg, ms = b.tune(probe_sweeps=4)
    assert ms > 0 and cfg["item_points"] in (4096, 8192, 16384, 32768, 65536) and cfg["order"] in (0, 1)
    assert b.config() == cfg
