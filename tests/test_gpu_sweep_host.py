"""GPU: jacc_sweep_host, a sweep sequence from and to host buffers in one call.

The result field and residuals equal those of jacc_sweep on device buffers bit
for bit, for page-locked and pageable host memory, and calls on two streams
with two sets of device buffers (the overlapped whole-job path) give each
call's own result.
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


def device_reference(k, u, n):
    a = torch.from_numpy(u).cuda()
    b = torch.empty_like(a)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    fb = jacc.sweep(k, a, b, n, r)
    torch.cuda.synchronize()
    return (b if fb else a).cpu().numpy(), r.cpu().numpy()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n", [1, 2, 7])
def test_sweep_host_matches_device_sweep(orc, pinned, n):
    side = 36
    u = inputs.heat3d_field(side, seed=61)
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    want, wres = device_reference(k, u, n)
    u_host = torch.from_numpy(u.copy())
    out = torch.empty_like(u_host)
    res_host = torch.full((n,), -1.0, dtype=torch.float64)
    if pinned:
        u_host, out, res_host = u_host.pin_memory(), out.pin_memory(), res_host.pin_memory()
    d0 = torch.empty(u.shape, dtype=torch.float64, device="cuda")
    d1 = torch.empty_like(d0)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    fb = jacc.sweep_host(k, u_host, out, d0, d1, n, r, res_host)
    torch.cuda.synchronize()
    assert fb == n % 2
    assert np.array_equal(out.numpy().view(np.int64), want.view(np.int64))
    assert np.array_equal(res_host.numpy(), wres)
    o, orr = orc.heat3d_run(u, 0.125, n)
    assert nerr(out.numpy(), o) <= TOL64
    assert_resid(res_host.numpy(), orr, np.max(np.abs(u)))


def test_two_streams_two_buffer_sets_overlap_correctly():
    side, n = 48, 10
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    hosts = [inputs.heat3d_field(side, seed=70 + i) for i in range(4)]
    want = [device_reference(k, h, n)[0] for h in hosts]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sets = [(torch.empty((side,) * 3, dtype=torch.float64, device="cuda"),
             torch.empty((side,) * 3, dtype=torch.float64, device="cuda"),
             torch.zeros(n, dtype=torch.float64, device="cuda")) for _ in range(2)]
    ins = [torch.from_numpy(h.copy()).pin_memory() for h in hosts]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    torch.cuda.synchronize()
    for i in range(4):  # call i on stream i % 2 with buffer set i % 2
        s = streams[i % 2]
        d0, d1, r = sets[i % 2]
        jacc.sweep_host(k, ins[i], outs[i], d0, d1, n, r, stream=s)
    torch.cuda.synchronize()
    for i in range(4):
        assert np.array_equal(outs[i].numpy().view(np.int64), want[i].view(np.int64)), i


def test_events_keep_the_sweeps_of_consecutive_calls_in_order():
    # the bench's whole-job loop: two streams, two buffer sets, each call's
    # sweeps wait for the previous call's; results as if run one by one
    side, n = 48, 10
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    hosts = [inputs.heat3d_field(side, seed=80 + i) for i in range(5)]
    want = [device_reference(k, h, n) for h in hosts]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    sets = [(torch.empty((side,) * 3, dtype=torch.float64, device="cuda"),
             torch.empty((side,) * 3, dtype=torch.float64, device="cuda"),
             torch.zeros(n, dtype=torch.float64, device="cuda")) for _ in range(2)]
    ins = [torch.from_numpy(h.copy()).pin_memory() for h in hosts]
    outs = [torch.empty_like(t).pin_memory() for t in ins]
    res = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in hosts]
    torch.cuda.synchronize()
    for i in range(5):
        d0, d1, r = sets[i % 2]
        jacc.sweep_host(k, ins[i], outs[i], d0, d1, n, r, res[i], stream=streams[i % 2],
                        wait_event=done[(i + 1) % 2] if i else None, done_event=done[i % 2])
    torch.cuda.synchronize()
    for i in range(5):
        assert np.array_equal(outs[i].numpy().view(np.int64), want[i][0].view(np.int64)), i
        assert np.array_equal(res[i].numpy(), want[i][1]), i


def test_sweep_host_argument_errors():
    side = 16
    k = jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, side, side, side, coeffs=(0.125,))
    u = torch.zeros((side,) * 3, dtype=torch.float64)
    d0 = torch.empty((side,) * 3, dtype=torch.float64, device="cuda")
    d1 = torch.empty_like(d0)
    with pytest.raises(ValueError):
        jacc.sweep_host(k, d0, u, d0, d1, 2)  # the input must be host memory
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep_host(k, u, u.clone(), d0, d1, 2, None, torch.zeros(2, dtype=torch.float64))
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep_host(k, u, u.clone(), d0, d0, 2)  # u0 and u1 overlap
