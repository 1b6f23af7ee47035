"""GPU parity at the full workload sizes, in the launch configuration bench.py times.

- heat 7-point FP64 512^3, 200 sweeps (the bench workload): every point and
  every residual against the oracle run on all host cores;
- batched Jacobi, 64 grids x 500 sweeps: every grid and every residual
  against the oracle, and bit-equal to the plain per-grid path;
- 27-point FP32 1024^3 x 100, plain and temporally blocked: sampled blocks
  of the result against the oracle (a block of side m + 200 around each
  sample, cut from the periodic input, gives the exact central m^3 after 100
  sweeps: values travel one point per sweep), the field sum against W^n S_0
  after every sweep, and a plane wave against its closed-form decay;
- 27-point FP32 512^3 x 100, plain and T = 2: every point and every sweep's
  sum against the oracle.
Tolerances: tests/tolerances.py.
"""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc
from tolerances import TOL32, TOL64, assert_resid, nerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def heat_mode(n):
    s = np.sin(np.pi * np.arange(n) / (n - 1))
    u = s[:, None, None] * s[None, :, None] * s[None, None, :]
    u[0] = u[-1] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    u[:, :, 0] = u[:, :, -1] = 0.0
    return u


def bench_kernel(n=512, r=0.125):
    """The bench's kernel: the library's tile for this shape, constant-folded NVRTC variant."""
    return jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, n, n, n, coeffs=(r,), jit=True)


def test_heat512_200_sweeps_elementwise(orc):
    n, ns = 512, 200
    u = inputs.heat3d_field(n, seed=2)
    k = bench_kernel()
    a = torch.from_numpy(u).cuda()
    b = torch.empty_like(a)
    res = torch.zeros(ns, dtype=torch.float64, device="cuda")
    fb = jacc.sweep(k, a, b, ns, res, graph=True)
    torch.cuda.synchronize()
    g = (a if fb == 0 else b).cpu().numpy()
    gr = res.cpu().numpy()
    del a, b
    with orc.threads():
        o, orr = orc.heat3d_run(u, 0.125, ns)
    e = nerr(g, o)
    print(f"heat 512^3 x 200: normwise error {e:.3e}, residual error {np.max(np.abs(gr - orr)):.3e}")
    assert e <= TOL64
    assert_resid(gr, orr, np.max(np.abs(u)))


def test_heat512_200_sweeps_eigenmode():
    n = 512
    lam = 1.0 - 12.0 * 0.125 * math.sin(math.pi / (2 * (n - 1))) ** 2
    k = bench_kernel()
    # noise-free: u_200 = lambda^200 phi pointwise; residual of sweep j = (1 - lambda) lambda^j max|phi|
    phi = heat_mode(n)
    a = torch.from_numpy(phi).cuda()
    b = torch.empty_like(a)
    res = torch.zeros(200, dtype=torch.float64, device="cuda")
    fb = jacc.sweep(k, a, b, 200, res)
    torch.cuda.synchronize()
    g = (a if fb == 0 else b)
    want = lam ** 200 * torch.from_numpy(phi).cuda()
    assert float((g - want).abs().max()) <= TOL64 * float(np.max(np.abs(phi)))
    j = np.arange(200)
    rclosed = (1.0 - lam) * lam ** j * np.max(np.abs(phi))
    assert_resid(res.cpu().numpy(), rclosed, np.max(np.abs(phi)))


def _batched_oracle(orc, hosts, ns):
    """Every grid's oracle run, grids spread over the host cores (one thread each)."""
    with orc.threads(1), cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(lambda h: orc.jacobi2d_run(h, ns), hosts))


def test_batched_64_grids_500_sweeps(orc):
    shapes = inputs.batched_shapes(64, seed=3)
    hosts = inputs.batched_fields(shapes, seed=4)
    fields = [(torch.from_numpy(h).cuda(), torch.zeros(h.shape, dtype=torch.float64, device="cuda")) for h in hosts]
    bt = jacc.Batch(fields)
    bt.tune(probe_sweeps=20)
    for (a, _), h in zip(fields, hosts):
        a.copy_(torch.from_numpy(h))
    rb = torch.zeros(64 * 500, dtype=torch.float64, device="cuda")
    fb = bt.sweep(500, rb)
    bt.status()
    got = [(a if fb == 0 else b).cpu().numpy() for a, b in fields]
    rbn = rb.cpu().numpy().reshape(64, 500)
    oracle_runs = _batched_oracle(orc, hosts, 500)
    for g, (nx, ny) in enumerate(shapes):
        o, orr = oracle_runs[g]
        assert nerr(got[g], o) <= TOL64, g
        assert_resid(rbn[g], orr, np.max(np.abs(hosts[g])))
        # and bit-equal to the plain per-grid path
        k = jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, nx, ny, 1)
        a = torch.from_numpy(hosts[g]).cuda()
        c = torch.zeros_like(a)
        r = torch.zeros(500, dtype=torch.float64, device="cuda")
        f2 = jacc.sweep(k, a, c, 500, r)
        assert np.array_equal(got[g], (a if f2 == 0 else c).cpu().numpy()), g
        assert np.array_equal(rbn[g], r.cpu().numpy()), g
        k.release()
    bt.release()


def _box27_kernel(n, T, shape=None, jit=False):
    """T = 0: single sweeps (jit: the constant-folded NVRTC variant); T = 2: two per launch."""
    w = inputs.box27_weights()
    nz, ny, nx = shape or (n, n, n)
    return jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, nx, ny, nz, coeffs=tuple(float(x) for x in w), tblock=T,
                       jit=jit)


def _wrap_block(t, corner, m, halo):
    """The periodic block of side m + 2 halo whose centre m^3 starts at `corner` (device or host array)."""
    idx = []
    for ax, c in enumerate(corner):
        n = t.shape[ax]
        i = (np.arange(c - halo, c + m + halo) % n).astype(np.int64)
        idx.append(torch.from_numpy(i).to(t.device) if isinstance(t, torch.Tensor) else i)
    if isinstance(t, torch.Tensor):
        return t.index_select(0, idx[0]).index_select(1, idx[1]).index_select(2, idx[2])
    return t[np.ix_(idx[0], idx[1], idx[2])]


@pytest.mark.parametrize("T,jit", [(0, False), (0, True), (2, False)])
def test_box27_1024_100_sweeps(orc, T, jit):
    n, ns, m = 1024, 100, 8
    w = inputs.box27_weights()
    k = _box27_kernel(n, T, jit=jit)
    a = inputs.uniform_torch(6, n ** 3, "cuda", torch.float32).mul_(2).sub_(1).view(n, n, n)
    corners = [(0, 0, 0), (1020, 3, 1019), (517, 1000, 260), (97, 511, 700)]
    blocks = [_wrap_block(a, c, m, ns).cpu().numpy() for c in corners]
    b = torch.empty_like(a)
    s0 = float(a.double().sum())
    sabs = float(a.abs().double().sum())
    res = torch.zeros(ns, dtype=torch.float64, device="cuda")
    fb = jacc.sweep(k, a, b, ns, res)
    torch.cuda.synchronize()
    g = a if fb == 0 else b
    # sampled blocks against the oracle
    with orc.threads():
        for c, blk in zip(corners, blocks):
            o, _ = orc.box27_run(blk, w, ns, with_sums=False)
            oc = o[ns:ns + m, ns:ns + m, ns:ns + m]
            gc = _wrap_block(g, c, m, 0).cpu().numpy()
            e = nerr(gc, oc)
            print(f"27-point 1024^3 x 100 T={T} jit={jit}: block at {c}: normwise error {e:.3e}")
            assert e <= TOL32, c
    # sums after every sweep (T > 0: after every T-th; the others are NaN)
    W = float(w.astype(np.float64) @ np.array([1, 6, 12, 8], dtype=np.float64))
    r = res.cpu().numpy()
    for i in range(ns):
        if T and (i + 1) % T:
            assert np.isnan(r[i])
        else:
            assert abs(r[i] - W ** (i + 1) * s0) <= 1e-6 * sabs
    assert abs(float(g.double().sum()) - W ** ns * s0) <= 1e-6 * sabs
    # plane wave cos(2 pi (x + 2y + 3z) / n): decays by its symbol per sweep
    x = torch.arange(n, device="cuda", dtype=torch.float64)
    ph = 2 * math.pi * (x[None, None, :] + 2 * x[None, :, None] + 3 * x[:, None, None]) / n
    a.copy_(torch.cos(ph).float())
    cs = [math.cos(2 * math.pi * kk / n) for kk in (1, 2, 3)]
    w64 = w.astype(np.float64)
    sym = (w64[0] + 2 * w64[1] * sum(cs) + 4 * w64[2] * (cs[0] * cs[1] + cs[0] * cs[2] + cs[1] * cs[2])
           + 8 * w64[3] * cs[0] * cs[1] * cs[2])
    fb = jacc.sweep(k, a, b, ns, res)
    torch.cuda.synchronize()
    g = (a if fb == 0 else b).double()
    assert float((g - sym ** ns * torch.cos(ph)).abs().max()) <= TOL32


def test_box27_512_100_sweeps_elementwise_plain_and_blocked(orc):
    n, ns = 512, 100
    w = inputs.box27_weights()
    u = (2.0 * inputs.uniform32(6, n ** 3) - 1.0).astype(np.float32).reshape(n, n, n)
    with orc.threads():
        o, osum = orc.box27_run(u, w, ns)
    A = float(np.sum(np.abs(o.astype(np.float64))))
    for T, jit in ((0, False), (0, True), (2, False)):
        k = _box27_kernel(n, T, jit=jit)
        a = torch.from_numpy(u).cuda()
        b = torch.empty_like(a)
        res = torch.zeros(ns, dtype=torch.float64, device="cuda")
        fb = jacc.sweep(k, a, b, ns, res)
        torch.cuda.synchronize()
        g = (a if fb == 0 else b).cpu().numpy()
        e = nerr(g, o)
        print(f"27-point 512^3 x 100 T={T} jit={jit}: normwise error {e:.3e}")
        assert e <= TOL32
        r = res.cpu().numpy()
        for i in range(ns):
            if T and (i + 1) % T:
                assert np.isnan(r[i])
            else:
                assert abs(r[i] - osum[i]) <= 1e-6 * A, i
        k.release()
