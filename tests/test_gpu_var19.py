"""GPU parity of the variable-coefficient 19-point stencil (FP32) with the oracle.

The fields must equal the oracle's bit for bit (both evaluate the definition
term by term in IEEE FP32); the residual (sum of ss^2) within 1e-5 of the
oracle's, relative to its value.  Shapes span several 128 x 4 tiles and
64-plane chunks with ragged tails, a z chunk holding only a boundary plane,
and the smallest grid the kernel accepts.
"""
import numpy as np
import pytest
import torch

from paper_2110_14340_gb300 import inputs, jacc

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def run(p, fields, omega, nsweeps, graph=True):
    nz, ny, nx = p.shape
    k = jacc.Kernel(jacc.STENCIL_19PT, jacc.F32, nx, ny, nz, coeffs=(omega,))
    a = torch.from_numpy(np.ascontiguousarray(p)).cuda()
    b = torch.zeros_like(a)
    fs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fields]
    r = torch.full((nsweeps,), -1.0, dtype=torch.float64, device="cuda")
    fb = jacc.sweep_coeffs(k, a, b, nsweeps, fs, r, graph=graph)
    torch.cuda.synchronize()
    return (b if fb else a).cpu().numpy(), r.cpu().numpy(), k


@pytest.mark.parametrize("shape", [(3, 3, 4), (11, 9, 132), (20, 17, 260), (70, 5, 8), (66, 12, 36)])
@pytest.mark.parametrize("graph", [True, False])
def test_var19_matches_oracle(orc, shape, graph):
    nz, ny, nx = shape
    p, fields = inputs.var19_problem(nx, ny, nz, seed=3)
    g, gr, k = run(p, fields, 0.8, 3, graph)
    o, orr = orc.var19_run(p, fields, 0.8, 3)
    # both evaluate the definition term by term in IEEE FP32 (no contraction):
    # the fields agree bit for bit; the residual sums the same ss^2 in another
    # order (FP32 squares, double-float accumulation on the GPU)
    assert np.array_equal(g, o)
    assert np.all(np.abs(gr - orr) <= TOL32 * np.abs(orr))
    assert k.status() == 0


def test_var19_affine_fixed_point_bit_exact():
    nz, ny, nx = 9, 7, 12
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    p = (3 * x - 2 * y + z + 5).astype(np.float32)
    one = np.ones(p.shape, np.float32)
    zero = np.zeros(p.shape, np.float32)
    fields = [one, one, 2 * one, np.full(p.shape, 0.125, np.float32), zero, zero, zero, one, one, 2 * one, zero, one]
    g, gr, _ = run(p, fields, 1.7, 4)
    assert np.array_equal(g, p) and np.all(gr == 0.0)


def test_var19_rejections():
    k = jacc.Kernel(jacc.STENCIL_19PT, jacc.F32, 8, 8, 8, coeffs=(1.0,))
    a = torch.zeros(8, 8, 8, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep(k, a, b, 1)
    fs = [torch.zeros_like(a) for _ in range(12)]
    fs[3] = a  # overlaps u0
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        jacc.sweep_coeffs(k, a, b, 1, fs)
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        jacc.Kernel(jacc.STENCIL_19PT, jacc.F32, 10, 8, 8)
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        jacc.Kernel(jacc.STENCIL_19PT, jacc.F64, 8, 8, 8)
