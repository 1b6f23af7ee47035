"""The seeded input generators: host and device variants draw the same numbers."""
import numpy as np
import torch

from paper_2110_14340_gb300 import inputs


def test_torch_generator_matches_numpy():
    for seed, stream in ((1, 0), (4, 7), (6, 0)):
        a = inputs.uniform64(seed, 5000, stream)
        b = inputs.uniform_torch(seed, 5000, "cpu", torch.float64, stream).numpy()
        assert np.array_equal(a, b)
        a = inputs.uniform32(seed, 5000, stream)
        b = inputs.uniform_torch(seed, 5000, "cpu", torch.float32, stream).numpy()
        assert np.array_equal(a, b)


def test_ranges_and_independence():
    u = inputs.uniform64(1, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    assert not np.array_equal(inputs.uniform64(1, 100), inputs.uniform64(2, 100))
    assert not np.array_equal(inputs.uniform64(1, 100, 0), inputs.uniform64(1, 100, 1))
    # chunked generation is position-exact
    assert np.array_equal(inputs.bits(3, 10, 0, 5), inputs.bits(3, 15)[5:])


def test_workload_fields():
    u = inputs.jacobi2d_field(256, 256, seed=1)
    assert u.shape == (256, 256) and np.all(u[0] == 1.0) and np.all(u[:, -1] == 1.0)
    assert 0.0 <= u[1:-1, 1:-1].min() and u[1:-1, 1:-1].max() < 1.0
    h = inputs.heat3d_field(9, seed=2)
    assert h.shape == (9, 9, 9) and np.all(h[0] == 0.0) and np.all(h[:, :, -1] == 0.0)
    b = inputs.box27_field(8, seed=6)
    assert b.dtype == np.float32 and b.min() >= -1.0 and b.max() < 1.0
    shapes = inputs.batched_shapes(64, seed=3)
    assert len(shapes) == 64 and all(128 <= s <= 2048 for sh in shapes for s in sh)
    assert len(set(shapes)) > 50
