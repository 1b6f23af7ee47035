"""The boundary from plain C: tests/c/heat_c_client.c is compiled against
include/jacc.h and linked with libjacc.so and the CUDA runtime (no Python in
the loop); on a GPU its result must match the oracle."""
import os
import subprocess

import numpy as np
import pytest

from paper_2110_14340_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "heat_c_client.c")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    from paper_2110_14340_gb300 import build
    lib = build.build()
    out = str(tmp_path_factory.mktemp("c") / "heat_c_client")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-Werror", SRC, "-o", out,
           "-I" + os.path.join(ROOT, "include"), "-I/usr/local/cuda/include",
           "-L" + libdir, "-ljacc", "-Wl,-rpath," + libdir, "-L/usr/local/cuda/lib64", "-lcudart",
           "-Wl,-rpath,/usr/local/cuda/lib64"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return out


def test_c_client_compiles_and_links(client):
    assert os.access(client, os.X_OK)


@pytest.mark.gpu
def test_c_client_matches_oracle(client, orc, tmp_path):
    n, ns = 40, 6
    u = inputs.heat3d_field(n, seed=2)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    u.astype(np.float64).tofile(fin)
    r = subprocess.run([client, str(n), str(ns), fin, fout], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(fout, dtype=np.float64)
    g, gres = got[: n ** 3].reshape(n, n, n), got[n ** 3:]
    o, ores = orc.heat3d_run(u, 0.125, ns)
    scale = np.max(np.abs(o))
    assert np.max(np.abs(g - o)) <= 1e-12 * scale
    assert np.max(np.abs(gres - ores)) <= 1e-12 * scale
