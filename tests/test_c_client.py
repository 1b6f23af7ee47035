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
TIMING_SRC = os.path.join(ROOT, "tests", "c", "region_timing.c")


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


def test_region_analysis_from_c(tmp_path):
    # host-only: the 5-point interior nest of a 256 x 256 grid analysed from
    # plain C, with the hulls of the golden fixture and a time per call
    from paper_2110_14340_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "region_timing")
    subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-Werror", TIMING_SRC, "-o", exe,
                    "-I" + os.path.join(ROOT, "include"), "-L" + libdir, "-ljacc", "-Wl,-rpath," + libdir,
                    "-L/usr/local/cuda/lib64", "-lcudart", "-Wl,-rpath,/usr/local/cuda/lib64"],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe, "256", "20000"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    assert lines[0] == "write [1,254]x[1,254] linear [257,65278]; read [0,255]x[0,255] linear [1,65534]"
    us = float(lines[1].split()[1])
    assert 0.0 < us < 1000.0


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
