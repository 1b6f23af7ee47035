"""Host-side checks of the C ABI (CPU only: no kernel is launched).

The library loads without a GPU, exports every function include/jacc.h
declares, and its region analyser (pure host code) matches the oracle
bit-exactly on the same nests the oracle is pinned on.
"""
import os
import random
import re

import pytest

from paper_2110_14340_gb300 import jacc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_14340_gb300 import build
    build.build()
    return jacc.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(jacc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "jacc_region_analyze" in names and "jacc_sweep" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(jacc.SIGNATURES), set(names) - set(jacc.SIGNATURES)


def test_version_and_tiles(lib):
    assert "sm_103a" in jacc.version()
    seen = set()
    for t in range(jacc.NUM_TILES):
        info = jacc.tile_info(t)
        seen.add((info["bx"], info["by"], info["vec16"], info["zc"]))
    assert len(seen) == jacc.NUM_TILES
    with pytest.raises(jacc.JaccError):
        jacc.tile_info(24)


def test_specialize_rejects_bad_descriptors_on_host(lib):
    # validation happens before any CUDA call
    with pytest.raises(jacc.JaccError) as e:
        jacc.Kernel(6, jacc.F64, 10, 10, 10)
    assert e.value.status == jacc.ERR_INVALID_ARG
    with pytest.raises(jacc.JaccError) as e:
        jacc.Kernel(jacc.STENCIL_5PT, jacc.F64, 10, 10, 4)
    assert e.value.status == jacc.ERR_INVALID_ARG
    with pytest.raises(jacc.JaccError) as e:
        jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, 2, 10, 10)
    assert e.value.status == jacc.ERR_INVALID_ARG
    with pytest.raises(jacc.JaccError) as e:
        jacc.Kernel(jacc.STENCIL_7PT, jacc.F64, 11, 10, 10, tile_id=1)  # 16-byte vectors need even nx
    assert e.value.status == jacc.ERR_INVALID_ARG
    with pytest.raises(jacc.JaccError) as e:
        jacc.Kernel(jacc.STENCIL_27PT, jacc.F32, 10, 10, 10, boundary=jacc.DIRICHLET)
    assert e.value.status == jacc.ERR_UNSUPPORTED


def test_region_analysis_matches_oracle_bit_exactly(lib, orc):
    from tests.test_oracle_region import five_point_nest, listing5_nest, random_nest
    cases = [five_point_nest(256), five_point_nest(7), listing5_nest()]
    rng = random.Random(14340)
    cases += [random_nest(rng) for _ in range(2000)]
    # overflow and error cases
    INT64_MAX = (1 << 63) - 1
    cases += [([(0, 4, 1)], [dict(array=0, coef=[[1 << 62]], off=[0])], [[4]]),
              ([(0, 1, 1), (0, 1, 1)], [dict(array=0, coef=[[INT64_MAX, INT64_MAX]], off=[0])], [[4]]),
              ([(0, 0, 1)], [dict(array=0, coef=[[0], [0], [0]], off=[0, 0, 0])], [[2, 1 << 40, 1 << 40]]),
              ([(0, 3, 0)], [dict(array=0, coef=[[1]], off=[0])], [[4]]),
              ([(10, 2, -3)], [dict(array=0, coef=[[1]], off=[0])], [[11]]),
              ([(0, 9, 1), (5, 4, 1)], [dict(array=0, write=True, coef=[[1, 0]], off=[0])], [[10]])]
    for loops, refs, arrays in cases:
        st_o, out_o = orc.region_analyze(loops, refs, arrays)
        st_j, out_j = jacc.region_analyze(loops, refs, arrays)
        assert st_o == st_j, (loops, refs, arrays)
        if st_o in (0, -2):
            assert out_o == out_j, (loops, refs, arrays)


def _table(stencil, dtype, side, ms, valid):
    return dict(stencil=stencil, dtype=dtype, side=side, ms=ms, valid=valid)


def test_costmodel_fixed_tile_and_regret_host_calls(lib):
    # three queries; tile 2 has the lowest times but is invalid in query 1,
    # so the best tile valid everywhere is tile 5 (lowest mean ln time)
    ms = [[10.0] * 24 for _ in range(3)]
    valid = [[1] * 24 for _ in range(3)]
    for q in range(3):
        ms[q][2] = 1.0
        ms[q][5] = 2.0 + q  # mean ln = ln(2*3*4)/3
        ms[q][9] = 3.0      # mean ln = ln 3 > ln(24)/3 = 1.059
    valid[1][2] = 0
    tables = [_table(7, 64, 300.0 + q, ms[q], valid[q]) for q in range(3)]
    assert jacc.fixed_tile(tables) == 5
    r = jacc.regret(tables, [5, 9, 2])
    assert r == [2.0 / 1.0 - 1.0, 3.0 / 3.0 - 1.0, 1.0 / 1.0 - 1.0]  # query 1's best valid tile is 9 (3.0 < 3.0 + 1)
    with pytest.raises(jacc.JaccError):
        jacc.regret(tables, [2, 2, 2])  # tile 2 is not valid for query 1
    with pytest.raises(jacc.JaccError):
        jacc.regret(tables, [24, 0, 0])
    nothing = [_table(5, 32, 100.0, [1.0] * 24, [0] * 24)]
    with pytest.raises(jacc.JaccError) as e:
        jacc.fixed_tile(nothing)
    assert e.value.status == jacc.ERR_UNSUPPORTED


# ctypes structures of the binding and the C types of include/jacc.h they mirror
ABI_STRUCTS = [("Loop", "jacc_loop"), ("Ref", "jacc_ref"), ("Array", "jacc_array"), ("Region", "jacc_region"),
               ("KernelDesc", "jacc_kernel_desc"), ("KernelInfo", "jacc_kernel_info_t"), ("Grid", "jacc_grid"),
               ("BatchConfig", "jacc_batch_config"), ("TuneTable", "jacc_tune_table"),
               ("CostModelEval", "jacc_costmodel_eval"), ("BatchTile", "jacc_batch_tile"),
               ("TuneResult", "jacc_tune_result"), ("LoopAffine", "jacc_loop_affine"), ("Box", "jacc_box"),
               ("Tile", "jacc_tile")]


def test_binding_structs_match_the_header_layout(tmp_path):
    # a C program compiled against include/jacc.h prints the size of every
    # struct the binding mirrors and the offset of each of its fields (a field
    # the header lacks fails the compile); the ctypes layout must agree
    import ctypes
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "jacc.h"', "int main(void) {"]
    for py, c in ABI_STRUCTS:
        cls = getattr(jacc, py)
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi_layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "abi_layout")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", str(src), "-o", exe, "-I" + os.path.join(root, "include")],
                   check=True, capture_output=True, text=True)
    got = {}
    for ln in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines():
        cls, key, val = ln.split()
        got[(cls, key)] = int(val)
    for py, _ in ABI_STRUCTS:
        cls = getattr(jacc, py)
        assert got[(py, "size")] == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert got[(py, name)] == getattr(cls, name).offset, (py, name)


def test_binding_signatures_match_the_header_prototypes():
    # every function include/jacc.h declares has a binding entry with as many
    # arguments as its prototype
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "jacc.h")) as f:
        h = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    decls = re.findall(r"\b(jacc_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", h)
    assert len(decls) >= 50
    for name, args in decls:
        a = args.strip()
        n = 0 if a in ("", "void") else a.count(",") + 1
        assert name in jacc.SIGNATURES, name
        assert len(jacc.SIGNATURES[name][0]) == n, name
