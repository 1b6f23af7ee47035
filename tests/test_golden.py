"""Golden fixtures under tests/golden/: region-analysis values derived by hand
from the paper's definitions and listings (each file cites its passage).  The
oracle and the library must both reproduce them (CPU only)."""
import glob
import os

import pytest

from paper_2110_14340_gb300 import jacc

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = sorted(glob.glob(os.path.join(HERE, "golden", "region_*.txt")))


def parse(path):
    loops, arrays, names, refs, expect = [], [], [], [], []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        w = line.split()
        if w[0] == "loop":
            loops.append((int(w[1]), int(w[2]), int(w[3])))
        elif w[0] == "array":
            names.append(w[1])
            arrays.append([int(x) for x in w[2:]])
        elif w[0] == "ref":
            a = names.index(w[1])
            i_off, i_coef = w.index("off"), w.index("coef")
            off = [int(x) for x in w[i_off + 1:i_coef]]
            rows = " ".join(w[i_coef + 1:]).split("/")
            coef = [[int(x) for x in r.split()] for r in rows]
            refs.append(dict(array=a, write=w[2] == "w", coef=coef, off=off))
        elif w[0] == "expect":
            a = names.index(w[1])
            i_lo, i_hi = w.index("lo"), w.index("hi")
            i_lin = w.index("lin") if "lin" in w else len(w)
            e = dict(array=a, write=w[2] == "w", lo=[int(x) for x in w[i_lo + 1:i_hi]],
                     hi=[int(x) for x in w[i_hi + 1:i_lin]])
            if i_lin < len(w):
                e["lin"] = (int(w[i_lin + 1]), int(w[i_lin + 2]))
            expect.append(e)
    return loops, refs, arrays, expect


def check(out, expect):
    for e in expect:
        o = out[e["array"]]
        k = "w" if e["write"] else "r"
        assert o["has_write" if e["write"] else "has_read"]
        assert o[k + "lo"] == e["lo"] and o[k + "hi"] == e["hi"], (e, o)
        if "lin" in e:
            assert o[k + "lin"] == e["lin"], (e, o)


def test_fixtures_present():
    assert len(FILES) >= 3


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_oracle_reproduces_golden(orc, path):
    loops, refs, arrays, expect = parse(path)
    st, out = orc.region_analyze(loops, refs, arrays)
    assert st == orc.OK
    check(out, expect)


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_library_reproduces_golden(path):
    from paper_2110_14340_gb300 import build
    build.build()
    loops, refs, arrays, expect = parse(path)
    st, out = jacc.region_analyze(loops, refs, arrays)
    assert st == 0
    check(out, expect)
