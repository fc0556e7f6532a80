"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports every
declared entry point, and its host-side problem validation rejects bad input.
No compute call is made (there is no GPU here)."""
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_07607_gb300 import build, mdl
    build.build()
    return mdl.load()


def declared_symbols():
    out = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if not name.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", name)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        out |= set(re.findall(r"\b(mdl_[a-z0-9_]+)\s*\(", txt))
    return out


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "mdl_create" in syms and "mdl_step_to" in syms
    missing = [s for s in sorted(syms) if not hasattr(lib, s)]
    assert not missing, missing


def test_version_string(lib):
    assert b"sm_103a" in lib.mdl_version()


def test_problem_validation_rejects_bad_input_without_device(lib):
    """mdl_create validates before touching the device."""
    import ctypes as C
    from paper_2310_07607_gb300 import mdl
    bad = [W.plain_2d_q1_32x32().replace(dim=4), W.plain_2d_q1_32x32().replace(order=3),
           W.plain_2d_q1_32x32().replace(precision=16), W.plain_2d_q1_32x32().replace(n_lts_levels=0),
           W.plain_2d_q1_32x32().replace(max_refine=9), W.plain_2d_q1_32x32().replace(chi=0.0)]
    for p in bad:
        c = mdl.to_c(p)
        h = C.c_void_p()
        rc = lib.mdl_create(C.byref(c), C.byref(h))
        assert rc == -1, p
        assert lib.mdl_last_error(None)
    assert lib.mdl_step_to(None, 1.0) == -1


def test_struct_layout_matches_header():
    """The ctypes mirror of mdl_problem has the C layout (checked with the host compiler)."""
    import ctypes as C
    import subprocess
    import tempfile
    from paper_2310_07607_gb300 import mdl
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "mdl.h"
int main(){ printf("%zu %zu %zu %zu %zu\n", sizeof(mdl_problem), offsetof(mdl_problem, stim),
  offsetof(mdl_problem, lts_enabled), sizeof(mdl_stats), offsetof(mdl_stats, level_counts)); return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        open(os.path.join(d, "t.c"), "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), os.path.join(d, "t.c"), "-o",
                        os.path.join(d, "t")], check=True)
        out = subprocess.run([os.path.join(d, "t")], capture_output=True, text=True, check=True).stdout.split()
    exp = [C.sizeof(mdl.CProblem), mdl.CProblem.stim.offset, mdl.CProblem.lts_enabled.offset,
           C.sizeof(mdl.CStats), mdl.CStats.level_counts.offset]
    assert [int(x) for x in out] == exp
