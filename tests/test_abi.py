"""The C ABI library (built here without a GPU) loads, exports every entry
point declared in include/dlr.h, and refuses to run without a usable GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_18705_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    from paper_2601_18705_gb300 import _lib
    hdr = open(os.path.join(ROOT, "include", "dlr.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|size_t|const char \*)\s*\**\s*(dlr_\w+)\s*\(", hdr, re.M))
    assert declared == set(_lib.SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_footprint_without_gpu(lib):
    from paper_2601_18705_gb300 import ProblemSpec  # noqa: F401
    import paper_2601_18705_gb300 as dlr
    import workloads
    spec = dlr.problem_from_case(workloads.lattice32())
    assert dlr.footprint_bytes(spec) > 0


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2601_18705_gb300 as dlr
    from paper_2601_18705_gb300 import _lib
    import workloads
    spec = dlr.problem_from_case(workloads.lattice32())
    p, keep = spec.cstruct()
    h = C.c_void_p()
    rc = lib.dlr_create(C.byref(p), None, C.byref(h))
    assert rc == _lib.DLR_ECUDA and not h.value
    assert lib.dlr_last_error()


def test_invalid_arguments_rejected(lib):
    import paper_2601_18705_gb300 as dlr
    from paper_2601_18705_gb300 import _lib
    import workloads
    spec = dlr.problem_from_case(workloads.lattice32())
    spec.rank = 0
    p, keep = spec.cstruct()
    h = C.c_void_p()
    assert lib.dlr_create(C.byref(p), None, C.byref(h)) == _lib.DLR_EINVAL
    assert b"rank" in lib.dlr_last_error()


def test_oracle_and_product_are_independent():
    """Neither side imports the other; the product package has no path to the
    oracle (only tests, smoke and the benchmark's CPU leg may use it)."""
    pkg = os.path.join(ROOT, "paper_2601_18705_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2601_18705_gb300" not in txt and "dlr.h" not in txt, f


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of the public structs against the C compiler's layout
    import shutil
    import subprocess
    from paper_2601_18705_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"dlr_problem": _lib.DlrProblem, "dlr_stats": _lib.DlrStats,
               "dlr_runtime": _lib.DlrRuntime}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dlr.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"
