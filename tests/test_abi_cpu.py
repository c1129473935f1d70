"""The C-ABI library loads and exports every symbol include/asyrk.h declares (CPU only).

No compute call is made here: only argument checks that return before any CUDA
call, and the static status descriptions.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1401_4780_gb300 import asyrk
from paper_1401_4780_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    libbuild.build_library()
    return asyrk.load()


def declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(asyrk_\w+)\s*\(", text, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("asyrk_create", "asyrk_solve", "asyrk_residual", "asyrk_destroy"):
        assert required in names
    assert sorted(asyrk.EXPORTS) == sorted(names)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


_STRUCTS = {"asyrk_create_opts": "CreateOpts", "asyrk_solve_opts": "SolveOpts",
            "asyrk_solve_info": "SolveInfo", "asyrk_problem_stats": "ProblemStats",
            "asyrk_batch_opts": "BatchOpts", "asyrk_lsq_opts": "LsqOpts",
            "asyrk_batch_info": "BatchInfo", "asyrk_tune_result": "TuneResult",
            "asyrk_server_opts": "ServerOpts", "asyrk_server_stats": "ServerStats"}


def test_struct_layouts_match_header(tmp_path):
    # the C compiler's sizeof/offsetof of every option, info and stats struct of
    # the header against the binding's ctypes mirror, field by field
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "asyrk.h"', 'int main(void) {']
    for cname, pname in _STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in getattr(asyrk, pname)._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I" + os.path.join(ROOT, "include"), "-o", str(exe),
                           str(src)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, pname in _STRUCTS.items():
        cls = getattr(asyrk, pname)
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == got[(cname, field)], (cname, field)


def test_abi_version_and_status_strings(lib):
    assert asyrk.asyrk_abi_version() == 1
    assert asyrk.asyrk_strerror(asyrk.EINVAL).startswith("invalid")
    assert asyrk.asyrk_strerror(asyrk.NOT_CONVERGED).startswith("tolerance")
    assert asyrk.asyrk_strerror(12345) == "unknown status"


@pytest.mark.parametrize("m,n", [(0, 4), (4, 0), (-1, 4), (2**31, 4), (4, 2**31)])
def test_create_rejects_bad_sizes_before_touching_the_gpu(lib, m, n):
    rp = np.array([0, 1], dtype=np.int64)
    col = np.zeros(1, dtype=np.int32)
    val = np.ones(1)
    b = np.ones(1)
    st, h = asyrk.asyrk_create(m, n, rp, col, val, asyrk.F64, b)
    assert st == asyrk.EINVAL and not h.value
    assert "m and n" in asyrk.asyrk_last_error()


def test_server_argument_checks_before_touching_the_gpu(lib):
    assert asyrk.asyrk_server_create(0)[0] == asyrk.EINVAL
    assert asyrk.asyrk_server_create(1 << 20, max_slots=-1)[0] == asyrk.EINVAL
    assert asyrk.asyrk_server_submit(None, None)[0] == asyrk.EINVAL
    assert asyrk.asyrk_strerror(asyrk.ECANCELED) == "cancelled"


def test_probe_rejects_bad_arguments_before_touching_the_gpu(lib):
    assert asyrk.asyrk_probe(7, 100, 100)[0] == asyrk.EINVAL
    assert asyrk.asyrk_probe(0, 0, 100)[0] == asyrk.EINVAL
    assert asyrk.asyrk_probe(3, 100, 1000)[0] == asyrk.EINVAL


def test_create_rejects_null_arrays_and_bad_dtype(lib):
    rp = np.array([0, 1], dtype=np.int64)
    col = np.zeros(1, dtype=np.int32)
    val = np.ones(1)
    b = np.ones(1)
    st, _ = asyrk.asyrk_create(1, 1, None, col, val, asyrk.F64, b)
    assert st == asyrk.EINVAL
    st, _ = asyrk.asyrk_create(1, 1, rp, col, val, 7, b)
    assert st == asyrk.EINVAL


def test_solve_rejects_null_handle(lib):
    st, info = asyrk.asyrk_solve(None, np.zeros(1), 1.0, 1e-6, 1)
    assert st == asyrk.EINVAL and info.status == 0


def test_argument_errors_need_no_gpu():
    """Arguments are checked before any CUDA call: these return EINVAL on a host
    without a GPU (and without creating a CUDA context)."""
    rp = np.array([0, 1], dtype=np.int64)
    col = np.array([0], dtype=np.int32)
    val = np.array([1.0])
    b = np.array([1.0])
    for m, n in [(0, 1), (1, 0), (-3, 4), (2**31, 1), (1, 2**31)]:
        st, h = asyrk.asyrk_create(m, n, rp, col, val, asyrk.F64, b)
        assert st == asyrk.EINVAL and not h.value
    st, h = asyrk.asyrk_create(1, 1, rp, col, val, 7, b)  # unknown dtype
    assert st == asyrk.EINVAL and not h.value
    st, h = asyrk.asyrk_create(1, 1, None, col, val, asyrk.F64, b)
    assert st == asyrk.EINVAL and not h.value
    st, h = asyrk.asyrk_lsq_create(1, 1, rp, col, val, asyrk.F64, b, -1.0)
    assert st == asyrk.EINVAL and not h.value
    st, h = asyrk.asyrk_lsq_create(2**30, 2**30, rp, col, val, asyrk.F64, b, 1.0)
    assert st == asyrk.EINVAL and not h.value  # m + n > 2^31 - 1
    st, lo, hi = asyrk.asyrk_spectrum_estimate(1, 1, rp, col, val, asyrk.F64, steps=-1)
    assert st == asyrk.EINVAL
    st, info = asyrk.asyrk_solve(ctypes.c_void_p(), np.zeros(1), 1.0, 1e-6, 10)
    assert st == asyrk.EINVAL
    assert asyrk.asyrk_lsq_solution(ctypes.c_void_p(), np.zeros(1), np.zeros(1)) == asyrk.EINVAL
    assert asyrk.load().asyrk_strerror(asyrk.EINVAL)
