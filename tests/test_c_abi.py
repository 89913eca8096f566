"""include/lbm.h is a C header: a C99 program (tests/c/abi_host.c) compiles
against it with warnings as errors, links liblbm and calls the entry points
that need no GPU; the header also compiles as C++.  The struct sizes it
prints equal the ctypes mirrors of the Python binding, and the coexistence
densities at T = 0.8 equal the Maxwell values of the reduced van der Waals
fluid (Sec. 3).  CPU only."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1705_10045_gb300 import build as B
from paper_1705_10045_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lib = B.build()
    out = tmp_path_factory.mktemp("cabi") / "abi_host"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INC,
                           os.path.join(ROOT, "tests", "c", "abi_host.c"), "-o", str(out),
                           "-L", os.path.dirname(lib), "-llbm", "-Wl,-rpath," + os.path.dirname(lib)])
    text = subprocess.check_output([str(out)], text=True)
    return {line.split()[0]: line.split()[1:] for line in text.splitlines()}


def test_header_compiles_as_cxx(tmp_path):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    src = tmp_path / "h.cc"
    src.write_text('#include "lbm.h"\nint main() { lbm_params p; lbm_default_params(&p); return p.nz - 1; }\n')
    subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", INC, str(src)])


def test_struct_sizes_match_the_python_mirrors(program):
    assert int(program["sizeof_params"][0]) == ctypes.sizeof(lbm.lbm_params)
    assert int(program["sizeof_slab"][0]) == ctypes.sizeof(lbm.lbm_slab)


def test_error_codes_match_the_python_constants(program):
    assert [int(v) for v in program["codes"]] == [lbm.LBM_OK, lbm.LBM_ERR_INVALID_ARG, lbm.LBM_ERR_UNSTABLE_PARAMS,
                                                  lbm.LBM_ERR_OOM, lbm.LBM_ERR_CUDA, lbm.LBM_ERR_NONPHYSICAL,
                                                  lbm.LBM_ERR_TIMEOUT]


def test_host_calls_from_c(program):
    assert program["defaults"] == ["9", "64", "64", "1", "0.01", "-0.152", str(lbm.LBM_STORE_FP32)]
    rc, rv, rl = program["coexistence"]
    assert rc == "0"
    # Maxwell densities of the reduced vdW fluid at T = 0.8
    assert float(rv) == pytest.approx(0.239666921841, abs=1e-9)
    assert float(rl) == pytest.approx(1.93270582860, abs=1e-9)
    assert program["coexistence_bad"] == [str(lbm.LBM_ERR_INVALID_ARG)]
    # 40 planes into 3 slabs: 14, 13, 13; slab 1 owns [14, 27) with two halo
    # planes at both cuts; 40 planes into 21 slabs would own 1 plane, too thin
    assert program["slab"] == ["0", "14", "13", "2", "2", "0", "2", "17", "0"]
    assert program["slab_thin"] == [str(lbm.LBM_ERR_INVALID_ARG), "msg"]
    assert program["create_bad"] == [str(lbm.LBM_ERR_INVALID_ARG), "null"]
    assert program["null_step"] == [str(lbm.LBM_ERR_INVALID_ARG)]
    assert program["null_bytes"] == ["0"]
