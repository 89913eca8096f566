"""The C-ABI library builds, loads and exports every function include/lbm.h
declares; host-side validation answers without touching a GPU.  CPU only."""
import ctypes
import os
import re

import pytest

from paper_1705_10045_gb300 import build as B
from paper_1705_10045_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_function(libpath):
    declared = _declared()
    assert {"lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_destroy"} <= declared
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lbm.EXPORTED) <= declared


def test_params_struct_matches_header(libpath):
    """lbm_default_params fills the Python mirror of lbm_params consistently."""
    p = lbm.lbm_default_params()
    assert p.lattice == lbm.LBM_D2Q9 and (p.nx, p.ny, p.nz) == (64, 64, 1)
    assert p.kappa == 0.01 and p.A == -0.152 and p.tau == 1.0 and p.c_v == 1.5
    assert p.lambda_ == 0.05 and p.storage == lbm.LBM_STORE_FP32 and p.device == 0
    assert (p.pressure_work, p.conduction, p.pseudoforce) == (1, 1, 1)
    # the ctypes mirror has the size of the C struct (last field ends the struct)
    assert ctypes.sizeof(lbm.lbm_params) == lbm.lbm_params.device.offset + 8


@pytest.mark.parametrize("bad", [
    {"lattice": 7}, {"nx": 0}, {"nz": 2}, {"tau": 0.5}, {"tau_E": 0.4}, {"c_v": 0.0}, {"kappa": -1.0},
    {"storage": 5}, {"lattice": 19, "nz": 1, "wall": 1},
])
def test_create_rejects_invalid_parameters_on_host(libpath, bad):
    p = lbm.make_params(**bad)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG


def test_create_rejects_unstable_conduction(libpath):
    p = lbm.make_params(chi_mode=1, chi=0.3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.code == lbm.LBM_ERR_UNSTABLE_PARAMS


def test_null_handle_calls_fail_cleanly(libpath):
    L = lbm.load()
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_moments_f(None, None, None, None, None, lbm.LBM_MEM_HOST) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_slabs_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_get_planes(None, 0, 1, None, lbm.LBM_MEM_HOST) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_plane_bytes(None) == 0
    L.lbm_slabs_destroy(None)
    assert L.lbm_sync(None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_state_bytes(None) == 0
    L.lbm_destroy(None)
    assert b"null handle" in L.lbm_last_error()


def test_host_coexistence_agrees_with_the_oracle_maxwell_solver(libpath):
    """The library's own coexistence solver (bisection on the pressure until
    the chemical potentials agree) against the oracle's (equal-area
    construction) on the grid of the latent-heat table; they share no code."""
    from oracle import maxwell
    for j in range(0, 512, 5):
        T = 0.5 + j / 1024
        rv, rl = lbm.lbm_coexistence(T)
        ov, ol, _ = maxwell.coexistence(T)
        assert abs(rv - ov) <= 1e-11 * ov and abs(rl - ol) <= 1e-11 * ol, T
    for bad in (0.0, 1.0, 1.2, float("nan")):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_coexistence(bad)
