"""Walls on every axis on the GPU against the FP64 oracle (1e-10 after the
steps): x walls, y walls, x and z walls, a box closed on every side, each wall
adiabatic or held at its own temperature; D3Q19 and D2Q9; the fused step
(ragged and tile-exact sizes) and the three-launch step; a batch and slabs
with x walls reproduce the domain run alone bit for bit."""
import numpy as np
import pytest

from gpu_helpers import max_abs, run_gpu, run_oracle
from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("rho", "u", "T", "P")
STEPS = 80

CASES3 = {
    "x": dict(wall_x=1, T_fixed_x=(1, 0), T_x=(0.95, 0.0), gravity=(-1e-5, 0.0, 0.0)),
    "y": dict(wall_y=1, T_fixed_y=(0, 1), T_y=(0.0, 0.9), gravity=(0.0, 1e-5, 0.0)),
    "x+z": dict(wall_x=1, wall=1, T_fixed_lo=1, T_lo=0.95, T_fixed_x=(0, 1), T_x=(0.0, 0.75),
                gravity=(0.0, 0.0, -1e-5)),
    "closed": dict(wall_x=1, wall_y=1, wall=1, T_fixed_lo=1, T_lo=0.95, T_fixed_hi=1, T_hi=0.7,
                   T_fixed_x=(1, 1), T_x=(0.9, 0.85), T_fixed_y=(1, 0), T_y=(0.8, 0.0),
                   gravity=(0.0, 0.0, -1e-5)),
}


@pytest.mark.parametrize("step_kernel", [lbm.LBM_STEP_FUSED, lbm.LBM_STEP_THREE_LAUNCH])
@pytest.mark.parametrize("size", [(45, 37, 22), (64, 48, 20)], ids=["ragged", "tile-exact"])
@pytest.mark.parametrize("case", list(CASES3))
def test_d3q19_walls_fp64_match_oracle(case, size, step_kernel):
    nx, ny, nz = size
    f = W.pool_boiling_3d(nx=nx, ny=ny, nz=nz, T=0.8, depth=nz // 3, noise=1e-3, seed=17)
    kw = dict(lattice=19, nx=nx, ny=ny, nz=nz, **CASES3[case])
    g = run_gpu(f, STEPS, storage=lbm.LBM_STORE_FP64, step_kernel=step_kernel, **kw)
    o = run_oracle(f, STEPS, **kw)
    errs = {k: max_abs(g[k], o[k]) for k in KEYS}
    assert max(errs.values()) <= 1e-10, errs
    assert g["diag"]["bad"] == 0 and g["diag"]["clamps"] == 0


@pytest.mark.parametrize("step_kernel", [lbm.LBM_STEP_FUSED, lbm.LBM_STEP_THREE_LAUNCH])
@pytest.mark.parametrize("walls", ["x", "x+y"])
def test_d2q9_walls_fp64_match_oracle(walls, step_kernel):
    f = W.flat_slab_2d(nx=150, ny=70, T=0.8, slab=50, noise=1e-3)
    kw = dict(lattice=9, nx=150, ny=70, nz=1, wall_x=1, T_fixed_x=(1, 0), T_x=(0.9, 0.0),
              gravity=(1e-5, 0.0, 0.0))
    if walls == "x+y":
        kw.update(wall=1, T_fixed_hi=1, T_hi=0.75)
    g = run_gpu(f, 150, storage=lbm.LBM_STORE_FP64, step_kernel=step_kernel, **kw)
    o = run_oracle(f, 150, **kw)
    errs = {k: max_abs(g[k], o[k]) for k in KEYS}
    assert max(errs.values()) <= 1e-10, errs


def test_fp32_closed_box_within_bounds_and_conserves_mass():
    """FP32 on the closed box: within the FP32 bounds of the other parity
    tests after 300 steps, and walls on every side keep the mass up to the
    FP32 storage rounding, which drifts the total by about 1.5e-8 relative
    per step (measured over 10,000 steps of the pool boiling): 1e-5 after 300
    steps, where a wall that let populations through would lose 1e-3 or
    more."""
    nx, ny, nz = 64, 40, 24
    f = W.pool_boiling_3d(nx=nx, ny=ny, nz=nz, T=0.8, depth=8, noise=1e-4, seed=19)
    kw = dict(lattice=19, nx=nx, ny=ny, nz=nz, **CASES3["closed"])
    g = run_gpu(f, 300, storage=lbm.LBM_STORE_FP32, **kw)
    o = run_oracle(f, 300, **kw)
    errs = {k: max_abs(g[k], o[k]) for k in KEYS}
    tol = {"rho": 2e-4, "T": 5e-5, "u": 5e-6, "P": 2e-5}
    assert all(errs[k] <= tol[k] for k in KEYS), errs
    assert abs(g["diag"]["mass"] / o["state"].N.sum() - 1) < 1e-5


def test_batch_and_slabs_with_x_walls_equal_alone():
    nx, ny, nz = 40, 24, 30
    f = W.pool_boiling_3d(nx=nx, ny=ny, nz=nz, T=0.8, depth=10, noise=1e-3, seed=23)
    kw = dict(nx=nx, ny=ny, nz=nz, **CASES3["x+z"])
    alone = run_gpu(f, 40, lattice=19, storage=lbm.LBM_STORE_FP32, **kw)
    b = lbm.LbmBatch(lattice=19, storage=lbm.LBM_STORE_FP32)
    try:
        i = b.add(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T, 40, **kw)
        b.step(40)
        got = b.moments(i)
    finally:
        b.close()
    for k in KEYS:
        assert np.array_equal(got[k], alone[k]), k
    s = lbm.Slabs(3, lattice=19, storage=lbm.LBM_STORE_FP32, **kw)
    try:
        s.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
        s.step(40)
        got = s.moments()
    finally:
        s.close()
    for k in KEYS:
        assert np.array_equal(got[k], alone[k]), k


def test_d2q9_rejects_a_y_wall_flag():
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(lbm.make_params(lattice=9, nx=16, ny=16, wall_y=1))
