"""Oracle parity of the instances the other parity tests do not reach.

* The FP32 D3Q19 step that the benchmark times (32 x 8 tile, 128 producer
  threads, explicit FMAs, approximate FP32 division and square root): 500
  steps of the pool-boiling structure (walls on z, floor held at 0.95, liquid
  layer, gravity) on a 64 x 48 x 32 box and on a ragged box whose sides are
  no multiple of the tile, against the FP64 oracle node by node.
* Every CTA shape of the batched kernel, for D2Q9 and D3Q19, in FP64: each
  job of a batch against the oracle at 1e-10 after its own step budget.
* The serving loop in FP64: each served job against the oracle at 1e-10.

FP32 bounds (max-abs after 500 steps): populations of order w_k carry a unit
roundoff of 6e-8 per operation and take about 10 rounded operations a step,
so a node's density picks up ~3e-7 relative error a step.  Over 500 steps the
errors add as a random walk (x sqrt(500) ~ 22) to ~7e-6 relative; interfaces
amplify it a few times (the liquid density is up to 1.93), giving
|err(rho)| ~ 4e-5.  The temperature is E/(rho c_v), a ratio of two such sums:
~1e-5.  u* is a momentum sum of order 1e-3 over rho: its absolute error is
the population error, ~1e-6.  P = kappa p~ with kappa = 0.01 and
dp~/drho of order 10: ~5e-6.  Bounds: rho 2e-4, T 5e-5, u* 5e-6, P 2e-5.
"""
import numpy as np
import pytest

from gpu_helpers import max_abs, run_gpu, run_oracle
from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import serve
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_TOL = {"rho": 2e-4, "T": 5e-5, "u": 5e-6, "P": 2e-5}
FP64_TOL = 1e-10
KEYS = ("rho", "u", "T", "P")


def _pool(nx, ny, nz, depth, seed=3):
    f = W.pool_boiling_3d(nx=nx, ny=ny, nz=nz, T=0.8, depth=depth, noise=1e-4, seed=seed)
    kw = dict(lattice=19, nx=nx, ny=ny, nz=nz, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5))
    return f, kw


@pytest.mark.parametrize("shape", [(64, 48, 32, 8), (45, 37, 27, 7)], ids=["64x48x32", "ragged45x37x27"])
def test_fp32_d3q19_benchmark_instance_500_steps(shape):
    nx, ny, nz, depth = shape
    f, kw = _pool(nx, ny, nz, depth)
    o = run_oracle(f, 500, **kw)
    g = run_gpu(f, 500, storage=lbm.LBM_STORE_FP32, step_kernel=lbm.LBM_STEP_FUSED, **kw)
    errs = {k: max_abs(g[k], o[k]) for k in KEYS}
    bad = {k: v for k, v in errs.items() if not v <= FP32_TOL[k]}
    assert not bad, errs
    assert g["diag"]["bad"] == 0 and g["diag"]["clamps"] == 0


def _batch_jobs(lattice):
    if lattice == 9:
        return [
            (W.droplet_2d(64, 0.75, 10.0, seed=41), dict(nx=64, ny=64), 40),
            (W.moving_droplet_2d(n=41, ny=37, radius=9.0, hot_offset=15.0, hot_sigma=3.0), dict(nx=41, ny=37), 23),
            (W.flat_slab_2d(nx=70, ny=33, T=0.8, slab=30, noise=1e-3),
             dict(nx=70, ny=33, wall=1, T_fixed_lo=1, T_lo=0.85, gravity=(0.0, -1e-5, 0.0)), 31),
            (W.droplet_2d(96, 0.7, 20.0, seed=44), dict(nx=96, ny=96, chi_mode=1, chi=0.05), 40),
        ]
    return [
        (W.pool_boiling_3d(nx=40, ny=36, nz=24, depth=8, noise=1e-3, seed=3),
         dict(nx=40, ny=36, nz=24, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5)), 30),
        (W.droplet_or_slab_3d(24, 0.8, "droplet", seed=7), dict(nx=24, ny=24, nz=24, chi_mode=1, chi=0.05), 17),
        (W.droplet_or_slab_3d(19, 0.75, "slab", seed=8), dict(nx=19, ny=19, nz=19, chi_mode=1, chi=0.05), 30),
    ]


@pytest.mark.parametrize("lattice", [9, 19])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_fp64_batch_every_shape_matches_oracle(lattice, variant):
    jobs = _batch_jobs(lattice)
    batch = lbm.LbmBatch(lattice=lattice, storage=lbm.LBM_STORE_FP64)
    try:
        batch.set_variant(variant)
        d = 2 if lattice == 9 else 3
        ids = [batch.add(f.rho, np.ascontiguousarray(f.u[:d]), 1.5 * f.T, steps, **kw) for f, kw, steps in jobs]
        batch.step(max(s for _, _, s in jobs))
        for i, (f, kw, steps) in zip(ids, jobs):
            assert batch.status(i) == (steps, 0)
            got = batch.moments(i)
            o = run_oracle(f, steps, lattice=lattice, **kw)
            errs = {k: max_abs(got[k], o[k]) for k in KEYS}
            assert max(errs.values()) <= FP64_TOL, (variant, kw, errs)
    finally:
        batch.close()


def test_fp64_served_jobs_match_oracle():
    trace = W.serving_trace(count=6, rate=400.0, seed=21, side_lo=12, side_hi=28, steps_lo=10, steps_hi=60)
    jobs = serve.trace_jobs(trace)
    srv = serve.Server(lbm.LBM_D3Q19, lbm.LBM_STORE_FP64, quantum=16)
    try:
        st = srv.run(jobs)
    finally:
        srv.close()
    assert st.completed == len(jobs) and st.max_resident >= 2
    for j in jobs:
        rho, u, T = j.fields()
        f = W.Fields(rho, u, T)
        o = run_oracle(f, j.steps, lattice=19, **j.params)
        errs = {k: max_abs(j.result[k], o[k]) for k in KEYS}
        assert max(errs.values()) <= FP64_TOL, (j.name, errs)
