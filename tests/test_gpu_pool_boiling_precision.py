"""The pool-boiling workload (D3Q19, 384 x 384 x 256, walls on z, floor held
at T = 0.95, liquid 64 deep at T = 0.8 under its vapour, gravity -1e-5 z,
+-1e-4 noise) run for 10,000 steps with FP32 populations and with FP16
shifted storage, compared with each other.  FP64 is too slow to run at this
size, so neither run has an exact reference; what is checked is that they
tell the same story:

* the horizontal-mean temperature profile T(z) agrees to 1e-2 (the storage
  rounding walk of FP16, ~2e-3 per population over 10,000 steps, amplified
  by the interface dynamics);
* the mass drifts by less than 5e-4 (FP32) and 3e-3 (FP16) relative: walls
  and streaming conserve it, only storage rounding moves it;
* the heated floor raises the total energy by the same amount in both runs
  to within 0.5 % of the initial energy;
* no node turns non-physical and no U >= 0 clamp occurs.

The figures are printed (pytest -s) for the design record."""
import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NX, NY, NZ, STEPS = 384, 384, 256, 10000
KW = dict(lattice=19, nx=NX, ny=NY, nz=NZ, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5))


def _run(storage, f):
    sim = lbm.Lbm(storage=storage, **KW)
    try:
        sim.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
        d0 = sim.diagnostics()
        sim.step(STEPS)
        d1 = sim.diagnostics()
        m = sim.moments()
    finally:
        sim.close()
    Tz = m["T"].reshape(NZ, -1).mean(1)
    rz = m["rho"].reshape(NZ, -1).mean(1)
    return d0, d1, Tz, rz


def test_pool_boiling_fp32_vs_fp16_over_10000_steps():
    f = W.pool_boiling_3d(nx=NX, ny=NY, nz=NZ, T=0.8, depth=64, noise=1e-4, seed=3)
    a0, a1, Ta, ra = _run(lbm.LBM_STORE_FP32, f)
    b0, b1, Tb, rb = _run(lbm.LBM_STORE_FP16, f)
    dT = float(np.max(np.abs(Ta - Tb)))
    mass32 = a1["mass"] / a0["mass"] - 1
    mass16 = b1["mass"] / b0["mass"] - 1
    e32 = a1["energy"] / a0["energy"] - 1
    e16 = b1["energy"] / b0["energy"] - 1
    print(f"\npool boiling {NX}x{NY}x{NZ}, {STEPS} steps: max |T32(z) - T16(z)| = {dT:.3e}; "
          f"max |rho32(z) - rho16(z)| = {float(np.max(np.abs(ra - rb))):.3e}; mass drift FP32 {mass32:.3e}, "
          f"FP16 {mass16:.3e}; energy change FP32 {e32:.4f}, FP16 {e16:.4f}")
    assert dT < 1e-2
    assert abs(mass32) < 5e-4 and abs(mass16) < 3e-3
    assert abs(e32 - e16) < 5e-3 and e32 > 0
    for d in (a1, b1):
        assert d["bad"] == 0 and d["clamps"] == 0
