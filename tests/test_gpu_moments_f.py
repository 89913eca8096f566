"""lbm_moments_f, the FP32 twin of lbm_moments: every field equals the FP64
output rounded to the nearest float, through host and device buffers, for
every storage format and both lattices; host output is staged through the
idle population buffer, so a run that reads moments mid-way must continue
bit for bit like one that does not."""
import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    (dict(lattice=9, nx=48, ny=40, nz=1), (1, 40, 48)),
    (dict(lattice=19, nx=20, ny=16, nz=12, wall=1, T_fixed_lo=1, T_lo=0.85), (12, 16, 20)),
]


def _sim(kw, shape, storage):
    f = W.spinodal(shape, rho0=0.9, T0=0.8, noise=2e-2, seed=51)
    sim = lbm.Lbm(storage=storage, **kw)
    sim.init(f.rho, np.ascontiguousarray(f.u[: sim.d]), 1.5 * f.T)
    return sim


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP64, lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16])
@pytest.mark.parametrize("case", CASES)
def test_fp32_moments_are_the_fp64_moments_rounded(case, storage):
    import torch
    kw, shape = case
    sim = _sim(kw, shape, storage)
    try:
        sim.step(25)
        ref = sim.moments()
        host = {"rho": np.empty(shape, np.float32), "u": np.empty((sim.d,) + shape, np.float32),
                "T": np.empty(shape, np.float32), "P": np.empty(shape, np.float32)}
        lbm.lbm_moments_f(sim.h, host["rho"], host["u"], host["T"], host["P"])
        dev = {k: torch.empty(v.shape, dtype=torch.float32, device="cuda") for k, v in host.items()}
        lbm.lbm_moments_f(sim.h, dev["rho"], dev["u"], dev["T"], dev["P"])
        for k in ("rho", "u", "T", "P"):
            want = ref[k].astype(np.float32)
            assert np.array_equal(host[k], want), k
            assert np.array_equal(dev[k].cpu().numpy(), want), k
        # any subset of the outputs
        T_only = np.empty(shape, np.float32)
        lbm.lbm_moments_f(sim.h, T=T_only)
        assert np.array_equal(T_only, ref["T"].astype(np.float32))
    finally:
        sim.close()


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16])
def test_reading_fp32_moments_mid_run_leaves_the_trajectory_unchanged(storage):
    kw, shape = CASES[1]
    a, b = _sim(kw, shape, storage), _sim(kw, shape, storage)
    try:
        a.step(10)
        T = np.empty(shape, np.float32)
        u = np.empty((3,) + shape, np.float32)
        lbm.lbm_moments_f(a.h, T=T, u=u)
        a.step(10)
        b.step(20)
        ma, mb = a.moments(), b.moments()
        for k in ("rho", "u", "T", "P"):
            assert np.array_equal(ma[k], mb[k]), k
    finally:
        a.close()
        b.close()


def test_fp32_moments_reject_bad_arguments():
    kw, shape = CASES[0]
    sim = lbm.Lbm(**kw)
    try:
        out = np.empty(shape, np.float32)
        with pytest.raises(lbm.LbmError) as e:      # no state yet
            lbm.lbm_moments_f(sim.h, T=out)
        assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        assert lbm.load().lbm_moments_f(sim.h, None, None, None, None, 7) == lbm.LBM_ERR_INVALID_ARG
        with pytest.raises(TypeError):
            lbm.lbm_moments_f(sim.h, T=np.empty(shape))   # float64 is not the FP32 twin's type
    finally:
        sim.close()
