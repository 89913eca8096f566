"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

FP64 GPU runs must match the oracle to max-abs 1e-10 on rho, u*, T (and P)
after the stated number of steps.  FP32 and FP16-storage runs are held to
tolerances derived in the module docstring of test_gpu_precision.py.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import max_abs, run_gpu, run_oracle
from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _compare(g, o, tol, keys=("rho", "u", "T", "P")):
    errs = {k: max_abs(g[k], o[k]) for k in keys}
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, errs
    return errs


def test_fp64_flat_slab_128_500_steps():
    """D2Q9 128x128 periodic, vdW T = 0.8, liquid slab 64 wide at the Maxwell
    densities with a tanh interface of width 4, tau = tau_E = 1, c_v = 1.5,
    lambda = 0.05, A = -0.152, u = 0: 500 FP64 steps."""
    f = W.flat_slab_2d(nx=128, ny=128, T=0.8, slab=64)
    kw = dict(lattice=9, nx=128, ny=128, nz=1, storage=lbm.LBM_STORE_FP64)
    g = run_gpu(f, 500, **kw)
    o = run_oracle(f, 500, **kw)
    _compare(g, o, TOL64)
    assert g["diag"]["clamps"] == 0 and g["diag"]["bad"] == 0


def test_fp64_pool_boiling_box_walls_heated_gravity():
    """D3Q19 48x48x32 box with the pool-boiling structure: bounce-back walls on
    z, bottom wall at T = 0.95, adiabatic top, liquid layer 8 deep at T = 0.8,
    gravity -1e-5 z via EDM, +-1e-4 noise: 500 FP64 steps."""
    f = W.pool_boiling_3d(nx=48, ny=48, nz=32, T=0.8, depth=8, noise=1e-4, seed=3)
    kw = dict(lattice=19, nx=48, ny=48, nz=32, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5),
              storage=lbm.LBM_STORE_FP64)
    g = run_gpu(f, 500, **kw)
    o = run_oracle(f, 500, **kw)
    _compare(g, o, TOL64)


@pytest.mark.parametrize("case", [
    # ragged 2-D moving drop with a hot spot
    dict(lattice=9, nx=37, ny=23, nz=1, steps=200,
         fields=lambda: W.moving_droplet_2d(n=37, ny=23, radius=8.0, hot_offset=12.0, hot_sigma=3.0)),
    # ragged 3-D slab, constant chi, tau != tau_E
    dict(lattice=19, nx=13, ny=11, nz=9, steps=200, chi_mode=1, chi=0.05, tau=0.7, tau_E=0.6,
         fields=lambda: _slab3d(13, 11, 9)),
    # 3-D walls with both wall temperatures fixed, pressure work off
    dict(lattice=19, nx=7, ny=5, nz=12, steps=150, wall=1, T_fixed_lo=1, T_lo=0.9, T_fixed_hi=1, T_hi=0.75,
         pressure_work=0, fields=lambda: _slab3d(7, 5, 12)),
    # energy pseudoforce off: the parasitic spreading of Sec. 4 makes this
    # case blow up after about 120 steps (in the oracle too), so it runs 40
    dict(lattice=19, nx=7, ny=5, nz=12, steps=40, wall=1, T_fixed_lo=1, T_lo=0.9, pseudoforce=0,
         fields=lambda: _slab3d(7, 5, 12)),
    # 1-D lattice (ny = 1), barotropic EOS
    dict(lattice=9, nx=64, ny=1, nz=1, steps=300, barotropic=1, T0=0.8,
         fields=lambda: W.flat_slab_2d(nx=64, ny=1, T=0.8, slab=32)),
    # D2Q9 with walls on y and gravity
    dict(lattice=9, nx=16, ny=20, nz=1, steps=200, wall=1, T_fixed_hi=1, T_hi=0.7, gravity=(0.0, -1e-4, 0.0),
         fields=lambda: _slab2d_y(16, 20)),
    # degenerate column: nx = ny = 1 with walls
    dict(lattice=19, nx=1, ny=1, nz=24, steps=100, wall=1, T_fixed_lo=1, T_lo=0.85,
         fields=lambda: _slab3d(1, 1, 24)),
])
def test_fp64_edge_cases(case):
    case = dict(case)
    steps = case.pop("steps")
    f = case.pop("fields")()
    kw = dict(case, storage=lbm.LBM_STORE_FP64)
    g = run_gpu(f, steps, **kw)
    o = run_oracle(f, steps, **kw)
    _compare(g, o, TOL64)


@pytest.mark.parametrize("step_kernel", [lbm.LBM_STEP_FUSED, lbm.LBM_STEP_THREE_LAUNCH])
@pytest.mark.parametrize("case", ["slab2d", "box3d"])
def test_fp64_both_step_forms(step_kernel, case):
    """The fused single-launch step and the three-launch form both match the
    oracle (a ragged, walled, heated 3-D box and a periodic 2-D slab)."""
    if case == "slab2d":
        f = W.flat_slab_2d(nx=70, ny=33, T=0.75, slab=30, noise=1e-3)
        kw = dict(lattice=9, nx=70, ny=33, nz=1)
    else:
        f = W.pool_boiling_3d(nx=21, ny=19, nz=26, T=0.8, depth=9, noise=1e-3, seed=5)
        kw = dict(lattice=19, nx=21, ny=19, nz=26, wall=1, T_fixed_lo=1, T_lo=0.92, T_fixed_hi=1, T_hi=0.78,
                  gravity=(2e-6, -1e-6, -1e-5), tau=0.9, tau_E=0.7)
    g = run_gpu(f, 250, storage=lbm.LBM_STORE_FP64, step_kernel=step_kernel, **kw)
    o = run_oracle(f, 250, **kw)
    _compare(g, o, TOL64)


def _slab3d(nx, ny, nz):
    rv, rl = W.coexistence(0.8)
    z = np.arange(nz, dtype=float)
    s = np.minimum(z - nz / 4 + 0.5, 3 * nz / 4 - 0.5 - z)
    prof = 0.5 * (rl + rv) + 0.5 * (rl - rv) * np.tanh(2 * s / 4.0)
    rho = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).copy()
    rho += W.uniform_noise(rho.shape, 1e-3, 11)
    return W.Fields(rho, np.zeros((3, nz, ny, nx)), np.full((nz, ny, nx), 0.8))


def _slab2d_y(nx, ny):
    rv, rl = W.coexistence(0.8)
    y = np.arange(ny, dtype=float)
    s = 5.5 - y
    prof = 0.5 * (rl + rv) + 0.5 * (rl - rv) * np.tanh(2 * s / 4.0)
    rho = np.broadcast_to(prof[None, :, None], (1, ny, nx)).copy()
    return W.Fields(rho, np.zeros((2, 1, ny, nx)), np.full((1, ny, nx), 0.8))


def test_diagnostics_conservation_fp64():
    """Periodic, no gravity: mass and momentum sums of the GPU state stay at
    their initial values (Eq. (edm) conserves both; the force telescopes)."""
    f = W.moving_droplet_2d(n=96, radius=20.0, hot_offset=40.0)
    sim = lbm.Lbm(lattice=9, nx=96, ny=96, storage=lbm.LBM_STORE_FP64)
    try:
        sim.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
        d0 = sim.diagnostics()
        sim.step(300)
        d1 = sim.diagnostics()
    finally:
        sim.close()
    assert abs(d1["mass"] - d0["mass"]) < 1e-12 * d0["mass"]
    np.testing.assert_allclose(d1["momentum"], d0["momentum"], atol=1e-11 * d0["mass"])
    assert d1["steps"] == 300 and d1["clamps"] == 0 and d1["bad"] == 0
    # the same sums from the oracle's populations of the initial state
    s = oracle.State(oracle.Params(Q=9, nx=96, ny=96), f.rho, f.u, 1.5 * f.T)
    assert abs(s.N.sum() - d0["mass"]) < 1e-10
    assert abs(s.g.sum() - d0["energy"]) < 1e-10


def test_checkpoint_resume_is_bitwise():
    f = W.flat_slab_2d(nx=64, ny=32, T=0.8, slab=32, noise=1e-3)
    for storage in (lbm.LBM_STORE_FP64, lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16):
        a = lbm.Lbm(lattice=9, nx=64, ny=32, storage=storage)
        b = lbm.Lbm(lattice=9, nx=64, ny=32, storage=storage)
        try:
            a.init(f.rho, f.u, 1.5 * f.T)
            a.step(40)
            state = a.get_state()
            a.step(40)
            b.set_state(state)
            b.step(40)
            ma, mb = a.moments(), b.moments()
            for k in ("rho", "u", "T", "P"):
                assert np.array_equal(ma[k], mb[k]), (storage, k)
            assert b.diagnostics()["steps"] == 80
        finally:
            a.close()
            b.close()


def test_device_buffers_match_host_buffers():
    import torch
    f = W.flat_slab_2d(nx=48, ny=40, T=0.85, slab=20, noise=1e-3)
    sims = [lbm.Lbm(lattice=9, nx=48, ny=40, storage=lbm.LBM_STORE_FP64) for _ in range(2)]
    try:
        sims[0].init(f.rho, f.u, 1.5 * f.T)
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.rho, f.u, 1.5 * f.T)]
        sims[1].init(*dev)
        for s in sims:
            s.step(25)
        host = sims[0].moments()
        out = {k: torch.empty(v.shape, dtype=torch.float64, device="cuda") for k, v in host.items()}
        lbm.lbm_moments(sims[1].h, out["rho"], out["u"], out["T"], out["P"])
        for k in host:
            assert np.array_equal(host[k], out[k].cpu().numpy()), k
    finally:
        for s in sims:
            s.close()


def test_init_rejects_nonphysical_and_unstable_fields():
    f = W.flat_slab_2d(nx=16, ny=8, T=0.8, slab=8)
    sim = lbm.Lbm(lattice=9, nx=16, ny=8, storage=lbm.LBM_STORE_FP64)
    try:
        with pytest.raises(lbm.LbmError) as e:
            sim.step(1)
        assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        bad = f.rho.copy()
        bad[0, 3, 4] = -1.0
        with pytest.raises(lbm.LbmError) as e:
            sim.init(bad, f.u, 1.5 * f.T)
        assert e.value.code == lbm.LBM_ERR_NONPHYSICAL
        nan = f.rho.copy()
        nan[0, 0, 0] = np.nan
        with pytest.raises(lbm.LbmError) as e:
            sim.init(nan, f.u, 1.5 * f.T)
        assert e.value.code == lbm.LBM_ERR_NONPHYSICAL
        # a dilute node makes chi = lambda/(rho c_v) exceed 0.5/d
        thin = f.rho.copy()
        thin[0, 2, 2] = 0.01
        with pytest.raises(lbm.LbmError) as e:
            sim.init(thin, f.u, 1.5 * f.T)
        assert e.value.code == lbm.LBM_ERR_UNSTABLE_PARAMS
        sim.init(f.rho, f.u, 1.5 * f.T)
        sim.step(5)
    finally:
        sim.close()
