"""The allocation-free conservation sums against lbm_diagnostics.

lbm_conservation_sums_noalloc serves callers that cannot allocate device
memory (device memory owned by another framework's pool, or loops where an
allocation's device-wide synchronisation would stall other work).  It must
give the same sums as the allocating path on the same state, call after call,
while sharing one static scratch array.  This file is collected last so that a
run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEADER = 16   # bytes before the population planes in lbm_get_state


def _device_state(sim):
    import torch
    buf = torch.empty(lbm.lbm_state_bytes(sim.h), dtype=torch.uint8, device="cuda")
    rc = lbm.load().lbm_get_state(sim.h, buf.data_ptr(), lbm.LBM_MEM_DEVICE)
    assert rc == lbm.LBM_OK, lbm.load().lbm_last_error()
    return buf


def _noalloc_sums(sim, state):
    import torch
    p = sim.params
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    lbm.lbm_conservation_sums_noalloc(p.lattice, p.storage, p.nx, p.ny, p.nz, p.rho_ref, p.E_ref,
                                      state.data_ptr() + HEADER, out.data_ptr(), 0)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("lattice,storage", [(9, lbm.LBM_STORE_FP64), (19, lbm.LBM_STORE_FP32),
                                             (19, lbm.LBM_STORE_FP16)])
def test_noalloc_sums_match_diagnostics_on_two_calls(lattice, storage):
    if lattice == 9:
        f = W.flat_slab_2d(nx=96, ny=40, T=0.8, slab=40, noise=1e-3)
        kw = dict(lattice=9, nx=96, ny=40, nz=1)
    else:
        f = W.pool_boiling_3d(nx=40, ny=36, nz=24, T=0.8, depth=8, noise=1e-3, seed=3)
        kw = dict(lattice=19, nx=40, ny=36, nz=24, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5))
    sim = lbm.Lbm(storage=storage, **kw)
    try:
        sim.init(f.rho, f.u, 1.5 * f.T)
        for steps in (7, 13):   # two calls in a row on two different states
            sim.step(steps)
            d = lbm.lbm_diagnostics(sim.h)
            got = _noalloc_sums(sim, _device_state(sim))
            want = d[:5]
            scale = abs(want[0])
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)
    finally:
        sim.close()


def test_noalloc_two_ordered_calls_on_one_stream():
    """Two states summed by two calls queued back to back on one non-default
    stream, with a single synchronisation at the end: the calls share the
    scratch array, and stream order alone keeps them apart."""
    import torch
    sims, states = [], []
    try:
        for seed, steps in ((3, 5), (4, 11)):
            f = W.pool_boiling_3d(nx=64, ny=40, nz=24, T=0.8, depth=8, noise=1e-3, seed=seed)
            sim = lbm.Lbm(lattice=19, nx=64, ny=40, nz=24, wall=1, T_fixed_lo=1, T_lo=0.95,
                          storage=lbm.LBM_STORE_FP32)
            sim.init(f.rho, f.u, 1.5 * f.T)
            sim.step(steps)
            sims.append(sim)
            states.append(_device_state(sim))
        torch.cuda.synchronize()
        stream = torch.cuda.Stream()
        outs = [torch.full((5,), float("nan"), dtype=torch.float64, device="cuda") for _ in sims]
        for sim, st, out in zip(sims, states, outs):
            p = sim.params
            lbm.lbm_conservation_sums_noalloc(p.lattice, p.storage, p.nx, p.ny, p.nz, p.rho_ref, p.E_ref,
                                              st.data_ptr() + HEADER, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        for sim, out in zip(sims, outs):
            want = lbm.lbm_diagnostics(sim.h)[:5]
            np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=1e-12 * abs(want[0]))
    finally:
        for sim in sims:
            sim.close()


def test_noalloc_rejects_bad_sizes_and_pointers():
    import torch
    L = lbm.load()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    pop = torch.empty(16, dtype=torch.float32, device="cuda")
    too_many = L.lbm_conservation_sums_noalloc(19, lbm.LBM_STORE_FP32, 2048, 1024, 1024, 0.0, 0.0,
                                               pop.data_ptr(), out.data_ptr(), None)
    assert too_many == lbm.LBM_ERR_INVALID_ARG
    assert b"2^31" in L.lbm_last_error()
    assert L.lbm_conservation_sums_noalloc(19, lbm.LBM_STORE_FP32, 4, 4, 4, 0.0, 0.0, None, out.data_ptr(),
                                           None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_conservation_sums_noalloc(9, lbm.LBM_STORE_FP32, 4, 4, 2, 0.0, 0.0, pop.data_ptr(),
                                           out.data_ptr(), None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_conservation_sums_noalloc(9, 7, 4, 4, 1, 0.0, 0.0, pop.data_ptr(), out.data_ptr(),
                                           None) == lbm.LBM_ERR_INVALID_ARG
