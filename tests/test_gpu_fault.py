"""Failure detection on the GPU without faulting it: the fused step's
producer/consumer hand-off waits are bounded (about half a second), after
which the CTA finishes without waiting and counts the timeout.  The test
makes one wait run out through the library's test hook
(lbm_test_drop_handoff: the first CTA withholds one plane's hand-off) and
checks that the host gets LBM_ERR_TIMEOUT, that the error stays latched until
the handle gets a new state, and that the device context stays usable: a
handle created afterwards steps bit for bit like a fresh one.  A domain
larger than device memory is refused with LBM_ERR_OOM (its first allocation
already fails, so nothing is held) and leaves the device usable."""
import time

import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sim(storage=lbm.LBM_STORE_FP32):
    f = W.spinodal((16, 12, 32), rho0=0.9, T0=0.8, noise=1e-2, seed=61)
    sim = lbm.Lbm(lattice=19, nx=32, ny=12, nz=16, storage=storage)
    sim.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
    return sim, f


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP64])
def test_a_withheld_hand_off_times_out_and_is_reported(storage):
    sim, f = _sim(storage)
    lbm.lbm_test_drop_handoff(sim.h, 5)
    try:
        t0 = time.monotonic()
        sim.step(1)
        with pytest.raises(lbm.LbmError) as e:
            sim.sync()
        waited = time.monotonic() - t0
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        assert "hand-off" in str(e.value)
        assert 0.1 < waited < 10.0, waited          # one bounded wait, not a hang
        with pytest.raises(lbm.LbmError) as e:      # latched
            sim.moments()
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        sim.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)   # a new state clears it
        sim.sync()
    finally:
        sim.close()
    # the context is still usable and a handle without the hook is unaffected
    a, _ = _sim(storage)
    b, _ = _sim(storage)
    try:
        a.step(4)
        b.step(4)
        ma, mb = a.moments(), b.moments()
        for k in ("rho", "u", "T", "P"):
            assert np.array_equal(ma[k], mb[k]), k
        assert a.diagnostics()["bad"] == 0
    finally:
        a.close()
        b.close()


def test_a_batch_item_that_never_reports_times_out_its_domain_alone():
    """The persistent batch kernel orders the steps of a domain through
    completion counters.  With the test hook, work item 0 (the first tile of
    domain 0) never reports the end of its first step: the items of domain 0's
    next step wait until their bounded wait runs out, mark the domain aborted
    and skip it, so the request ends in about half a second and domain 0
    reports LBM_ERR_TIMEOUT.  Domain 1 evolves exactly as it does alone."""
    f0 = W.droplet_or_slab_3d(24, 0.8, "droplet", seed=7)
    f1 = W.droplet_or_slab_3d(20, 0.75, "slab", seed=8)
    kw0 = dict(nx=24, ny=24, nz=24, chi_mode=1, chi=0.05)
    kw1 = dict(nx=20, ny=20, nz=20, chi_mode=1, chi=0.05)
    b = lbm.LbmBatch(lattice=19, storage=lbm.LBM_STORE_FP32)
    try:
        i0 = b.add(f0.rho, np.ascontiguousarray(f0.u), 1.5 * f0.T, 6, **kw0)
        i1 = b.add(f1.rho, np.ascontiguousarray(f1.u), 1.5 * f1.T, 6, **kw1)
        assert lbm.load().lbm_batch_test_drop_item(b.b, 0) == lbm.LBM_OK
        t0 = time.monotonic()
        b.step(6)
        with pytest.raises(lbm.LbmError) as e:
            b.sync()
        waited = time.monotonic() - t0
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        assert 0.1 < waited < 10.0, waited
        with pytest.raises(lbm.LbmError) as e:
            b.moments(i0)
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        got = b.moments(i1)
    finally:
        b.close()
    sim = lbm.Lbm(lattice=19, storage=lbm.LBM_STORE_FP32, **kw1)
    try:
        sim.init(f1.rho, np.ascontiguousarray(f1.u), 1.5 * f1.T)
        sim.step(6)
        alone = sim.moments()
    finally:
        sim.close()
    for k in ("rho", "u", "T", "P"):
        assert np.array_equal(got[k], alone[k]), k


def test_a_domain_larger_than_device_memory_is_refused_cleanly():
    import torch
    # 2048 x 1024 x 1023 nodes (just under the 2^31-node limit) in FP64: the
    # first population buffer alone would be 2 Q 8 B = 304 B x 2.1e9 = 652 GB
    p = lbm.make_params(lattice=19, nx=2048, ny=1024, nz=1023, storage=lbm.LBM_STORE_FP64)
    assert lbm.lbm_domain_bytes(p) > torch.cuda.get_device_properties(0).total_memory
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.code == lbm.LBM_ERR_OOM
    sim, _ = _sim()
    try:
        sim.step(2)
        assert sim.diagnostics()["bad"] == 0
    finally:
        sim.close()
