"""Failure detection on the GPU without faulting it: the fused step's
producer/consumer hand-off waits are bounded (about half a second), after
which the CTA finishes without waiting and counts the timeout.  The test
makes one wait run out through the library's fault-injection hook
(LBM_FAULT_DROP_HANDOFF: the first CTA withholds one plane's hand-off) and
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
def test_a_withheld_hand_off_times_out_and_is_reported(monkeypatch, storage):
    monkeypatch.setenv("LBM_FAULT_DROP_HANDOFF", "5")
    sim, f = _sim(storage)
    monkeypatch.delenv("LBM_FAULT_DROP_HANDOFF")
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
