"""A step in pieces (lbm_step_begin / lbm_step_end): planes stepped in any
order of disjoint ranges that cover the last axis reproduce lbm_step bit for
bit (every plane reads the step's input and writes its own pushes); while a
step is open the state calls act on its output, and the calls that would
start another step or replace the state refuse."""
import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("rho", "u", "T", "P")


def _cases():
    f3 = W.spinodal((30, 20, 28), rho0=0.9, T0=0.8, noise=2e-2, seed=51)
    kw3 = dict(lattice=19, nx=28, ny=20, nz=30, wall=1, wall_x=1, T_fixed_lo=1, T_lo=0.86,
               gravity=(0.0, 0.0, -2e-5), latent=0.02)
    f2 = W.spinodal((1, 44, 70), rho0=1.0, T0=0.8, noise=1e-2, seed=52)
    kw2 = dict(lattice=9, nx=70, ny=44, nz=1)
    return [(f3, kw3, [(12, 9), (0, 3), (27, 3), (3, 9), (21, 6)]), (f2, kw2, [(40, 4), (0, 20), (20, 20)])]


def _sim(f, kw, storage):
    sim = lbm.Lbm(storage=storage, **kw)
    sim.init(f.rho, np.ascontiguousarray(f.u[: sim.d]), sim.params.c_v * f.T)
    return sim


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP64, lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16])
def test_split_steps_equal_whole_steps_bit_for_bit(storage):
    for f, kw, ranges in _cases():
        a, b = _sim(f, kw, storage), _sim(f, kw, storage)
        try:
            a.step(7)
            for _ in range(7):
                for first, count in ranges:
                    lbm.lbm_step_begin(b.h, first, count)
                lbm.lbm_step_end(b.h)
            assert np.array_equal(a.get_state(), b.get_state()), (kw["lattice"], storage)
            da, db = a.diagnostics(), b.diagnostics()
            assert da["steps"] == db["steps"] == 7
            ma, mb = a.moments(), b.moments()
            for k in KEYS:
                assert np.array_equal(ma[k], mb[k]), k
        finally:
            a.close()
            b.close()


def test_an_open_step_exposes_its_output_and_blocks_other_steps():
    f, kw, ranges = _cases()[0]
    sim = _sim(f, kw, lbm.LBM_STORE_FP32)
    ref = _sim(f, kw, lbm.LBM_STORE_FP32)
    try:
        ref.step(1)
        pb = lbm.lbm_plane_bytes(sim.h)
        want = np.empty(pb, dtype=np.uint8)
        lbm.lbm_get_planes(ref.h, 15, 1, want)
        lbm.lbm_step_begin(sim.h, 14, 3)      # plane 15 and its pushes from 14 and 16
        got = np.empty(pb, dtype=np.uint8)
        lbm.lbm_get_planes(sim.h, 15, 1, got)  # the open step's output
        assert np.array_equal(got, want)
        for call in (lambda: lbm.lbm_step(sim.h, 1), lambda: lbm.lbm_profile_step(sim.h, 1),
                     lambda: sim.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T), lambda: sim.get_state(),
                     lambda: lbm.lbm_moments_f(sim.h)):
            with pytest.raises(lbm.LbmError) as e:
                call()
            assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        for first, count in ((-1, 2), (29, 2), (5, 0)):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_step_begin(sim.h, first, count)
            assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        lbm.lbm_step_begin(sim.h, 0, 14)
        lbm.lbm_step_begin(sim.h, 17, 13)
        lbm.lbm_step_end(sim.h)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step_end(sim.h)
        assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        assert np.array_equal(sim.get_state(), ref.get_state())
        sim.step(2)   # whole steps work again
        ref.step(2)
        assert np.array_equal(sim.get_state(), ref.get_state())
    finally:
        sim.close()
        ref.close()


def test_the_three_launch_form_refuses_split_steps():
    f, kw, _ = _cases()[1]
    sim = _sim(f, dict(kw, step_kernel=lbm.LBM_STEP_THREE_LAUNCH), lbm.LBM_STORE_FP32)
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step_begin(sim.h, 0, 4)
        assert e.value.code == lbm.LBM_ERR_INVALID_ARG
    finally:
        sim.close()
