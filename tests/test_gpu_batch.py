"""Batched domains (lbm_batch_*): every domain of a batch evolves bit for bit
as the same job run alone through lbm_step, whatever the mix, the CTA shape
the autotuner picks, the step budgets and additions or removals between
steps."""
import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _alone(fields, steps, **kw):
    sim = lbm.Lbm(**kw)
    try:
        sim.init(fields.rho, np.ascontiguousarray(fields.u[: sim.d]), 1.5 * fields.T)
        sim.step(steps)
        return sim.moments()
    finally:
        sim.close()


def _same(a, b):
    for k in ("rho", "u", "T", "P"):
        assert np.array_equal(a[k], b[k]), k


def _jobs2d():
    return [
        (W.droplet_2d(64, 0.75, 10.0, seed=41), dict(nx=64, ny=64), 90),
        (W.droplet_2d(96, 0.9, 20.0, seed=42), dict(nx=96, ny=96), 37),
        (W.moving_droplet_2d(n=41, ny=37, radius=9.0, hot_offset=15.0, hot_sigma=3.0), dict(nx=41, ny=37), 64),
        (W.flat_slab_2d(nx=160, ny=33, T=0.8, slab=60, noise=1e-3), dict(nx=160, ny=33), 90),
        (W.droplet_2d(128, 0.7, 30.0, seed=44), dict(nx=128, ny=128, chi_mode=1, chi=0.05), 5),
    ]


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16, lbm.LBM_STORE_FP64])
def test_batch_d2q9_matches_jobs_run_alone(storage):
    jobs = _jobs2d()
    batch = lbm.LbmBatch(lattice=9, storage=storage)
    try:
        ids = [batch.add(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T, steps, **kw) for f, kw, steps in jobs]
        assert batch.size() == len(jobs)
        batch.step(70)      # graph replays of 32 plus a remainder; budgets 37 and 5 stop early
        batch.step(20)
        for i, (f, kw, steps) in zip(ids, jobs):
            done, left = batch.status(i)
            assert done == min(steps, 90) and left == steps - done
            _same(batch.moments(i), _alone(f, done, lattice=9, storage=storage, **kw))
    finally:
        batch.close()


def test_batch_paused_domains_keep_their_state():
    """A domain whose budget is 0 for a request (the serving loop's paused
    jobs) takes no work items and keeps its state bit for bit; the stepping
    domains are unaffected, and every domain, resumed, still matches the same
    job run alone.  The work table changes with the set of stepping domains
    (and the tuner's table of every domain is not kept for stepping)."""
    jobs = [
        (W.pool_boiling_3d(nx=40, ny=36, nz=24, depth=8, noise=1e-3, seed=3),
         dict(nx=40, ny=36, nz=24, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5))),
        (W.droplet_or_slab_3d(24, 0.8, "droplet", seed=7), dict(nx=24, ny=24, nz=24, chi_mode=1, chi=0.05)),
        (W.droplet_or_slab_3d(19, 0.75, "slab", seed=8), dict(nx=19, ny=19, nz=19, chi_mode=1, chi=0.05)),
    ]
    batch = lbm.LbmBatch(lattice=19, storage=lbm.LBM_STORE_FP32)
    try:
        ids = [batch.add(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T, 60, **kw) for f, kw in jobs]
        batch.step(10)
        frozen = batch.get_state(ids[1]).copy()
        batch.set_budget(ids[1], 0)             # paused: 50 steps left, none this request
        batch.step(20)
        assert batch.status(ids[1]) == (10, 0)
        assert np.array_equal(batch.get_state(ids[1]), frozen)
        assert batch.status(ids[0]) == (30, 30) and batch.status(ids[2]) == (30, 30)
        batch.set_budget(ids[1], 50)
        batch.tune(reps=1)                      # a table of every domain, for one step each
        for i in (ids[0], ids[2]):
            batch.set_budget(i, 0)
        batch.step(15)                          # only the resumed domain steps
        assert batch.status(ids[1]) == (25, 35)
        for i in (ids[0], ids[2]):
            batch.set_budget(i, 30)
        batch.step(40)
        for i, (f, kw) in zip(ids, jobs):
            done = batch.status(i)[0]
            assert done == 60
            _same(batch.moments(i), _alone(f, done, lattice=19, storage=lbm.LBM_STORE_FP32, **kw))
    finally:
        batch.close()


def test_batch_d3q19_walls_autotune_and_remove():
    jobs = [
        (W.pool_boiling_3d(nx=40, ny=36, nz=24, depth=8, noise=1e-3, seed=3),
         dict(nx=40, ny=36, nz=24, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5)), 50),
        (W.droplet_or_slab_3d(32, 0.8, "droplet", seed=7), dict(nx=32, ny=32, nz=32, chi_mode=1, chi=0.05), 50),
        (W.droplet_or_slab_3d(24, 0.75, "slab", seed=8), dict(nx=24, ny=24, nz=24, chi_mode=1, chi=0.05), 50),
    ]
    batch = lbm.LbmBatch(lattice=19, storage=lbm.LBM_STORE_FP32)
    try:
        ids = [batch.add(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T, steps, **kw) for f, kw, steps in jobs]
        batch.step(10)
        before = [batch.get_state(i).copy() for i in ids]
        best, ms = batch.tune(reps=2)
        assert 0 <= best < len(batch.variants()) and all(t > 0 for t in ms)
        for i, s in zip(ids, before):     # tuning leaves every state untouched
            assert np.array_equal(batch.get_state(i), s)
        batch.remove(ids[1])
        batch.step(40)
        for j, (i, (f, kw, steps)) in enumerate(zip(ids, jobs)):
            if j == 1:
                continue
            assert batch.status(i) == (50, 0)
            _same(batch.moments(i), _alone(f, 50, lattice=19, storage=lbm.LBM_STORE_FP32, **kw))
        # a domain added later starts from its own initial state
        f, kw, _ = jobs[1]
        k = batch.add(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T, 33, **kw)
        batch.step(40)
        assert batch.status(k) == (33, 0)
        _same(batch.moments(k), _alone(f, 33, lattice=19, storage=lbm.LBM_STORE_FP32, **kw))
    finally:
        batch.close()


def test_batch_rejects_mismatched_domains():
    batch = lbm.LbmBatch(lattice=9, storage=lbm.LBM_STORE_FP32)
    try:
        f = W.droplet_2d(32, 0.8, 8.0)
        with pytest.raises(lbm.LbmError):
            batch.add(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T, 10, nx=32, ny=32, storage=lbm.LBM_STORE_FP64)
        with pytest.raises(lbm.LbmError):
            batch.status(3)
        assert lbm.lbm_domain_bytes(lbm.make_params(nx=32, ny=32)) >= 2 * 2 * 9 * 32 * 32 * 4
    finally:
        batch.close()
