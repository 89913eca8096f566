"""The continuous-batching server: every job's result equals the job run
alone, admission respects the device-memory budget, and jobs that arrive
while others run join the mix."""
import numpy as np
import pytest

from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import serve
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_trace(count=10, seed=11):
    trace = W.serving_trace(count=count, rate=400.0, seed=seed, side_lo=16, side_hi=40, steps_lo=20, steps_hi=150)
    return serve.trace_jobs(trace)


def _alone(job):
    rho, u, T = job.fields()
    sim = lbm.Lbm(lattice=lbm.LBM_D3Q19, storage=lbm.LBM_STORE_FP32, **job.params)
    try:
        sim.init(rho, np.ascontiguousarray(u), 1.5 * T)
        sim.step(job.steps)
        return sim.moments()
    finally:
        sim.close()


@pytest.mark.parametrize("policy", [dict(policy="all"), dict(policy="fill", fill_nodes=0, ride=0.25)])
def test_served_results_equal_jobs_run_alone(policy):
    # fill_nodes = 0 makes the fill policy pause every job much larger than
    # the oldest, so jobs stop and resume between rounds
    jobs = _small_trace()
    srv = serve.Server(lbm.LBM_D3Q19, lbm.LBM_STORE_FP32, quantum=32, **policy)
    try:
        st = srv.run(jobs)
    finally:
        srv.close()
    assert st.completed == len(jobs) and st.max_resident >= 2
    for j in jobs:
        assert j.completed >= j.arrival and j.latency > 0
        alone = _alone(j)
        for k in ("rho", "u", "T", "P"):
            assert np.array_equal(j.result[k], alone[k]), (j.name, k)


def test_admission_respects_memory_budget():
    jobs = _small_trace(count=8, seed=12)
    per_job = [lbm.lbm_domain_bytes(lbm.make_params(lattice=19, storage=lbm.LBM_STORE_FP32, **j.params))
               for j in jobs]
    budget = 2 * max(per_job)
    srv = serve.Server(lbm.LBM_D3Q19, lbm.LBM_STORE_FP32, memory_budget=budget, quantum=16)
    try:
        st = srv.run(jobs)
    finally:
        srv.close()
    assert st.completed == len(jobs)
    assert st.peak_bytes <= budget
    # first come, first served: completion order never lets a later arrival be admitted first
    adm = [j.admitted for j in sorted(jobs, key=lambda j: j.arrival)]
    assert adm == sorted(adm)


def test_late_arrivals_wait_and_sequential_baseline_matches():
    jobs = _small_trace(count=3, seed=13)
    jobs[-1].arrival += 0.3          # the server idles until it arrives
    srv = serve.Server(lbm.LBM_D3Q19, lbm.LBM_STORE_FP32)
    try:
        st = srv.run(jobs)
    finally:
        srv.close()
    assert st.completed == 3 and st.wall_s >= 0.3
    seq = _small_trace(count=3, seed=13)
    seq[-1].arrival += 0.3
    st2 = serve.run_sequential(seq, lbm.LBM_D3Q19, lbm.LBM_STORE_FP32)
    assert st2.completed == 3
    for a, b in zip(jobs, seq):
        assert np.array_equal(a.result["rho"], b.result["rho"])


def test_a_failing_job_fails_alone():
    """A job whose initial density is not positive is refused when it is
    added, and one larger than the budget is rejected on arrival; both get an
    error and free nothing they did not take, and the other jobs' results
    are the ones they get alone."""
    jobs = _small_trace(count=6, seed=13)
    bad_fields = jobs[1].fields

    def negative_density():
        rho, u, T = bad_fields()
        rho = rho.copy()
        rho.flat[7] = -0.1
        return rho, u, T

    jobs[1].fields = negative_density
    per_job = max(lbm.lbm_domain_bytes(lbm.make_params(lattice=19, storage=lbm.LBM_STORE_FP32, **j.params))
                  for j in jobs)
    budget = 3 * per_job
    jobs[3].params = dict(jobs[3].params, nx=256, ny=256, nz=256)   # far over the budget
    srv = serve.Server(lbm.LBM_D3Q19, lbm.LBM_STORE_FP32, memory_budget=budget, quantum=16)
    try:
        st = srv.run(jobs)
        assert not srv.resident and srv.bytes_in_use == 0 and srv.batch.size() == 0
    finally:
        srv.close()
    assert st.failed == 2 and st.completed == len(jobs) - 2
    assert jobs[1].error and "lbm_init" in jobs[1].error and jobs[1].result is None
    assert jobs[3].error and "budget" in jobs[3].error and jobs[3].result is None
    for k, j in enumerate(jobs):
        if k in (1, 3):
            continue
        assert j.error is None
        alone = _alone(j)
        for f in ("rho", "u", "T", "P"):
            assert np.array_equal(j.result[f], alone[f]), (j.name, f)
