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
