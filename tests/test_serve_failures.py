"""A failing job fails alone (host logic of serve.Server, no GPU): a stand-in
batch raises the library's errors where the library would.  A job larger
than the memory budget is rejected on arrival; one the library refuses when
it is added, or whose results cannot be read because its state turned
non-physical, gets an error.  Every such job gives back its slot and memory,
and the other jobs complete with their results."""
import numpy as np

from paper_1705_10045_gb300 import lbm, serve

BAD_ADD, BAD_RESULT, HUGE = 11, 13, 999


class FakeBatch:
    """Steps counted per slot; nx selects the failure a job meets."""

    def __init__(self):
        self.slots = {}
        self.removed = []

    def add(self, rho, u, eps, steps, **kw):
        if kw["nx"] == BAD_ADD:
            raise lbm.LbmError(lbm.LBM_ERR_NONPHYSICAL, "lbm_init: 3 nodes with rho <= 0")
        slot = max(self.slots, default=-1) + 1
        self.slots[slot] = {"nx": kw["nx"], "done": 0, "left": steps}
        return slot

    def status(self, slot):
        d = self.slots[slot]
        return d["done"], d["left"]

    def set_budget(self, slot, steps):
        self.slots[slot]["left"] = steps

    def step(self, n):
        for d in self.slots.values():
            k = min(n, d["left"])
            d["done"] += k
            d["left"] -= k

    def moments(self, slot):
        d = self.slots[slot]
        if d["nx"] == BAD_RESULT:
            raise lbm.LbmError(lbm.LBM_ERR_NONPHYSICAL, "non-physical state at 40 node-steps")
        return {"rho": np.full(3, float(d["done"]))}

    def diagnostics(self, slot):
        return np.zeros(8)

    def remove(self, slot):
        self.removed.append(slot)
        del self.slots[slot]


def _server(budget):
    s = object.__new__(serve.Server)
    s.lattice, s.storage = lbm.LBM_D3Q19, lbm.LBM_STORE_FP32
    s.memory_budget, s.max_slots, s.quantum, s.keep_fields = budget, 8, 16, True
    s.policy, s.fill_nodes, s.ride = "all", 0, 0.0
    s.batch = FakeBatch()
    s.resident, s.bytes_in_use = {}, 0
    s.job_bytes = lambda job: 1000 * job.params["nx"]
    return s


def _job(name, nx, steps, arrival):
    def fields():
        z = np.zeros((3, 1, 1, 1))
        return np.ones((1, 1, 1)), z, np.ones((1, 1, 1))
    return serve.Job(name=name, params=dict(nx=nx, ny=1, nz=1), fields=fields, steps=steps, arrival=arrival)


def test_failing_jobs_fail_alone_and_free_their_slots():
    jobs = [_job("ok1", 20, 40, 0.0), _job("bad_add", BAD_ADD, 40, 0.0), _job("huge", HUGE, 40, 0.0),
            _job("bad_result", BAD_RESULT, 30, 0.0), _job("ok2", 21, 50, 0.0)]
    s = _server(budget=100_000)
    st = s.run(jobs)
    by = {j.name: j for j in jobs}
    for name, steps in (("ok1", 40), ("ok2", 50)):
        assert by[name].error is None and by[name].result["rho"][0] == steps
    assert "rho <= 0" in by["bad_add"].error and by["bad_add"].result is None
    assert "budget" in by["huge"].error and by["huge"].admitted is None
    assert "non-physical" in by["bad_result"].error and by["bad_result"].result is None
    assert all(j.completed is not None for j in jobs)
    assert st.completed == 2 and st.failed == 3
    # every admitted job gave its slot and memory back
    assert not s.batch.slots and not s.resident and s.bytes_in_use == 0
    assert sorted(s.batch.removed) == [0, 1, 2]


def test_a_trace_of_only_failures_ends():
    jobs = [_job("bad", BAD_ADD, 10, 0.0), _job("huge", HUGE, 10, 0.0)]
    st = _server(budget=10_000).run(jobs)
    assert st.completed == 0 and st.failed == 2
