"""Continuous-batching service for simulation jobs on one GPU.

Jobs (a lattice size, physics parameters, initial fields and a number of
steps) arrive over time.  The server keeps every admitted job's populations
resident in device memory inside one ``LbmBatch`` and advances all resident
jobs together, one launch per step for the whole mix.  A job is admitted as
soon as it has arrived and its device memory (``lbm_domain_bytes``) fits in
the budget next to the jobs already resident, and a slot is free; it leaves
when its step budget is spent, its moments are copied to the host and its
memory is freed for the next arrivals.  Admission is first come, first
served: a job that does not fit blocks later arrivals (no reordering), so
large jobs are not starved.

A failing job fails alone.  A job larger than the whole memory budget is
rejected on arrival.  The library may refuse a job when it is added (bad
parameters, a non-physical or unstable initial state, no device memory).
Or its state may turn non-physical while it runs, which shows when its
results are read.  In each case the job gets an ``error`` and no result,
its slot and memory are freed, and the other jobs go on.

Which resident jobs advance in a round is the policy's choice:

* ``"fill"`` (default): jobs in admission order, the oldest first, are
  advanced while their node count adds up to at most the larger of
  ``fill_nodes`` (enough nodes to keep the GPU busy) and (1 + ``ride``) times
  the oldest job's; the others wait with their state resident.  Large jobs
  then run nearly one at a time in arrival order, and small jobs ride along
  at almost no cost, which keeps the latency of both low.
* ``"all"``: every resident job advances every round (processor sharing).

Latency of a job is completion (results on the host) minus arrival;
throughput is completed jobs per wall-clock second.  ``run_sequential`` runs
the same trace the plain way (one job at a time, lbm_step per job) for
comparison.  Each job's result is bit for bit the one it gets alone (the
batch kernel and the single-domain kernel share their per-node code).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import lbm


@dataclass
class Job:
    """One simulation request.  `fields()` returns (rho, u, T) host arrays."""
    name: str
    params: dict
    fields: Callable[[], tuple]
    steps: int
    arrival: float = 0.0                       # seconds after the start of the trace
    admitted: Optional[float] = None
    completed: Optional[float] = None
    result: Optional[dict] = None
    error: Optional[str] = None                # why the job failed (None: it succeeded)

    @property
    def latency(self) -> Optional[float]:
        return None if self.completed is None else self.completed - self.arrival


@dataclass
class ServeStats:
    completed: int
    wall_s: float
    jobs_per_s: float
    p50_s: float
    p99_s: float
    max_resident: int
    peak_bytes: int
    lattice_updates: float
    mlups: float
    extra: dict = field(default_factory=dict)
    failed: int = 0


def _percentile(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if xs else float("nan")


def _stats(jobs, wall, max_resident, peak_bytes, lu) -> ServeStats:
    lat = [j.latency for j in jobs if j.latency is not None and j.error is None]
    done = len(lat)
    return ServeStats(completed=done, wall_s=wall, jobs_per_s=done / wall if wall > 0 else float("nan"),
                      p50_s=_percentile(lat, 50), p99_s=_percentile(lat, 99), max_resident=max_resident,
                      peak_bytes=peak_bytes, lattice_updates=lu, mlups=lu / wall / 1e6 if wall > 0 else float("nan"),
                      failed=sum(1 for j in jobs if j.error is not None))


def _nodes(params: dict) -> int:
    return int(params.get("nx", 1)) * int(params.get("ny", 1)) * int(params.get("nz", 1))


class Server:
    """Continuous batching of jobs of one lattice and storage format."""

    def __init__(self, lattice: int, storage: int, memory_budget: Optional[int] = None, max_slots: int = 4096,
                 quantum: int = 128, device: int = 0, keep_fields: bool = True, policy: str = "fill",
                 fill_nodes: int = 8_000_000, ride: float = 0.25):
        import torch
        self.lattice, self.storage = lattice, storage
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            memory_budget = int(0.8 * free)
        self.memory_budget = int(memory_budget)
        self.max_slots = max_slots
        self.quantum = int(quantum)
        self.keep_fields = keep_fields
        if policy not in ("fill", "all"):
            raise ValueError(f"unknown policy {policy}")
        self.policy, self.fill_nodes, self.ride = policy, int(fill_nodes), float(ride)
        self.batch = lbm.LbmBatch(lattice=lattice, storage=storage, device=device)
        self.resident = {}          # slot id -> (job, bytes)
        self.bytes_in_use = 0

    def job_bytes(self, job: Job) -> int:
        kw = dict(job.params, lattice=self.lattice, storage=self.storage)
        return lbm.lbm_domain_bytes(lbm.make_params(**kw))

    @staticmethod
    def _fail(job: Job, why: str, now: float) -> None:
        job.error = why
        job.completed = now

    def _admit(self, job: Job, nbytes: int, now: float) -> bool:
        rho, u, T = job.fields()
        kw = dict(job.params)
        c_v = kw.get("c_v", 1.5)
        d = 2 if self.lattice == lbm.LBM_D2Q9 else 3
        try:
            slot = self.batch.add(np.ascontiguousarray(rho), np.ascontiguousarray(u[:d]),
                                  np.ascontiguousarray(c_v * T), job.steps, **kw)
        except lbm.LbmError as e:
            self._fail(job, str(e), now)
            return False
        self.resident[slot] = (job, nbytes)
        self.bytes_in_use += nbytes
        job.admitted = now
        return True

    def _retire(self, slot: int, now_fn) -> None:
        job, nbytes = self.resident.pop(slot)
        try:
            res = self.batch.moments(slot)
            res["diagnostics"] = self.batch.diagnostics(slot)
            job.result = res if self.keep_fields else {"diagnostics": res["diagnostics"]}
        except lbm.LbmError as e:      # e.g. its state turned non-physical
            job.error = str(e)
        finally:
            self.batch.remove(slot)
            self.bytes_in_use -= nbytes
            job.completed = now_fn()

    def run(self, jobs: list, clock: Callable[[], float] = time.perf_counter) -> ServeStats:
        """Serve a trace: jobs become available at their arrival times
        (seconds after the call), in arrival order."""
        queue = sorted(jobs, key=lambda j: j.arrival)
        t0 = clock()
        now = lambda: clock() - t0
        nxt = 0
        max_resident, peak = 0, 0
        lu = 0.0
        while nxt < len(queue) or self.resident:
            t = now()
            # admit arrivals in order while memory and slots allow (head-of-line blocking)
            while nxt < len(queue) and queue[nxt].arrival <= t and len(self.resident) < self.max_slots:
                job = queue[nxt]
                try:
                    need = self.job_bytes(job)
                except (lbm.LbmError, AttributeError, ValueError, TypeError) as e:
                    self._fail(job, f"bad parameters: {e}", t)
                    nxt += 1
                    continue
                if need > self.memory_budget:
                    self._fail(job, f"needs {need} bytes of device memory, the budget is {self.memory_budget}", t)
                    nxt += 1
                    continue
                if self.resident and self.bytes_in_use + need > self.memory_budget:
                    break
                self._admit(job, need, t)
                nxt += 1
            max_resident = max(max_resident, len(self.resident))
            peak = max(peak, self.bytes_in_use)
            if not self.resident:
                # idle until the next arrival
                if nxt < len(queue):
                    wait = queue[nxt].arrival - now()
                    if wait > 0:
                        time.sleep(wait)
                continue
            # advance the chosen jobs by the quantum (each stops at its own budget);
            # a shorter quantum when a job is about to finish keeps its latency low
            active = self._choose()
            left = [self.batch.status(s)[1] for s in active]
            q = max(1, min(self.quantum, min(left)))
            paused = [(s, self.batch.status(s)[1]) for s in self.resident if s not in active]
            for s, _ in paused:
                self.batch.set_budget(s, 0)
            lu += sum(min(q, l) * _nodes(self.resident[s][0].params) for s, l in zip(active, left))
            self.batch.step(q)
            for s, l in paused:
                self.batch.set_budget(s, l)
            for s in [s for s in active if self.batch.status(s)[1] == 0]:
                self._retire(s, now)
        return _stats(queue, now(), max_resident, peak, lu)

    def _choose(self) -> list:
        """Resident slots that advance this round (admission order)."""
        order = list(self.resident)
        if self.policy == "all":
            return order
        head = _nodes(self.resident[order[0]][0].params)
        target = max(self.fill_nodes, (1.0 + self.ride) * head)
        active, total = [], 0
        for s in order:
            n = _nodes(self.resident[s][0].params)
            if not active or total + n <= target:
                active.append(s)
                total += n
        return active

    def close(self):
        self.batch.close()


def run_sequential(jobs: list, lattice: int, storage: int, device: int = 0, keep_fields: bool = True,
                   clock: Callable[[], float] = time.perf_counter) -> ServeStats:
    """The plain way: jobs in arrival order, one at a time, each on its own
    handle (create, init, lbm_step(steps), moments, destroy)."""
    queue = sorted(jobs, key=lambda j: j.arrival)
    t0 = clock()
    now = lambda: clock() - t0
    lu = 0.0
    for job in queue:
        wait = job.arrival - now()
        if wait > 0:
            time.sleep(wait)
        job.admitted = now()
        rho, u, T = job.fields()
        kw = dict(job.params)
        sim = None
        try:
            sim = lbm.Lbm(lattice=lattice, storage=storage, device=device, **kw)
            c_v = kw.get("c_v", 1.5)
            sim.init(np.ascontiguousarray(rho), np.ascontiguousarray(u[: sim.d]), np.ascontiguousarray(c_v * T))
            sim.step(job.steps)
            res = sim.moments()
            res["diagnostics"] = lbm.lbm_diagnostics(sim.h)
            job.result = res if keep_fields else {"diagnostics": res["diagnostics"]}
            lu += job.steps * _nodes(job.params)
        except lbm.LbmError as e:
            job.error = str(e)
        finally:
            if sim is not None:
                sim.close()
        job.completed = now()
    return _stats(queue, now(), 1, 0, lu)


def trace_jobs(trace: list, chi: float = 0.05, noise: float = 1e-3) -> list:
    """Jobs of a serving trace (``workloads.serving_trace``): D3Q19 periodic
    cubes holding a centred drop or a liquid slab at the job's temperature,
    constant thermal diffusivity chi."""
    from . import workloads as W

    jobs = []
    for k, t in enumerate(trace):
        n = t["side"]

        def make(n=n, T=t["T"], kind=t["kind"], seed=t["seed"]):
            f = W.droplet_or_slab_3d(n, T, kind, noise=noise, seed=seed)
            return f.rho, f.u, f.T

        jobs.append(Job(name=f"job{k}", params=dict(nx=n, ny=n, nz=n, chi_mode=1, chi=chi), fields=make,
                        steps=t["steps"], arrival=t["arrival"]))
    return jobs
