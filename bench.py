"""Benchmark of the thermal multiphase LB lattice update on GB300.

Workload: D3Q19 thermal pool boiling, 384 x 384 x 256 (37,748,736 nodes),
bounce-back walls on z with the bottom wall at T = 0.95 and an adiabatic top,
liquid layer 64 nodes deep at T = 0.8 under its saturated vapour, gravity
-1e-5 z via EDM, +-1e-4 seeded density noise, FP32 populations.  One step is
one lattice update of every node (moments, EOS, force, finite-difference
energy change, collision of both population sets, streaming, walls).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--mode slabs|replicas]

Prints one JSON line (rank 0).  With one GPU the workload runs undivided.
With N > 1 ranks (torchrun, one GPU each) the default mode cuts the one
domain into N slabs along z, one per rank, each holding two halo planes beyond
each cut; every step a rank steps the planes next to its cuts, sends each
neighbour the populations it pushed across the cut and its two edge planes
over NCCL point to point while its interior steps, and then refreshes its
halo planes (strong scaling: value = the domain's lattice updates per
second); --mode replicas
runs an independent copy per rank instead (weak scaling).  The populations
(11.5 GB of reads and writes per step) are far larger than L2, so no flush is
needed.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY, NZ = 384, 384, 256
WORKLOAD = "D3Q19 thermal pool boiling 384x384x256, walls on z (bottom T=0.95 fixed, top adiabatic), " \
           "liquid 64 deep at T=0.8, g=-1e-5 z, FP32"
METRIC = "MLUPS (thermal D3Q19 FP32, pool boiling 384x384x256)"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # HBM3e nominal of the GB300, context only
PARAMS = dict(lattice=19, nx=NX, ny=NY, nz=NZ, wall=1, T_fixed_lo=1, T_lo=0.95, gravity=(0.0, 0.0, -1e-5),
              kappa=0.01, A=-0.152, tau=1.0, tau_E=1.0, c_v=1.5, lambda_=0.05)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


DEPTH = 64


def _set_size(spec: str) -> None:
    """Rescale the pool-boiling box (NXxNYxNZ, liquid a quarter of the height
    deep), e.g. for a profiler capture that must stay small."""
    global NX, NY, NZ, DEPTH, WORKLOAD
    NX, NY, NZ = (int(v) for v in spec.lower().split("x"))
    DEPTH = max(4, NZ // 4)
    PARAMS.update(nx=NX, ny=NY, nz=NZ)
    WORKLOAD = (f"D3Q19 thermal pool boiling {NX}x{NY}x{NZ}, walls on z (bottom T=0.95 fixed, top adiabatic), "
                f"liquid {DEPTH} deep at T=0.8, g=-1e-5 z, FP32")


def _fields():
    from paper_1705_10045_gb300 import workloads as W
    return W.pool_boiling_3d(nx=NX, ny=NY, nz=NZ, T=0.8, depth=DEPTH, noise=1e-4, seed=3)


KERNEL_SOURCES = ("fused.cuh", "kernels.cuh", "lattice.cuh", "backend.cuh")
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "fused_step_kernel_d3q19_fp32.md")


def _kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1705_10045_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def _measured_traffic_per_node():
    """DRAM bytes per node of one fused launch from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    if not os.path.exists(TRAFFIC_SUMMARY):
        return None, None
    vals = {}
    for line in open(TRAFFIC_SUMMARY):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel source sha1") != _kernel_source_hash():
        return None, "stale"
    try:
        return float(vals["dram bytes per node"]), "ncu"
    except (KeyError, ValueError):
        return None, None


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest x over all ranks (the job's time is its slowest rank's);
    x itself when there is no process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Lattice updates of all ranks (one replica each) per second, in millions."""
    return nodes_per_rank * steps * world / seconds / 1e6


def _peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    v = d[key]
                    v = v.get("value", v) if isinstance(v, dict) else v
                    return float(v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_worker(args):
    """One oracle process: a pool-boiling box of side (nx, ny, nz), `warmup`
    untimed steps, then `steps` timed steps (or steps until `budget_s` when
    steps is None).  Returns (nodes * steps, seconds, steps)."""
    nx, ny, nz, depth, seed, warmup, steps, budget_s = args
    import oracle
    from paper_1705_10045_gb300 import workloads as W
    f = W.pool_boiling_3d(nx=nx, ny=ny, nz=nz, T=0.8, depth=depth, noise=1e-4, seed=seed)
    p = oracle.Params(Q=19, nx=nx, ny=ny, nz=nz, wall=True, T_fixed_lo=True, T_lo=0.95, g=(0.0, 0.0, -1e-5))
    s = oracle.State(p, f.rho, f.u, p.c_v * f.T)
    if steps is None:
        t0 = time.perf_counter()
        s.step(1)
        one = time.perf_counter() - t0
        steps = max(1, int(budget_s / max(one, 1e-6)) - 1)
    elif warmup:
        s.step(warmup)
    t0 = time.perf_counter()
    s.step(steps)
    return nx * ny * nz * steps, time.perf_counter() - t0, steps


def oracle_on_cores(box, depth, processes, warmup=0, steps=None, budget_s=15.0):
    """The FP64 C oracle, unchanged, as `processes` independent processes
    (spawned, one box each, different noise seeds) on the host cores.
    Returns (MLUPS over all processes, seconds of the slowest, steps each)."""
    import multiprocessing as mp
    jobs = [(*box, depth, 3 + i, warmup, steps, budget_s) for i in range(processes)]
    if processes == 1:
        res = [_oracle_worker(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(processes) as pool:
            res = pool.map(_oracle_worker, jobs)
    wall = max(r[1] for r in res)
    return sum(r[0] for r in res) / wall / 1e6, wall, res[0][2]


def cpu_baseline(budget_s: float = 15.0):
    """The FP64 C oracle on a bounded sample of the workload: a 96 x 96 x 64
    box of the same structure (walls, heated floor, liquid 16 deep, gravity),
    stepped for about `budget_s` seconds; once on one core, then as one
    process per host core (the oracle is single-threaded; each process steps
    its own box)."""
    box = (96, 96, 64)
    cores = os.cpu_count() or 1
    one, wall1, n1 = oracle_on_cores(box, 16, 1, budget_s=budget_s)
    many, wall_n, n_n = oracle_on_cores(box, 16, cores, steps=n1)
    return {"value": many, "unit": "MLUPS", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"FP64 C oracle, {cores} processes (one per host core), each a D3Q19 96x96x64 box of the "
                      f"same structure (walls, heated floor, liquid 16 deep, gravity), {n_n} steps in {wall_n:.1f} s",
            "single_core": {"value": one, "unit": "MLUPS", "cores": 1,
                            "sample": f"one process, {n1} steps in {wall1:.1f} s"}}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, one process per core,
    each stepping a 64 x 64 x 64 box of the workload's structure."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    n = 64
    cores = os.cpu_count() or 1
    v, dt, _ = oracle_on_cores((n, n, n), 16, cores, warmup=args.warmup, steps=args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{cores} x {n}^3 boxes of the same structure"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"FP64 C oracle, {cores} processes (one per host core), {n}^3 box each, "
                                       f"{args.steps} steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _digest(res: dict) -> str:
    import hashlib
    h = hashlib.sha1()
    for k in ("rho", "u", "T", "P"):
        h.update(np.ascontiguousarray(res[k]).tobytes())
    return h.hexdigest()


BATCH_STEPS = 5000


def storage_leg(storage: int, steps: int, rho_h, u_h, eps_h, stream, dev) -> dict:
    """The headline workload with another population storage format: FP16
    shifted storage (FP32 arithmetic, 152 B per lattice update) or FP64
    (608 B per update; FP64 arithmetic)."""
    import torch
    from paper_1705_10045_gb300 import lbm
    sim = lbm.Lbm(storage=storage, device=dev, stream=stream.cuda_stream, **PARAMS)
    try:
        sim.init(rho_h, u_h, eps_h)
        sim.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        diag = sim.diagnostics()
    finally:
        sim.close()
    nn = NX * NY * NZ
    per_node = {lbm.LBM_STORE_FP16: 152, lbm.LBM_STORE_FP64: 608}[storage]
    peak, kind = _peak()
    gbs = per_node * nn / (ms * 1e-3) / 1e9
    return {"storage": {lbm.LBM_STORE_FP16: "fp16-shifted", lbm.LBM_STORE_FP64: "fp64"}[storage],
            "value": nn / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
            "algorithmic_bytes_per_node": per_node, "achieved_gbs": gbs, "frac": gbs / peak, "peak_kind": kind,
            "bad_nodes": diag["bad"]}


def slabs_leg(count: int, steps: int, rho_h, u_h, eps_h, stream, dev) -> dict:
    """The headline workload cut into `count` slabs along z on this GPU
    (lbm_slabs_*): every slab collides its owned planes, then each cut's
    crossing populations and two halo planes per cut side are copied from the
    neighbours.  Measures what the decomposition costs on one device: the
    copies, the extra launches and each slab's own partial last wave."""
    import torch
    from paper_1705_10045_gb300 import lbm
    s = lbm.Slabs(count, storage=lbm.LBM_STORE_FP32, device=dev, stream=stream.cuda_stream, **PARAMS)
    try:
        s.init(rho_h, u_h, eps_h)
        s.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        diag = s.diagnostics()
        plans = [s.plan(i) for i in range(count)]
    finally:
        s.close()
    nn = NX * NY * NZ
    sides = sum((p.lo > 0) + (p.hi > 0) for p in plans)     # halos, one copy of each per round
    plane_bytes = 2 * 19 * 4 * NX * NY
    crossing_bytes = 2 * 5 * 4 * NX * NY                     # 5 of 19 directions, both sets
    return {"slabs": count, "value": nn / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
            "halo_planes_held": sum(p.lo + p.hi for p in plans), "halo_planes_collided": 0,
            "bytes_copied_per_step": sides * (lbm.LBM_SLAB_HALO * plane_bytes + crossing_bytes),
            # the slabs' fused steps, then one launch per phase of the swap
            # (crossing populations, halo planes) for all cuts together
            "launches_per_step": count + (2 if count > 1 else 0), "bad_nodes": diag["bad"]}


D2Q9_NX, D2Q9_NY = 8192, 4608


def d2q9_leg(steps: int, stream, dev) -> dict:
    """One large D2Q9 domain, FP32: 8192 x 4608 nodes (as many as the D3Q19
    workload), periodic, a liquid slab 4096 nodes across x in its vapour at
    T = 0.8, +-1e-4 noise (144 B per lattice update)."""
    import torch
    from paper_1705_10045_gb300 import lbm
    from paper_1705_10045_gb300 import workloads as W
    f = W.flat_slab_2d(nx=D2Q9_NX, ny=D2Q9_NY, T=0.8, slab=D2Q9_NX // 2, noise=1e-4)
    sim = lbm.Lbm(lattice=9, nx=D2Q9_NX, ny=D2Q9_NY, nz=1, storage=lbm.LBM_STORE_FP32, device=dev,
                  stream=stream.cuda_stream, kappa=0.01, A=-0.152, tau=1.0, tau_E=1.0, c_v=1.5, lambda_=0.05)
    try:
        sim.init(f.rho, np.ascontiguousarray(f.u[:2]), 1.5 * f.T)
        del f
        sim.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        diag = sim.diagnostics()
    finally:
        sim.close()
    nn = D2Q9_NX * D2Q9_NY
    peak, kind = _peak()
    gbs = 144 * nn / (ms * 1e-3) / 1e9
    return {"workload": f"D2Q9 FP32 {D2Q9_NX}x{D2Q9_NY}, periodic, liquid slab across x in vapour at T=0.8",
            "value": nn / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
            "algorithmic_bytes_per_node": 144, "achieved_gbs": gbs, "frac": gbs / peak, "peak_kind": kind,
            "bad_nodes": diag["bad"]}


def batched_bench(count: int = 256, steps: int = BATCH_STEPS):
    """Many uneven D2Q9 droplet domains, FP32: square sides uniform in
    {64, 96, ..., 512}, T uniform in [0.7, 0.95], radius uniform in
    [8, side/4], +-1e-3 noise, constant thermal diffusivity 0.05 (a constant
    conductivity would break the explicit limit in the thinnest vapour at
    T = 0.7), `steps` steps each.  Batched arm: one LbmBatch
    (add every domain from host fields, autotune the CTA shape, advance all
    domains together, copy every domain's moments to the host).  Plain arm:
    the same jobs one after another through lbm_create/lbm_init/lbm_step/
    lbm_moments.  Both timed end to end on the host clock; each job's moments
    are compared bit for bit between the arms."""
    import torch
    from paper_1705_10045_gb300 import lbm
    from paper_1705_10045_gb300 import workloads as W
    jobs = W.batched_droplet_jobs(count)
    kw = dict(lattice=9, storage=lbm.LBM_STORE_FP32, chi_mode=1, chi=0.05)
    inputs = []
    for j in jobs:
        f = W.droplet_2d(j["side"], j["T"], j["radius"], noise=1e-3, seed=j["seed"])
        inputs.append((f.rho, np.ascontiguousarray(f.u), 1.5 * f.T))
    nodes = sum(j["side"] ** 2 for j in jobs)
    torch.cuda.synchronize()

    t0 = time.perf_counter()
    b = lbm.LbmBatch(**kw)
    ids = [b.add(rho, u, eps, steps, nx=j["side"], ny=j["side"], chi_mode=1, chi=0.05)
           for j, (rho, u, eps) in zip(jobs, inputs)]
    best, tune_ms = b.tune(reps=3)
    b.sync()
    t1 = time.perf_counter()
    b.step(steps)
    b.sync()
    t2 = time.perf_counter()
    got = [_digest(b.moments(i)) for i in ids]
    b.close()
    t3 = time.perf_counter()
    batched_s = t3 - t0

    t0 = time.perf_counter()
    ref = []
    for j, (rho, u, eps) in zip(jobs, inputs):
        sim = lbm.Lbm(nx=j["side"], ny=j["side"], **kw)
        sim.init(rho, u, eps)
        sim.step(steps)
        ref.append(_digest(sim.moments()))
        sim.close()
    plain_s = time.perf_counter() - t0
    variants = lbm.LbmBatch(**kw)
    names = variants.variants()
    variants.close()
    return {
        "workload": f"{count} D2Q9 droplet domains, sides 64..512 step 32 ({nodes} nodes), T in [0.7, 0.95], "
                    f"radius in [8, side/4], +-1e-3 noise, chi=0.05, FP32, {steps} steps each",
        "metric": "jobs/s", "value": count / batched_s, "plain_value": count / plain_s,
        "speedup_vs_plain": plain_s / batched_s, "batched_s": batched_s, "plain_s": plain_s,
        "batched_step_s": t2 - t1, "batched_step_mlups": nodes * steps / (t2 - t1) / 1e6,
        "tuned_variant": names[best], "tune_ms_per_launch": dict(zip(names, tune_ms)),
        "bitwise_equal_to_plain": got == ref,
        "timing": "host clock, end to end: host fields in, autotune, all steps, moments of every job out",
    }


def serving_bench(count: int = 128, storage: int = None, seed: int = 5, rate: float = 200.0):
    """Serving stream: Poisson arrivals at 200 jobs/s of D3Q19 droplet/slab
    cubes, sides uniform in [32, 192], steps uniform in [500, 5000], T in
    [0.7, 0.9], constant thermal diffusivity 0.05, FP32 storage (FP16 when
    asked); the first `count` arrivals of the trace.  Served by continuous
    batching (Server) and by plain sequential runs in arrival order; each
    request carries its initial fields (built before the clock starts)."""
    from paper_1705_10045_gb300 import lbm
    from paper_1705_10045_gb300 import serve
    from paper_1705_10045_gb300 import workloads as W
    storage = lbm.LBM_STORE_FP32 if storage is None else storage
    trace = W.serving_trace(count=count, rate=rate, seed=seed)

    def jobs():
        out = serve.trace_jobs(trace)
        for j in out:
            data = j.fields()
            j.fields = (lambda d=data: d)
        return out

    served = jobs()
    srv = serve.Server(lbm.LBM_D3Q19, storage)
    try:
        st = srv.run(served)
    finally:
        srv.close()
    a = {j.name: _digest(j.result) for j in served}
    del served
    plain = jobs()
    sq = serve.run_sequential(plain, lbm.LBM_D3Q19, storage)
    b = {j.name: _digest(j.result) for j in plain}
    del plain
    return {
        "workload": f"first {count} arrivals of a Poisson trace at {rate:g} jobs/s: D3Q19 droplet/slab cubes, side "
                    f"32..192, steps 500..5000, T in [0.7, 0.9], chi=0.05, "
                    f"{'FP16 shifted' if storage == lbm.LBM_STORE_FP16 else 'FP32'} storage",
        "metric": "jobs/s", "value": st.jobs_per_s, "p50_s": st.p50_s, "p99_s": st.p99_s,
        "plain_value": sq.jobs_per_s, "plain_p50_s": sq.p50_s, "plain_p99_s": sq.p99_s,
        "speedup_vs_plain": st.jobs_per_s / sq.jobs_per_s, "p99_vs_plain": st.p99_s / sq.p99_s,
        "mlups": st.mlups, "plain_mlups": sq.mlups, "max_resident": st.max_resident,
        "peak_device_bytes": st.peak_bytes, "wall_s": st.wall_s, "plain_wall_s": sq.wall_s,
        "bitwise_equal_to_plain": a == b,
        "timing": "host clock from the first arrival; latency = results on the host minus arrival",
    }


def slab_main(args, ws, rank, dist):
    """One domain cut into `ws` z-slabs, slab r on rank r (slabs.SlabRank over
    NCCL): every step launches the slab's fused step over the planes next to
    its cuts, posts the swap (crossing populations and two edge planes to each
    neighbour), steps its interior planes while the messages travel, and then
    applies what it received.  Timed like the undivided run; value is the
    whole domain's MLUPS (strong scaling)."""
    import torch
    from paper_1705_10045_gb300 import lbm
    from paper_1705_10045_gb300 import slabs as SL
    stream = torch.cuda.current_stream()
    dev = torch.cuda.current_device()
    f = _fields()
    nn = NX * NY * NZ
    c_v = PARAMS["c_v"]
    r = SL.SlabRank(dist, storage=lbm.LBM_STORE_FP32, device=dev, **PARAMS)
    rho, u, eps = f.rho, np.ascontiguousarray(f.u), c_v * f.T
    del f
    r.init(rho, u, eps)
    r.step(args.warmup)
    prof = lbm.lbm_profile_step(r.h, max(3, min(20, args.steps // 10)))
    own_nodes = NX * NY * r.slab.own
    local_nodes = NX * NY * (r.slab.lo + r.slab.own + r.slab.hi)
    sides = (r.slab.lo > 0) + (r.slab.hi > 0)
    # sent per step: per neighbour the crossing populations and two edge planes
    halo_bytes = sides * (r.cross_bytes + lbm.LBM_SLAB_HALO * r.plane_bytes)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        e0.record(stream)
        r.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    dist.barrier()
    # end to end: host fields in, steps, owned planes' moments out
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    r.init(rho, u, eps)
    r.step(args.steps)
    out = r.moments()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    h2d = local_nodes * (2 + 3) * 8
    d2h = sum(v.size for v in out.values()) * 8
    r.close()
    if rank == 0:
        peak, peak_kind = _peak()
        top = max(prof, key=prof.get)
        # algorithmic bytes: the populations of the owned nodes read and written
        achieved = 4 * 19 * 4 * own_nodes / (prof[top] * 1e-3) / 1e9
        value = nn * args.steps / (ms * 1e-3) / 1e6
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": nn, "parallelism": f"z-slabs x{ws} (2 halo planes per cut, crossing populations then halo planes)",
                       "l2": "inputs larger than L2, no flush", "nodes_per_rank_owned": own_nodes,
                       "nodes_per_rank_stepped": local_nodes},
            "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "algorithmic_bytes_per_node": 4 * 19 * 4, "kernel_ms": prof},
            "e2e": {"value": nn * args.steps / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps},
            "halo_bytes_per_rank_per_step": halo_bytes * 2,
            # per step: the fused step in ranges (planes next to the cuts, then
            # the interior), and per neighbour five copy kernels (crossing
            # populations and edge planes out; halo planes, own crossing
            # populations and the neighbour's in)
            "gpu_launches": args.steps * (sum(len(x) for x in r._ranges()) + 5 * sides),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-domains measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--no-storage-legs", action="store_true", help="skip the FP16 and FP64 storage legs")
    ap.add_argument("--no-slabs", action="store_true", help="skip the slab-decomposition measurement")
    ap.add_argument("--no-d2q9", action="store_true", help="skip the single-domain D2Q9 measurement")
    ap.add_argument("--d2q9-size", default=None, help="NXxNY of a smaller D2Q9 domain (profiling)")
    ap.add_argument("--serve-jobs", type=int, default=128,
                    help="arrivals served in each serving measurement (saturated and below saturation)")
    ap.add_argument("--size", default=None, help="NXxNYxNZ of a smaller pool-boiling box (profiling)")
    ap.add_argument("--mode", default="slabs", choices=["slabs", "replicas"],
                    help="with several ranks: one domain in z-slabs (default) or a replica per rank")
    args = ap.parse_args()
    if args.size:
        _set_size(args.size)
    if args.d2q9_size:
        global D2Q9_NX, D2Q9_NY
        D2Q9_NX, D2Q9_NY = (int(v) for v in args.d2q9_size.lower().split("x"))
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if args.mode == "slabs":
            return slab_main(args, ws, rank, dist)
    else:
        torch.cuda.set_device(local)
    from paper_1705_10045_gb300 import lbm
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    f = _fields()
    nn = NX * NY * NZ
    c_v = PARAMS["c_v"]
    # pinned host copies of the inputs (used by the end-to-end leg)
    rho_h = torch.from_numpy(f.rho).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(f.u)).pin_memory()
    eps_h = torch.from_numpy(c_v * f.T).pin_memory()
    del f

    sim = lbm.Lbm(storage=lbm.LBM_STORE_FP32, device=dev, stream=stream.cuda_stream, **PARAMS)
    sim.init(rho_h, u_h, eps_h)
    launches = lbm.lbm_launches_per_step(sim.h)

    # warm-up, then per-kernel event timing of a few steps for the roofline
    sim.step(args.warmup)
    prof = lbm.lbm_profile_step(sim.h, max(3, min(20, args.steps // 10)))
    torch.cuda.synchronize()

    # timed region: K steps between events on the library's stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if dist:
        ms = max_over_ranks(ms, dist)
        dist.barrier()
    diag = sim.diagnostics()

    # end to end through the C-ABI with host buffers: init from pinned host
    # fields, K steps, moments back to pinned host buffers
    out = {k: torch.empty(shape, dtype=torch.float64).pin_memory()
           for k, shape in (("rho", (NZ, NY, NX)), ("u", (3, NZ, NY, NX)), ("T", (NZ, NY, NX)),
                            ("P", (NZ, NY, NX)))}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # events around the steps and host clock marks split the end-to-end time
    # into init (fields in), steps and moments (fields out); clocks sampled
    # over the whole leg
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as e2e_clk:
        t0 = time.perf_counter()
        sim.init(rho_h, u_h, eps_h)
        t_init = time.perf_counter()
        s0.record(stream)
        sim.step(args.steps)
        s1.record(stream)
        lbm.lbm_moments(sim.h, out["rho"], out["u"], out["T"], out["P"])
        e2e_s = time.perf_counter() - t0
    e2e_parts = {"init_ms": (t_init - t0) * 1e3, "steps_ms_per_step": s0.elapsed_time(s1) / args.steps,
                 "moments_ms": (e2e_s - (t_init - t0)) * 1e3 - s0.elapsed_time(s1), "clocks": e2e_clk.summary()}
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist)
    h2d = (rho_h.numel() + u_h.numel() + eps_h.numel()) * 8
    d2h = sum(v.numel() for v in out.values()) * 8
    sim.close()
    extra_storage = {}
    if not args.no_storage_legs:
        extra_storage["fp16_storage"] = storage_leg(lbm.LBM_STORE_FP16, min(args.steps, 200), rho_h, u_h, eps_h,
                                                    stream, dev)
        extra_storage["fp64"] = storage_leg(lbm.LBM_STORE_FP64, min(args.steps, 10), rho_h, u_h, eps_h, stream, dev)
    if not args.no_d2q9:
        extra_storage["d2q9_fp32"] = d2q9_leg(min(args.steps, 200), stream, dev)
    if not args.no_slabs:
        extra_storage["slabs_on_one_gpu"] = [slabs_leg(c, min(args.steps, 100), rho_h, u_h, eps_h, stream, dev)
                                             for c in (2, 4)]

    if rank == 0:
        peak, peak_kind = _peak()
        top = max(prof, key=prof.get)
        # algorithmic bytes of the dominant kernel per node: the collide kernel
        # reads and writes both FP32 population sets (4 Q s = 304 B) and reads
        # the 8 field values it needs of its own node (32 B)
        algo_bytes = {"collide_kernel": 4 * 19 * 4 + 8 * 4}.get(top, 4 * 19 * 4)
        achieved = algo_bytes * nn / (prof[top] * 1e-3) / 1e9
        traffic_per_node, traffic_src = _measured_traffic_per_node() if top == "fused_step_kernel" else (None, None)
        value = whole_job_mlups(nn, args.steps, ws, ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": nn, "l2": f"inputs larger than L2 ({304 * nn / 1e9:.2f} GB of population "
                       "traffic per step vs 129 MB L2), no flush",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "one GPU, undivided domain"},
            "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic_per_node * nn if traffic_per_node else None,
                         "traffic_source": traffic_src,
                         "algorithmic_bytes_per_node": algo_bytes, "kernel_ms": prof,
                         "step_bytes_per_node": 4 * 19 * 4,
                         "step_frac": 4 * 19 * 4 * nn / (ms / args.steps * 1e-3) / 1e9 / peak,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
            "e2e": {"value": whole_job_mlups(nn, args.steps, ws, e2e_s), "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "parts": e2e_parts},
            "gpu_launches": launches * args.steps,
            "clocks": clk.summary(),
            "diagnostics": {"mass": diag["mass"], "energy": diag["energy"], "clamps": diag["clamps"],
                            "bad": diag["bad"]},
        }
        line.update(extra_storage)
        if ws == 1 and not args.no_batched:
            line["batched"] = batched_bench()
        if ws == 1 and not args.no_serving:
            line["serving"] = serving_bench(args.serve_jobs)
            # the 200 jobs/s stream saturates the GPU; latency percentiles of a
            # stream below saturation: arrivals at 0.7x the served completion rate
            sub_rate = 0.7 * line["serving"]["value"]
            line["serving_below_saturation"] = serving_bench(args.serve_jobs, seed=6, rate=sub_rate)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
