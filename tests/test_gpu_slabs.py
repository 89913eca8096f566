"""Slabs on the GPU (lbm_slabs_*, lbm_get_planes / lbm_set_planes,
lbm_get_crossing / lbm_set_crossing, lbm_set_step_planes, SlabRank): one
domain cut along its last axis into slabs that collide their owned planes
and, after every step, swap the populations crossing each cut and then two
halo planes.

* FP32 and FP64 slabs reproduce the undivided domain bit for bit (same
  per-node arithmetic), for 1 to 4 slabs, walls with a heated floor, latent
  heat and gravity, a periodic axis where both halos of a slab come from one
  neighbour, and both step forms; also at the full pool-boiling size.
* FP64 slabs match the FP64 oracle to 1e-10.
* FP16 slabs round with their own node keys: within the FP16 bounds of the
  undivided run (the bounds of test_gpu_precision.py).
* The sums over the owned planes equal the undivided domain's to rounding.
* Plane and crossing copies round-trip through host and device buffers and
  reject planes outside the slab; step ranges outside the axis are refused.
* Two processes on the same GPU, one slab each (SlabRank over gloo with host
  staging), reproduce the undivided domain bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from gpu_helpers import max_abs, run_oracle
from paper_1705_10045_gb300 import lbm
from paper_1705_10045_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("rho", "u", "T", "P")


def _walled3d():
    f = W.spinodal((40, 24, 32), rho0=0.9, T0=0.8, noise=2e-2, seed=41)
    kw = dict(lattice=19, nx=32, ny=24, nz=40, wall=1, T_fixed_lo=1, T_lo=0.86, T_fixed_hi=1, T_hi=0.78,
              latent=0.02, gravity=(0.0, 0.0, -2e-5))
    return f, kw, 200


def _periodic2d():
    f = W.spinodal((1, 60, 70), rho0=1.0, T0=0.8, noise=1e-2, seed=42)
    return f, dict(lattice=9, nx=70, ny=60, nz=1), 300


def _box3d():
    # walls on every axis, one x wall held at a temperature: at an x or y wall
    # part of what a cut receives is the receiving node's own bounce-back
    f = W.spinodal((36, 20, 26), rho0=0.9, T0=0.8, noise=2e-2, seed=43)
    kw = dict(lattice=19, nx=26, ny=20, nz=36, wall=1, wall_x=1, wall_y=1, T_fixed_x=(1, 0), T_x=(0.84, 0.0),
              T_fixed_lo=1, T_lo=0.86, gravity=(0.0, 0.0, -2e-5))
    return f, kw, 120


def _xwalls2d():
    f = W.spinodal((1, 48, 50), rho0=1.0, T0=0.8, noise=1e-2, seed=44)
    return f, dict(lattice=9, nx=50, ny=48, nz=1, wall_x=1, T_fixed_x=(0, 1), T_x=(0.0, 0.77)), 200


def _run_whole(f, steps, **kw):
    sim = lbm.Lbm(**kw)
    try:
        sim.init(f.rho, np.ascontiguousarray(f.u[: sim.d]), sim.params.c_v * f.T)
        sim.step(steps)
        return sim.moments(), sim.diagnostics()
    finally:
        sim.close()


def _run_slabs(f, steps, count, **kw):
    s = lbm.Slabs(count, **kw)
    try:
        s.init(f.rho, np.ascontiguousarray(f.u[: s.d]), s.params.c_v * f.T)
        s.step(steps)
        return s.moments(), s.diagnostics()
    finally:
        s.close()


@pytest.mark.parametrize("count", [1, 2, 3, 4])
@pytest.mark.parametrize("case", [_walled3d, _periodic2d, _box3d, _xwalls2d])
def test_fp32_slabs_equal_the_undivided_domain_bit_for_bit(case, count):
    f, kw, steps = case()
    kw = dict(kw, storage=lbm.LBM_STORE_FP32)
    whole, dw = _run_whole(f, steps, **kw)
    part, dp = _run_slabs(f, steps, count, **kw)
    for k in KEYS:
        assert np.array_equal(whole[k], part[k]), k
    assert dp["steps"] == steps
    assert dp["mass"] == pytest.approx(dw["mass"], rel=1e-12)
    assert dp["energy"] == pytest.approx(dw["energy"], rel=1e-12)
    assert np.allclose(dp["momentum"], dw["momentum"], rtol=0, atol=1e-9 * dw["mass"])


@pytest.mark.parametrize("step_kernel", [lbm.LBM_STEP_FUSED, lbm.LBM_STEP_THREE_LAUNCH])
def test_fp64_slabs_equal_the_undivided_domain_and_the_oracle(step_kernel):
    f, kw, steps = _walled3d()
    steps = 60
    kw = dict(kw, storage=lbm.LBM_STORE_FP64, step_kernel=step_kernel)
    whole, _ = _run_whole(f, steps, **kw)
    part, _ = _run_slabs(f, steps, 3, **kw)
    for k in KEYS:
        assert np.array_equal(whole[k], part[k]), k
    o = run_oracle(f, steps, **{k: v for k, v in kw.items() if k not in ("storage", "step_kernel")})
    errs = {k: max_abs(part[k], o[k]) for k in KEYS}
    assert all(v <= 1e-10 for v in errs.values()), errs


def test_fp64_slabs_with_walls_across_the_cut_match_the_oracle():
    f, kw, _ = _box3d()
    steps = 40
    kw = dict(kw, storage=lbm.LBM_STORE_FP64)
    whole, _ = _run_whole(f, steps, **kw)
    part, _ = _run_slabs(f, steps, 3, **kw)
    for k in KEYS:
        assert np.array_equal(whole[k], part[k]), k
    o = run_oracle(f, steps, **{k: v for k, v in kw.items() if k != "storage"})
    errs = {k: max_abs(part[k], o[k]) for k in KEYS}
    assert all(v <= 1e-10 for v in errs.values()), errs


def test_fp16_slabs_stay_within_the_fp16_bounds_of_the_undivided_run():
    f, kw, steps = _periodic2d()
    kw = dict(kw, storage=lbm.LBM_STORE_FP16)
    whole, dw = _run_whole(f, steps, **kw)
    part, dp = _run_slabs(f, steps, 3, **kw)
    bounds = {"rho": 3e-2, "T": 1.5e-2, "u": 5e-3, "P": 5e-4}
    errs = {k: max_abs(whole[k], part[k]) for k in KEYS}
    assert all(errs[k] <= bounds[k] for k in KEYS), errs
    assert dp["mass"] == pytest.approx(dw["mass"], rel=1e-4)


def test_full_size_pool_boiling_in_slabs_equals_the_undivided_run():
    sys.path.insert(0, ROOT)
    import bench
    f = bench._fields()
    kw = dict(bench.PARAMS, storage=lbm.LBM_STORE_FP32)
    steps = 6
    whole, _ = _run_whole(f, steps, **kw)
    for count in (2, 4):
        part, _ = _run_slabs(f, steps, count, **kw)
        for k in KEYS:
            assert np.array_equal(whole[k], part[k]), (count, k)


def test_plane_copies_round_trip_through_host_and_device_buffers():
    import torch
    f, kw, _ = _walled3d()
    for storage in (lbm.LBM_STORE_FP64, lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16):
        a = lbm.Lbm(**dict(kw, storage=storage))
        b = lbm.Lbm(**dict(kw, storage=storage))
        try:
            a.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
            b.init(np.full_like(f.rho, 0.5), np.zeros_like(f.u), np.full_like(f.T, 1.2))
            a.step(5)
            pb = lbm.lbm_plane_bytes(a.h)
            assert pb == 2 * 19 * 32 * 24 * {0: 8, 1: 4, 2: 2}[storage]
            host = np.empty(7 * pb, dtype=np.uint8)
            lbm.lbm_get_planes(a.h, 10, 7, host)
            dev = torch.empty(7 * pb, dtype=torch.uint8, device="cuda")
            lbm.lbm_get_planes(a.h, 10, 7, dev)
            lbm.lbm_sync(a.h)
            assert np.array_equal(host, dev.cpu().numpy())
            # copy every plane of a into b, alternating host and device buffers
            for first in range(0, 40, 8):
                n = min(8, 40 - first)
                if first % 16:
                    buf = np.empty(n * pb, dtype=np.uint8)
                else:
                    buf = torch.empty(n * pb, dtype=torch.uint8, device="cuda")
                lbm.lbm_get_planes(a.h, first, n, buf)
                lbm.lbm_set_planes(b.h, first, n, buf)
            lbm.lbm_sync(b.h)
            sa, sb = a.get_state(), b.get_state()
            assert np.array_equal(sa[16:], sb[16:])
            for bad in ((38, 3), (-1, 2), (0, 41)):
                with pytest.raises(lbm.LbmError) as e:
                    lbm.lbm_get_planes(a.h, bad[0], bad[1], np.empty(max(bad[1], 1) * pb, dtype=np.uint8))
                assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        finally:
            a.close()
            b.close()


def test_crossing_copies_round_trip_and_reject_bad_arguments():
    import torch
    f, kw, _ = _walled3d()
    for storage in (lbm.LBM_STORE_FP64, lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16):
        a = lbm.Lbm(**dict(kw, storage=storage))
        b = lbm.Lbm(**dict(kw, storage=storage))
        try:
            a.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
            b.init(np.full_like(f.rho, 0.5), np.zeros_like(f.u), np.full_like(f.T, 1.2))
            a.step(3)
            cb = lbm.lbm_crossing_bytes(a.h)
            assert cb == 5 * 32 * 24 * 2 * {0: 8, 1: 4, 2: 2}[storage]
            for sign in (1, -1):
                host = np.empty(cb, dtype=np.uint8)
                lbm.lbm_get_crossing(a.h, 17, sign, host)
                dev = torch.empty(cb, dtype=torch.uint8, device="cuda")
                lbm.lbm_get_crossing(a.h, 17, sign, dev)
                lbm.lbm_sync(a.h)
                assert np.array_equal(host, dev.cpu().numpy())
                lbm.lbm_set_crossing(b.h, 5, sign, dev)
                back = np.empty(cb, dtype=np.uint8)
                lbm.lbm_get_crossing(b.h, 5, sign, back)
                assert np.array_equal(back, host)
            # the crossing rows are rows of the plane copy: direction k's row
            pb = lbm.lbm_plane_bytes(a.h) // 19
            plane = np.empty(19 * pb, dtype=np.uint8)
            lbm.lbm_get_planes(a.h, 17, 1, plane)
            host = np.empty(cb, dtype=np.uint8)
            lbm.lbm_get_crossing(a.h, 17, 1, host)
            sys.path.insert(0, ROOT)
            import oracle
            up = np.flatnonzero(oracle.lattice(19)["c"][:, 2] == 1)   # directions with c_z = +1
            assert len(up) == 5
            assert np.array_equal(host, np.concatenate([plane[k * pb:(k + 1) * pb] for k in up]))
            for bad in ((40, 1), (-1, 1), (3, 0), (3, 2)):
                with pytest.raises(lbm.LbmError) as e:
                    lbm.lbm_get_crossing(a.h, bad[0], bad[1], np.empty(cb, dtype=np.uint8))
                assert e.value.code == lbm.LBM_ERR_INVALID_ARG
            for bad in ((-1, 3), (30, 11), (0, -1)):
                with pytest.raises(lbm.LbmError) as e:
                    lbm.lbm_set_step_planes(a.h, *bad)
                assert e.value.code == lbm.LBM_ERR_INVALID_ARG
        finally:
            a.close()
            b.close()


def test_crossing_copies_leave_the_wall_columns_of_the_receiver_alone():
    """With walls on x and y, lbm_set_crossing writes every node of a
    crossing row except the wall column (row) of a direction whose velocity
    points away from that wall, through a host buffer, an aligned device
    buffer and a device buffer one value off a pair boundary (staged)."""
    import torch
    sys.path.insert(0, ROOT)
    import oracle
    f, kw, _ = _box3d()
    nx, ny = kw["nx"], kw["ny"]
    c = oracle.lattice(19)["c"]
    for storage in (lbm.LBM_STORE_FP64, lbm.LBM_STORE_FP32, lbm.LBM_STORE_FP16):
        esz = {0: 8, 1: 4, 2: 2}[storage]
        a = lbm.Lbm(**dict(kw, storage=storage))
        b = lbm.Lbm(**dict(kw, storage=storage))
        try:
            a.init(f.rho, np.ascontiguousarray(f.u), 1.5 * f.T)
            b.init(np.full_like(f.rho, 0.5), np.zeros_like(f.u), np.full_like(f.T, 1.2))
            a.step(3)
            cb = lbm.lbm_crossing_bytes(a.h)
            pb = lbm.lbm_plane_bytes(a.h)
            for sign in (1, -1):
                ks = np.flatnonzero(c[:, 2] == sign)
                rows = np.empty(cb, dtype=np.uint8)
                lbm.lbm_get_crossing(a.h, 11, sign, rows)
                for how in ("host", "device", "unaligned"):
                    before = np.empty(pb, dtype=np.uint8)
                    lbm.lbm_get_planes(b.h, 7, 1, before)
                    if how == "host":
                        buf = rows
                    else:
                        off = 0 if how == "device" else esz
                        big = torch.empty(cb + off, dtype=torch.uint8, device="cuda")
                        big[off:] = torch.from_numpy(rows).cuda()
                        buf = big[off:]
                    lbm.lbm_set_crossing(b.h, 7, sign, buf)
                    lbm.lbm_sync(b.h)
                    after = np.empty(pb, dtype=np.uint8)
                    lbm.lbm_get_planes(b.h, 7, 1, after)
                    want = before.reshape(19, ny, nx, 2 * esz).copy()
                    got_rows = rows.reshape(len(ks), ny, nx, 2 * esz)
                    for j, k in enumerate(ks):
                        keep = np.ones((ny, nx), dtype=bool)
                        if c[k, 0]:
                            keep[:, 0 if c[k, 0] > 0 else nx - 1] = False
                        if c[k, 1]:
                            keep[0 if c[k, 1] > 0 else ny - 1, :] = False
                        want[k][keep] = got_rows[j][keep]
                    assert np.array_equal(after, want.reshape(-1)), (storage, sign, how)
                    # put b back for the next buffer kind
                    lbm.lbm_set_planes(b.h, 7, 1, before)
                    lbm.lbm_sync(b.h)
        finally:
            a.close()
            b.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab_rank(rank, world, port, steps, out, case="walled"):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1705_10045_gb300.slabs import SlabRank
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f, kw, _ = {"walled": _walled3d, "box": _box3d}[case]()
        r = SlabRank(dist, **dict(kw, storage=lbm.LBM_STORE_FP32))
        try:
            r.init(f.rho, f.u, 1.5 * f.T)
            r.step(steps)
            out[rank] = (r.slab.first, r.slab.own, r.moments())
        finally:
            r.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["walled", "box"])
def test_slab_ranks_in_two_processes_equal_the_undivided_domain(case):
    world, steps = 2, 80
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.spawn(_slab_rank, args=(world, _free_port(), steps, out, case), nprocs=world, join=True)
        got = dict(out)
    f, kw, _ = {"walled": _walled3d, "box": _box3d}[case]()
    whole, _ = _run_whole(f, steps, **dict(kw, storage=lbm.LBM_STORE_FP32))
    for r in range(world):
        first, own, m = got[r]
        for k in KEYS:
            ref = whole[k][:, first:first + own] if k == "u" else whole[k][first:first + own]
            assert np.array_equal(ref, m[k]), (r, k)
