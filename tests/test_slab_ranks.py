"""Slabs over processes on the CPU: gloo ranks each advance one slab of a
domain (the plan of lbm_slab_plan) with the FP64 oracle as the per-slab
step, and swap halos with exchange_halos after every step.  The owned planes,
put back together, must equal the undivided oracle run bit for bit: this
checks the halo depth (two planes per cut), the swap (one message per
neighbour and direction: the populations that cross a cut and the two edge
planes; the receiver restores its own crossing pushes into its halo plane and
completes its edge plane with the neighbour's), the neighbour and tag pairing,
the periodic wrap and the treatment of the cut ends (fixed wall temperatures
only at the domain's walls) independently of the GPU.  The oracle collides its
halo planes too; their pushes across the cut are wrong (a halo plane lacks the
planes beyond it), and the crossing populations must replace them: without
them the run differs.  A rank that leaves between steps, or stays
but withholds its halo, makes its neighbour's swap fail (at once, or after
the process group's timeout) instead of hanging."""
import datetime
import os
import socket
import sys
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    # D2Q9 periodic: two slabs, so both halos of a slab come from the same peer
    "d2q9_periodic_2": dict(world=2, steps=40, p=dict(lattice=9, nx=24, ny=30)),
    # D2Q9 walls, heated floor, cooled lid, latent heat, gravity: three slabs
    "d2q9_walls_3": dict(world=3, steps=40, p=dict(lattice=9, nx=20, ny=33, wall=1, T_fixed_lo=1, T_lo=0.86,
                                                  T_fixed_hi=1, T_hi=0.76, latent=0.02, gravity=(0, -2e-5, 0))),
    # D3Q19 walls with a heated floor, variable conductivity
    "d3q19_walls_2": dict(world=2, steps=12, p=dict(lattice=19, nx=8, ny=6, nz=16, wall=1, T_fixed_lo=1,
                                                   T_lo=0.85, chi_mode=1, chi=0.05)),
    # D3Q19 periodic in three slabs of 6, 6 and 5 planes: the first slab's lower halo wraps to the top
    "d3q19_periodic_3": dict(world=3, steps=10, p=dict(lattice=19, nx=6, ny=6, nz=17, latent=0.02)),
    # D3Q19 closed box (walls on x, y and z, one x wall held at a temperature) in three slabs: at an x or y
    # wall the populations a cut receives come partly from the receiving node's own bounce-back
    "d3q19_box_3": dict(world=3, steps=10, p=dict(lattice=19, nx=7, ny=6, nz=15, wall=1, wall_x=1, wall_y=1,
                                                 T_fixed_x=(1, 0), T_x=(0.84, 0.0), T_fixed_lo=1, T_lo=0.85)),
    # D2Q9 walls on x, periodic last axis, two slabs
    "d2q9_x_walls_2": dict(world=2, steps=30, p=dict(lattice=9, nx=18, ny=26, wall_x=1, T_fixed_x=(0, 1),
                                                    T_x=(0.0, 0.76))),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fields(p):
    from paper_1705_10045_gb300 import workloads as W
    Q = p["lattice"]
    shape = (p.get("nz", 1), p["ny"], p["nx"])
    f = W.spinodal(shape, rho0=0.9 if Q == 19 else 1.0, T0=0.8, noise=2e-2, seed=31)
    return f.rho, f.u[: 2 if Q == 9 else 3], 1.5 * f.T


def _oracle_params(lp):
    """Oracle parameters from an lbm_params structure."""
    import oracle
    return oracle.Params(Q=lp.lattice, nx=lp.nx, ny=lp.ny, nz=lp.nz, kappa=lp.kappa, A=lp.A,
                         barotropic=bool(lp.barotropic), T0=lp.T0, tau=lp.tau, tau_E=lp.tau_E, c_v=lp.c_v,
                         chi_mode=bool(lp.chi_mode), lam=lp.lambda_, chi=lp.chi, g=tuple(lp.gravity),
                         wall=bool(lp.wall), T_fixed_lo=bool(lp.T_fixed_lo), T_fixed_hi=bool(lp.T_fixed_hi),
                         T_lo=lp.T_lo, T_hi=lp.T_hi, wall_x=bool(lp.wall_x), wall_y=bool(lp.wall_y),
                         T_fixed_x=(bool(lp.T_fixed_x[0]), bool(lp.T_fixed_x[1])),
                         T_fixed_y=(bool(lp.T_fixed_y[0]), bool(lp.T_fixed_y[1])),
                         T_x=(lp.T_x[0], lp.T_x[1]), T_y=(lp.T_y[0], lp.T_y[1]),
                         pressure_work=bool(lp.pressure_work),
                         conduction=bool(lp.conduction), pseudoforce=bool(lp.pseudoforce), latent=lp.latent)


def _plane_view(a, Q, first, count):
    """Planes [first, first + count) of the last axis of a (Q, nz, ny, nx) array."""
    return a[:, first:first + count] if Q == 19 else a[:, :, first:first + count]


def _rank(rank, world, port, case, out, leave_after, withhold_at=None, timeout_s=20, skip_round1=False,
          whole_rows=False):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1705_10045_gb300 import lbm
    from paper_1705_10045_gb300.slabs import exchange_halos, local_planes

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))
    try:
        cfg = CASES[case]
        whole = lbm.make_params(**cfg["p"])
        Q = whole.lattice
        nm = whole.ny if Q == 9 else whole.nz
        slab = lbm.lbm_slab_plan(whole, world, rank)
        ax = 0 if Q == 19 else 1
        rho, u, eps = _fields(cfg["p"])
        st = oracle.State(_oracle_params(slab.p), local_planes(rho, slab, ax, nm), local_planes(u, slab, ax + 1, nm),
                          local_planes(eps, slab, ax, nm))

        def get(first, count):
            return torch.from_numpy(np.ascontiguousarray(np.concatenate(
                [_plane_view(st.N, Q, first, count), _plane_view(st.g, Q, first, count)])))

        def put(first, count, t):
            a = t.numpy()
            _plane_view(st.N, Q, first, count)[...] = a[:Q]
            _plane_view(st.g, Q, first, count)[...] = a[Q:]

        # directions whose velocity component along the last axis is +1 / -1,
        # from the oracle's own velocity table
        c = oracle.lattice(Q)["c"]
        c_last = c[:, 2 if Q == 19 else 1]
        dirs = {sgn: np.flatnonzero(c_last == sgn) for sgn in (1, -1)}
        # in-plane axes of a plane slice (Q, ny, nx) for D3Q19, (Q, nx) for D2Q9,
        # with their walls: a crossing population that would come from beyond
        # such a wall is not pushed by the neighbour; the receiving node's own
        # bounce-back wrote it, so the crossing put must leave it alone
        walls = [(0, whole.wall_x, -1)] + ([(1, whole.wall_y, -2)] if Q == 19 else [])

        def get_cross(plane, sgn):
            k = dirs[sgn]
            return torch.from_numpy(np.ascontiguousarray(np.concatenate(
                [_plane_view(st.N, Q, plane, 1)[k], _plane_view(st.g, Q, plane, 1)[k]])))

        def put_cross(plane, sgn, t):
            if skip_round1:
                return
            a, k = t.numpy(), dirs[sgn]
            for f, vals in ((st.N, a[:len(k)]), (st.g, a[len(k):])):
                pv = _plane_view(f, Q, plane, 1)          # (Q, 1, ny, nx) or (Q, 1, 1, nx)
                shape = (len(k),) + ((pv.shape[2], pv.shape[3]) if Q == 19 else (pv.shape[3],))
                cur, new = pv[k].reshape(shape), vals.reshape(shape)
                keep = np.ones(shape, dtype=bool)
                if not whole_rows:
                    for j, kk in enumerate(k):
                        for axis, walled, ax in walls:
                            if walled and c[kk, axis] != 0:
                                idx = [slice(None)] * (len(shape) - 1)
                                idx[ax] = 0 if c[kk, axis] > 0 else -1
                                keep[j][tuple(idx)] = False
                cur[keep] = new[keep]
                pv[k] = cur.reshape(pv[k].shape)

        for s in range(cfg["steps"]):
            if leave_after is not None and rank == world - 1 and s == leave_after:
                out[rank] = "left"
                return          # leaves between steps: the process exits, its sockets close
            if withhold_at is not None and rank == world - 1 and s == withhold_at:
                time.sleep(timeout_s + 2)   # alive, but its halo never comes
                out[rank] = "withheld"
                return
            st.step(1)
            try:
                exchange_halos(dist, slab, get, put, get_cross, put_cross)
            except RuntimeError as e:
                out[rank] = ("failed", s, str(e)[:200])
                return
        out[rank] = (slab.first, slab.own, _plane_view(st.N, Q, slab.lo, slab.own).copy(),
                     _plane_view(st.g, Q, slab.lo, slab.own).copy())
    finally:
        if leave_after is None and withhold_at is None:
            dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_slabs_on_gloo_ranks_equal_the_undivided_oracle_bit_for_bit(case):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_10045_gb300 import lbm
    cfg = CASES[case]
    world = cfg["world"]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, out, None), nprocs=world, join=True)
        got = dict(out)
    whole = lbm.make_params(**cfg["p"])
    Q = whole.lattice
    ref = oracle.State(_oracle_params(whole), *_fields(cfg["p"]))
    ref.step(cfg["steps"])
    N = np.full_like(ref.N, np.nan)
    g = np.full_like(ref.g, np.nan)
    for r in range(world):
        first, own, n, e = got[r]
        _plane_view(N, Q, first, own)[...] = n
        _plane_view(g, Q, first, own)[...] = e
    assert np.array_equal(N, ref.N) and np.array_equal(g, ref.g)
    # the run moved: the state is not the initial one
    init = oracle.State(_oracle_params(whole), *_fields(cfg["p"]))
    assert not np.array_equal(init.N, ref.N)


@pytest.mark.parametrize("case", ["d2q9_walls_3", "d3q19_periodic_3"])
def test_without_the_crossing_populations_the_slabs_differ(case):
    """Negative control: the same runs without putting the crossing
    populations (the edge planes keep the halo planes' own, incomplete pushes
    across the cut) do not reproduce the undivided oracle."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_10045_gb300 import lbm
    cfg = CASES[case]
    world = cfg["world"]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, out, None, None, 20, True), nprocs=world, join=True)
        got = dict(out)
    whole = lbm.make_params(**cfg["p"])
    Q = whole.lattice
    ref = oracle.State(_oracle_params(whole), *_fields(cfg["p"]))
    ref.step(cfg["steps"])
    diff = 0.0
    for r in range(world):
        first, own, n, e = got[r]
        diff = max(diff, np.abs(n - _plane_view(ref.N, Q, first, own)).max())
    assert diff > 1e-12


def test_a_rank_that_leaves_makes_its_neighbours_swap_fail_not_hang():
    world, leave_after = 2, 5
    t0 = time.monotonic()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), "d2q9_periodic_2", out, leave_after), nprocs=world, join=True)
        got = dict(out)
    assert got[1] == "left"
    status, step, _ = got[0]
    assert status == "failed" and step == leave_after
    assert time.monotonic() - t0 < 60


def test_a_rank_that_withholds_its_halo_makes_the_swap_time_out():
    world, at, timeout_s = 2, 4, 3
    t0 = time.monotonic()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), "d2q9_periodic_2", out, None, at, timeout_s), nprocs=world,
                 join=True)
        got = dict(out)
    assert got[1] == "withheld"
    status, step, msg = got[0]
    assert status == "failed" and step == at
    assert "Timed out" in msg or "timeout" in msg.lower()
    assert time.monotonic() - t0 < 60


def test_whole_row_crossing_copies_break_walls_across_the_cut():
    """Negative control for the wall rule: putting whole rows of crossing
    populations overwrites what a node's own bounce-back at an x or y wall
    wrote, and the slabs no longer reproduce the undivided oracle."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1705_10045_gb300 import lbm
    case = "d3q19_box_3"
    cfg = CASES[case]
    world = cfg["world"]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, out, None, None, 20, False, True), nprocs=world,
                 join=True)
        got = dict(out)
    whole = lbm.make_params(**cfg["p"])
    Q = whole.lattice
    ref = oracle.State(_oracle_params(whole), *_fields(cfg["p"]))
    ref.step(cfg["steps"])
    diff = 0.0
    for r in range(world):
        first, own, n, e = got[r]
        diff = max(diff, np.abs(n - _plane_view(ref.N, Q, first, own)).max())
    assert diff > 1e-12
