"""Seeded synthetic input fields for the thermal multiphase LB workloads.

This module builds initial density, velocity and temperature fields (and job
lists for the batched and served forms).  It contains no step arithmetic of
the method: only geometry (distances to interfaces), tanh profiles, a
counter-based random number generator and a linear interpolation of the
stored Maxwell coexistence table.  Both the CUDA path and the CPU oracle are
fed from here, so the two always see identical inputs.

Conventions: scalar fields have shape (nz, ny, nx) (nz = 1 for D2Q9), velocity
(d, nz, ny, nx), all float64.  Interface profiles follow
rho = (rho_l + rho_v)/2 + (rho_l - rho_v)/2 * tanh(2 s / W) with s the signed
distance to the interface (positive in the liquid) and W the width.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

_TABLE = None


def _table():
    global _TABLE
    if _TABLE is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "coexistence_vdw.json")
        with open(path) as f:
            _TABLE = np.array(json.load(f)["rows"], dtype=np.float64)
    return _TABLE


def coexistence(T: float) -> tuple[float, float]:
    """(rho_v, rho_l) of the stored Maxwell table, linearly interpolated in T."""
    t = _table()
    if not (t[0, 0] <= T <= t[-1, 0]):
        raise ValueError(f"T={T} outside the coexistence table [{t[0, 0]}, {t[-1, 0]}]")
    return float(np.interp(T, t[:, 0], t[:, 1])), float(np.interp(T, t[:, 0], t[:, 2]))


# ---------------------------------------------------------------------------
# counter-based uniform noise: splitmix64 of (seed * golden + node index)

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_noise(shape, amplitude: float, seed: int, offset: int = 0) -> np.ndarray:
    """Additive noise uniform in [-amplitude, amplitude), one draw per node index."""
    n = int(np.prod(shape))
    with np.errstate(over="ignore"):
        idx = np.arange(offset, offset + n, dtype=np.uint64) + np.uint64(seed) * np.uint64(0xD1B54A32D192ED03)
    bits = splitmix64(idx) >> np.uint64(11)
    u01 = bits.astype(np.float64) * (1.0 / 9007199254740992.0)
    return (amplitude * (2.0 * u01 - 1.0)).reshape(shape)


def _profile(s, rho_v, rho_l, width):
    return 0.5 * (rho_l + rho_v) + 0.5 * (rho_l - rho_v) * np.tanh(2.0 * s / width)


@dataclass
class Fields:
    """Initial fields of one domain."""
    rho: np.ndarray
    u: np.ndarray
    T: np.ndarray

    @property
    def shape(self):
        return self.rho.shape


def flat_slab_2d(nx=128, ny=128, T=0.8, slab=64, width=4.0, noise=0.0, seed=1) -> Fields:
    """Liquid slab of `slab` nodes across x, centred, in its saturated vapour;
    periodic domain at rest, uniform temperature (D2Q9 two-phase workload)."""
    rv, rl = coexistence(T)
    x = np.arange(nx, dtype=np.float64)
    x0 = (nx - slab) / 2.0 - 0.5
    x1 = x0 + slab
    s = np.minimum(x - x0, x1 - x)
    rho = np.broadcast_to(_profile(s, rv, rl, width)[None, None, :], (1, ny, nx)).copy()
    if noise:
        rho += uniform_noise(rho.shape, noise, seed)
    return Fields(rho, np.zeros((2, 1, ny, nx)), np.full((1, ny, nx), T))


def moving_droplet_2d(n=512, T=0.85, radius=64.0, ux=0.05, uy=0.0, width=4.0, noise=1e-3, seed=2,
                      hot_dT=0.05, hot_sigma=10.0, hot_offset=192.0, ny=None) -> Fields:
    """Circular drop in a periodic n x n box (n x ny when ny is given), whole
    fluid moving at (ux, uy), with uniform density noise and a Gaussian hot
    spot in the vapour `hot_offset` nodes from the drop centre along x
    (D2Q9 moving-droplet workload)."""
    rv, rl = coexistence(T)
    nx = n
    ny = n if ny is None else ny
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    cx, cy = nx / 2.0, ny / 2.0
    s = radius - np.hypot(x - cx, y - cy)
    rho = _profile(s, rv, rl, width)[None]
    if noise:
        rho = rho + uniform_noise(rho.shape, noise, seed)
    u = np.zeros((2, 1, ny, nx))
    u[0] = ux
    u[1] = uy
    hx = (cx + hot_offset) % nx
    dx = np.minimum(np.abs(x - hx), nx - np.abs(x - hx))
    Tf = T + hot_dT * np.exp(-(dx ** 2 + (y - cy) ** 2) / (2.0 * hot_sigma ** 2))
    return Fields(rho, u, Tf[None])


def pool_boiling_3d(nx=384, ny=384, nz=256, T=0.8, depth=64, width=4.0, noise=1e-4, seed=3) -> Fields:
    """Liquid layer `depth` nodes deep on the bottom wall under its saturated
    vapour, at rest and uniform temperature, with uniform density noise
    (D3Q19 pool-boiling workload; walls on z)."""
    rv, rl = coexistence(T)
    z = np.arange(nz, dtype=np.float64)
    s = (depth - 0.5) - z
    prof = _profile(s, rv, rl, width)
    rho = np.empty((nz, ny, nx))
    rho[:] = prof[:, None, None]
    if noise:
        for k in range(nz):   # per plane keeps the temporary small at full size
            rho[k] += uniform_noise((ny, nx), noise, seed, offset=k * nx * ny)
    return Fields(rho, np.zeros((3, nz, ny, nx)), np.full((nz, ny, nx), T))


def droplet_2d(n, T, radius, width=4.0, noise=1e-3, seed=4) -> Fields:
    """Resting circular drop in a periodic n x n box (batched D2Q9 job)."""
    rv, rl = coexistence(T)
    y, x = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    s = radius - np.hypot(x - n / 2.0, y - n / 2.0)
    rho = _profile(s, rv, rl, width)[None]
    if noise:
        rho = rho + uniform_noise(rho.shape, noise, seed)
    return Fields(rho, np.zeros((2, 1, n, n)), np.full((1, n, n), T))


def droplet_or_slab_3d(n, T, kind, width=4.0, noise=1e-3, seed=5) -> Fields:
    """Cube of side n holding a centred drop (radius n/4) or a liquid slab
    (n/2 thick) in saturated vapour, periodic (served D3Q19 job)."""
    rv, rl = coexistence(T)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    c = n / 2.0
    if kind == "droplet":
        s = n / 4.0 - np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    else:
        x0 = n / 4.0 - 0.5
        s = np.minimum(x - x0, x0 + n / 2.0 - x)
    rho = _profile(s, rv, rl, width)
    if noise:
        rho = rho + uniform_noise(rho.shape, noise, seed)
    return Fields(rho, np.zeros((3, n, n, n)), np.full((n, n, n), T))


def uniform_gas(shape, rho, T, u=None) -> Fields:
    """Single-phase gas at rest (or moving at u)."""
    d = 2 if shape[0] == 1 else 3
    uu = np.zeros((d,) + tuple(shape))
    if u is not None:
        for a in range(d):
            uu[a] = u[a]
    return Fields(np.full(shape, float(rho)), uu, np.full(shape, float(T)))


def spinodal(shape, rho0=0.7, T0=0.8, noise=1e-3, seed=6) -> Fields:
    """Spinodal decomposition (Sec. 6.2, 6.3): a fluid at rest at uniform
    density rho0 inside the spinodal region and uniform T0, with seeded
    +-noise on the density that lets the unstable modes grow.  shape is
    (nz, ny, nx); nz = 1 for D2Q9, ny = nz = 1 for a row."""
    shape = tuple(shape)
    d = 2 if shape[0] == 1 else 3
    rho = np.full(shape, float(rho0)) + (uniform_noise(shape, noise, seed) if noise else 0.0)
    return Fields(rho, np.zeros((d,) + shape), np.full(shape, float(T0)))


# ---------------------------------------------------------------------------
# job lists

def batched_droplet_jobs(count=256, seed=4):
    """Domain list of the batched D2Q9 workload: square sides uniform in
    {64, 96, ..., 512}, T uniform in [0.7, 0.95], drop radius uniform in
    [8, side/4].  Returns a list of dicts (side, T, radius, seed)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(2, 17, size=count) * 32
    Ts = rng.uniform(0.7, 0.95, size=count)
    radii = np.array([rng.uniform(8.0, s / 4.0) for s in sides])
    return [{"side": int(s), "T": float(t), "radius": float(r), "seed": seed * 100003 + i}
            for i, (s, t, r) in enumerate(zip(sides, Ts, radii))]


def serving_trace(count=512, rate=200.0, seed=5, side_lo=32, side_hi=192, steps_lo=500, steps_hi=5000):
    """Poisson arrival trace of D3Q19 jobs: arrival time (s), cube side uniform
    in [side_lo, side_hi], requested steps uniform in [steps_lo, steps_hi],
    T uniform in [0.7, 0.9], droplet or slab with equal probability."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    steps = rng.integers(steps_lo, steps_hi + 1, size=count)
    Ts = rng.uniform(0.7, 0.9, size=count)
    kinds = np.where(rng.random(count) < 0.5, "droplet", "slab")
    return [{"arrival": float(a), "side": int(s), "steps": int(k), "T": float(tt), "kind": str(kd),
             "seed": seed * 100003 + i}
            for i, (a, s, k, tt, kd) in enumerate(zip(t, sides, steps, Ts, kinds))]
