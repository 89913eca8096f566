"""Pins of the oracle's walls on every axis (the paper runs periodic domains
only; the walls, their halfway bounce-back and the ghost values of the
stencils are the reading the walls on the last axis already follow, applied
to each axis).

* Rotation: the lattice update does not know which axis is which, so a
  domain with walls on x (or y) must evolve as the same domain rotated so
  that those walls lie on the last axis, up to the order in which the
  populations are summed (the velocity ordering is not rotation-invariant):
  1e-12.  This ties the x and y walls, their ghosts and their wall
  temperatures to the last-axis walls, which are pinned separately.
* A closed box (walls on every axis) conserves mass exactly and keeps a rest
  state at rest.
* Steady conduction along x between a held and an adiabatic wall: uniform
  wall temperature.
"""
import numpy as np
import pytest

import oracle
from paper_1705_10045_gb300 import workloads as W

STEPS = 60


def _moments(p, f, steps=STEPS):
    s = oracle.State(p, f.rho, f.u, p.c_v * f.T).step(steps)
    assert s.clamps == 0
    return s.moments()


def _pool(nx, ny, nz, seed=3):
    return W.pool_boiling_3d(nx=nx, ny=ny, nz=nz, T=0.8, depth=nz // 3, noise=1e-3, seed=seed)


def _rot(a, perm):
    """Scalar field (nz, ny, nx) under the axis permutation perm (new array axes)."""
    return np.ascontiguousarray(np.transpose(a, perm))


def _rot_fields(f, perm, comp):
    rho = _rot(f.rho, perm)
    u = np.stack([_rot(f.u[c], perm) for c in comp])
    T = _rot(f.T, perm)
    return W.Fields(rho, u, T)


# D3Q19 axis permutations: (array transpose, velocity components of the new x, y, z)
TO_X = ((2, 1, 0), (2, 1, 0))   # walls of z become walls of x: x' = z, z' = x
TO_Y = ((1, 0, 2), (0, 2, 1))   # walls of z become walls of y: y' = z, z' = y


@pytest.mark.parametrize("target", ["x", "y"])
def test_d3q19_walls_on_x_or_y_equal_rotated_last_axis_walls(target):
    nx, ny, nz = 6, 5, 10
    f = _pool(nx, ny, nz)
    g = (0.0, 0.0, -1e-4)
    base = oracle.Params(Q=19, nx=nx, ny=ny, nz=nz, wall=True, T_fixed_lo=True, T_lo=0.95,
                         T_fixed_hi=True, T_hi=0.7, g=g)
    m0 = _moments(base, f)
    perm, comp = TO_X if target == "x" else TO_Y
    fr = _rot_fields(f, perm, comp)
    shape = fr.rho.shape
    gr = tuple(g[c] for c in comp)
    if target == "x":
        p = oracle.Params(Q=19, nx=shape[2], ny=shape[1], nz=shape[0], wall_x=True, T_fixed_x=(True, True),
                          T_x=(0.95, 0.7), g=gr)
    else:
        p = oracle.Params(Q=19, nx=shape[2], ny=shape[1], nz=shape[0], wall_y=True, T_fixed_y=(True, True),
                          T_y=(0.95, 0.7), g=gr)
    m1 = _moments(p, fr)
    np.testing.assert_allclose(m1["rho"], _rot(m0["rho"], perm), rtol=0, atol=1e-12)
    np.testing.assert_allclose(m1["T"], _rot(m0["T"], perm), rtol=0, atol=1e-12)
    for a, c in enumerate(comp):
        np.testing.assert_allclose(m1["u"][a], _rot(m0["u"][c], perm), rtol=0, atol=1e-12)
    # the walls matter: the same rotated box without them evolves differently
    q = oracle.Params(Q=19, nx=shape[2], ny=shape[1], nz=shape[0], g=gr)
    assert np.max(np.abs(_moments(q, fr)["T"] - m1["T"])) > 1e-3


def test_d3q19_walls_on_x_and_z_equal_walls_on_y_and_z_swapped():
    nx, ny, nz = 6, 7, 8
    f = _pool(nx, ny, nz, seed=5)
    p = oracle.Params(Q=19, nx=nx, ny=ny, nz=nz, wall=True, wall_x=True, T_fixed_lo=True, T_lo=0.9,
                      T_fixed_x=(False, True), T_x=(0.0, 0.75), g=(-2e-5, 0.0, -1e-4))
    m0 = _moments(p, f)
    perm, comp = (0, 2, 1), (1, 0, 2)          # swap x and y
    fr = _rot_fields(f, perm, comp)
    q = oracle.Params(Q=19, nx=ny, ny=nx, nz=nz, wall=True, wall_y=True, T_fixed_lo=True, T_lo=0.9,
                      T_fixed_y=(False, True), T_y=(0.0, 0.75), g=(0.0, -2e-5, -1e-4))
    m1 = _moments(q, fr)
    np.testing.assert_allclose(m1["rho"], _rot(m0["rho"], perm), rtol=0, atol=1e-12)
    np.testing.assert_allclose(m1["T"], _rot(m0["T"], perm), rtol=0, atol=1e-12)
    for a, c in enumerate(comp):
        np.testing.assert_allclose(m1["u"][a], _rot(m0["u"][c], perm), rtol=0, atol=1e-12)


def test_d2q9_walls_on_x_equal_transposed_walls_on_y():
    f = W.flat_slab_2d(nx=12, ny=16, T=0.8, slab=6, noise=1e-3)
    # the slab lies across x; transposed it lies across y
    base = oracle.Params(Q=9, nx=12, ny=16, wall=True, T_fixed_hi=True, T_hi=0.85, g=(0.0, -1e-4, 0.0))
    m0 = _moments(base, f)
    perm, comp = (0, 2, 1), (1, 0)
    fr = _rot_fields(f, perm, comp)
    p = oracle.Params(Q=9, nx=16, ny=12, wall_x=True, T_fixed_x=(False, True), T_x=(0.0, 0.85),
                      g=(-1e-4, 0.0, 0.0))
    m1 = _moments(p, fr)
    np.testing.assert_allclose(m1["rho"], _rot(m0["rho"], perm), rtol=0, atol=1e-12)
    np.testing.assert_allclose(m1["T"], _rot(m0["T"], perm), rtol=0, atol=1e-12)
    for a, c in enumerate(comp):
        np.testing.assert_allclose(m1["u"][a], _rot(m0["u"][c], perm), rtol=0, atol=1e-12)


def test_closed_box_conserves_mass_and_keeps_rest():
    p = oracle.Params(Q=19, nx=5, ny=6, nz=7, wall=True, wall_x=True, wall_y=True)
    shape = p.shape
    s = oracle.State(p, np.full(shape, 0.2), np.zeros((3,) + shape), p.c_v * np.full(shape, 0.8)).step(40)
    m = s.moments()
    np.testing.assert_allclose(m["rho"], 0.2, rtol=1e-14)
    np.testing.assert_allclose(m["u"], 0, atol=1e-16)
    np.testing.assert_allclose(m["T"], 0.8, rtol=1e-14)
    f = _pool(8, 7, 12, seed=8)
    q = oracle.Params(Q=19, nx=8, ny=7, nz=12, wall=True, wall_x=True, wall_y=True, g=(1e-5, -2e-5, -1e-4))
    s = oracle.State(q, f.rho, f.u, q.c_v * f.T)
    m0 = s.N.sum()
    s.step(100)
    assert abs(s.N.sum() - m0) < 1e-12 * m0
    assert s.clamps == 0


@pytest.mark.parametrize("Q", [9, 19])
def test_steady_conduction_along_x(Q):
    """Single-phase gas between a held low x wall and an adiabatic high one:
    uniform T = T_w at steady state (tau_E near 1/2, as for the last axis)."""
    n = 24
    kw = dict(barotropic=True, T0=0.8, lam=0.02, tau_E=0.51, pressure_work=False, wall_x=True,
              T_fixed_x=(True, False), T_x=(0.85, 0.0))
    p = oracle.Params(Q=9, nx=n, ny=3, **kw) if Q == 9 else oracle.Params(Q=19, nx=n, ny=3, nz=3, **kw)
    s = oracle.State(p, np.full(p.shape, 0.1), np.zeros((p.d,) + p.shape), p.c_v * np.full(p.shape, 0.8))
    s.step(20000)
    np.testing.assert_allclose(s.moments()["T"], 0.85, atol=2e-4)


def test_d2q9_has_no_separate_y_wall_flag():
    with pytest.raises(ValueError):
        oracle.Params(Q=9, nx=8, ny=8, wall_y=True).to_c()
