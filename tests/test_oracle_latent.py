"""Pins of the oracle's latent-heat source (Sec. 5): inside the transition
layer rho_v(T) < rho < rho_l(T) the energy changes by
    dE = -(rho_liq Q) rho div(u*) / (rho_l - rho_v)
per step.  CPU only.

The closed form used here: on a periodic row with uniform rho and T and
u*_x = u0 sin(k x), the centred difference of the divergence is exactly
u0 sin(k) cos(k x) (a trigonometric identity), and rho_v, rho_l come from the
Maxwell construction solved at T itself, not from the oracle's table.  The
table's linear interpolation on a grid of spacing h = 1/1024 errs by at most
h^2/8 max|(rho_l - rho_v)''| over the interval, which sets the tolerance
(the second derivative taken by finite differences of the exact curve).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import maxwell

L = 0.02          # rho_liq Q, the value of the paper's 2-D spinodal run (Sec. 6.3)


def _interp_tol(T):
    """Relative bound of the table's interpolation error of rho_l - rho_v at T."""
    h = 1.0 / 1024

    def width(t):
        rv, rl, _ = maxwell.coexistence(t)
        return rl - rv

    d2 = max(abs(width(t + h) - 2 * width(t) + width(t - h)) / h ** 2 for t in (T - h, T, T + h))
    return 2.0 * h ** 2 / 8 * d2 / width(T) + 1e-12


def _row(n, rho0, T0, u0, latent=L, pressure_work=False, conduction=False):
    p = oracle.Params(Q=9, nx=n, ny=1, latent=latent, pressure_work=pressure_work, conduction=conduction)
    x = np.arange(n)
    k = 2 * math.pi / n
    rho = np.full(p.shape, rho0)
    T = np.full(p.shape, T0)
    us = np.zeros((2,) + p.shape)
    us[0, 0, 0, :] = u0 * np.sin(k * x)
    P = np.array([[[oracle.pressure(p, rho0, T0)] * n]])
    return p, rho, us, T, P, k, x


@pytest.mark.parametrize("rho0,T0", [(1.0, 0.8), (0.5, 0.75), (1.5, 0.9), (0.3, 0.71)])
def test_latent_source_matches_closed_form(rho0, T0):
    n, u0 = 64, 0.01
    p, rho, us, T, P, k, x = _row(n, rho0, T0, u0)
    rv, rl, _ = maxwell.coexistence(T0)
    assert rv < rho0 < rl
    dE = oracle.energy_source(p, rho, us, T, P)[0, 0]
    expect = -L * rho0 * u0 * math.sin(k) * np.cos(k * x) / (rl - rv)
    assert np.max(np.abs(dE - expect)) <= _interp_tol(T0) * np.max(np.abs(expect))
    # converging flow (div u* < 0) condenses vapour and releases heat
    conv = np.cos(k * x) < -0.5
    assert np.all(dE[conv] > 0)


def test_latent_source_adds_to_pressure_work():
    n, u0, rho0, T0 = 48, 0.02, 1.0, 0.8
    p, rho, us, T, P, k, x = _row(n, rho0, T0, u0, pressure_work=True)
    rv, rl, _ = maxwell.coexistence(T0)
    div = u0 * math.sin(k) * np.cos(k * x)
    dE = oracle.energy_source(p, rho, us, T, P)[0, 0]
    # the vdW pressure written out (kappa = 0.01), not the oracle's routine
    Pv = 0.01 * (8 * rho0 * T0 / (3 - rho0) - 3 * rho0 ** 2)
    expect = -Pv * div - L * rho0 * div / (rl - rv)
    assert np.max(np.abs(dE - expect)) <= _interp_tol(T0) * np.max(np.abs(expect))


@pytest.mark.parametrize("rho0,T0", [(0.1, 0.8), (2.0, 0.8), (1.0, 1.05), (0.15, 0.8)])
def test_no_latent_heat_outside_the_transition_layer(rho0, T0):
    p, rho, us, T, P, k, x = _row(32, rho0, T0, 0.01)
    dE = oracle.energy_source(p, rho, us, T, P)
    assert np.all(dE == 0.0)


def test_band_follows_the_local_temperature():
    # rho = 0.15 lies inside the band at T = 0.7 (rho_v = 0.128) but below it
    # at T = 0.8 (rho_v = 0.240): only the cold half of the row gets heat
    n = 32
    p, rho, us, T, P, k, x = _row(n, 0.15, 0.8, 0.01)
    T[0, 0, : n // 2] = 0.7
    dE = oracle.energy_source(p, rho, us, T, P)[0, 0]
    assert np.all(dE[n // 2:] == 0.0)
    assert np.count_nonzero(dE[: n // 2]) >= n // 2 - 2


def test_latent_heat_switch_off_gives_no_source():
    p, rho, us, T, P, k, x = _row(32, 1.0, 0.8, 0.01, latent=0.0)
    assert np.all(oracle.energy_source(p, rho, us, T, P) == 0.0)


def test_step_energy_change_equals_latent_source():
    """Over one full step with pressure work and conduction off, the total
    energy changes by exactly the summed source (the g collision conserves
    the rest), so the source reaches the populations with its sign."""
    n = 64
    p = oracle.Params(Q=9, nx=n, ny=8, latent=L, pressure_work=False, conduction=False)
    x = np.arange(n)
    rho = np.ones(p.shape) * (1.0 + 0.05 * np.sin(2 * math.pi * x / n))
    u = np.zeros((2,) + p.shape)
    u[0] = 0.02 * np.sin(2 * math.pi * x / n + 0.3)
    T = np.full(p.shape, 0.8)
    s = oracle.State(p, rho, u, p.c_v * T)
    f = s.fields()
    E0 = f["E"].sum()
    src = f["dE"].sum()
    assert abs(src) > 1e-6
    s.step(1)
    E1 = s.g.sum()
    assert abs((E1 - E0) - src) <= 1e-12 * abs(E0)
    p0 = oracle.Params(Q=9, nx=n, ny=8, latent=0.0, pressure_work=False, conduction=False)
    s0 = oracle.State(p0, rho, u, p0.c_v * T)
    s0.step(1)
    assert abs(s0.g.sum() - E0) <= 1e-12 * abs(E0)
