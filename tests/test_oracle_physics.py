"""Physics pins of the FP64 oracle: results the paper fixes or that follow in
closed form from its equations.  CPU only; each runs in seconds.

  * Maxwell coexistence with A = -0.152 within the paper's 0.2 % (Sec. 3)
  * uniform temperature is kept exactly by the energy pseudoforce, and is
    lost without it (Sec. 4, Fig. of parasitic spreading)
  * Gaussian heat diffusion with D = theta (tau_E - 1/2) + lambda/(rho c_v),
    including the paper's D_E = 0.001 at tau_E = 0.503 (Sec. 6.1)
  * isothermal and adiabatic sound speeds from a standing wave (Sec. 6.2)
  * walls: mass conservation, rest state, steady conduction to a heated wall
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from oracle import maxwell
from paper_1705_10045_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ---------------------------------------------------------------------------
# the Maxwell solver itself, against an independent quadrature + root find

@pytest.mark.parametrize("T", [0.6, 0.8, 0.95])
def test_maxwell_solver_against_quadrature(T):
    rv, rl, ps = maxwell.coexistence(T)
    assert abs(maxwell.p_red(rv, T) - ps) < 1e-12 and abs(maxwell.p_red(rl, T) - ps) < 1e-12

    # independent: for trial p_s find the outer roots of p(v) = p_s with brentq,
    # integrate p dv numerically, and zero the equal-area residual in p_s
    def roots(p0):
        vs = np.linspace(1.0 / 3.0 + 1e-6, 50.0, 200001)
        pv = 8 * T / (3 * vs - 1) - 3 / vs ** 2 - p0
        idx = np.nonzero(np.sign(pv[:-1]) != np.sign(pv[1:]))[0]
        f = lambda v: 8 * T / (3 * v - 1) - 3 / v ** 2 - p0
        return optimize.brentq(f, vs[idx[0]], vs[idx[0] + 1], xtol=1e-15), \
            optimize.brentq(f, vs[idx[-1]], vs[idx[-1] + 1], xtol=1e-15)

    def area(p0):
        vl, vv = roots(p0)
        val, _ = integrate.quad(lambda v: 8 * T / (3 * v - 1) - 3 / v ** 2 - p0, vl, vv,
                                epsabs=1e-14, epsrel=1e-13, limit=200)
        return val

    p_ind = optimize.brentq(area, ps * 0.995, ps * 1.005, xtol=1e-15)
    vl, vv = roots(p_ind)
    assert abs(p_ind - ps) < 1e-9
    assert abs(1 / vl - rl) < 1e-8 and abs(1 / vv - rv) < 1e-8


def test_maxwell_definition_holds_on_the_whole_temperature_grid():
    """Equal pressure and equal chemical potential of the two phases, and
    both densities outside the spinodal region, at every point of the
    latent-heat table's grid (T = 0.5 + j/1024).  The chemical potential is
    written here from the vdW free energy per particle
    f = -(8T/3) ln(3/rho - 1) - 3 rho: mu = f + p/rho."""
    def mu(r, T):
        return -(8 * T / 3) * math.log((3 - r) / r) + 8 * T / (3 - r) - 6 * r

    for j in range(0, 512, 3):
        T = 0.5 + j / 1024
        rv, rl, ps = maxwell.coexistence(T)
        s_v, s_l = maxwell.spinodals(T)
        assert 0 < rv < s_v < 1.0 < s_l < rl < 3, T
        assert abs(maxwell.p_red(rv, T) - maxwell.p_red(rl, T)) < 1e-12, T
        assert abs(mu(rl, T) - mu(rv, T)) < 1e-11, T


def test_eos_stability_and_pseudopotential_sign_at_default_scale():
    """With the default lattice pressure scale the vdW isotherms used here
    satisfy the stability criterion of Sec. 3, (dp/drho)_T <= (h/dt)^2 + theta,
    and U = p - rho theta < 0 so that Phi = sqrt(-U) exists (Eq. (force))."""
    p = oracle.Params()
    lim = GOLD["eos_stability"]["dp_drho_max"]
    for T in np.linspace(0.6, 0.99, 14):
        rv, rl = W.coexistence(T)
        rho = np.linspace(0.005, rl * 1.05, 400)
        assert np.all(p.kappa * maxwell.dp_drho(rho, T) <= lim)
        assert all(oracle.pressure(oracle.Params(T0=T), r, T) - r / 3.0 < 0 for r in rho)


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("T", [0.7, 0.9])
def test_flat_interface_coexistence_matches_maxwell(T):
    """Sec. 3: with A = -0.152 the simulated phase densities of the vdW fluid
    differ from the Maxwell rule by less than 0.2 %.  1-D slab (D2Q9, ny = 1),
    barotropic EOS at T so that only the density field evolves."""
    gold = GOLD["vdw_mixing"]
    p = oracle.Params(Q=9, nx=512, ny=1, barotropic=True, T0=T, A=gold["A"])
    f = W.flat_slab_2d(nx=512, ny=1, T=T, slab=256)
    s = oracle.State(p, f.rho, f.u, p.c_v * f.T)
    s.step(30000)
    m = s.moments()
    rho = m["rho"].ravel()
    rv, rl, _ = maxwell.coexistence(T)
    assert m["clamps"] == 0
    assert abs(rho.max() / rl - 1) < gold["max_relative_density_deviation"]
    assert abs(rho.min() / rv - 1) < gold["max_relative_density_deviation"]
    # the wrong mixing parameter misses the same bound (sensitivity of the pin)
    q = oracle.Params(Q=9, nx=512, ny=1, barotropic=True, T0=T, A=0.2)
    s2 = oracle.State(q, f.rho, f.u, q.c_v * f.T).step(30000)
    assert abs(s2.moments()["rho"].min() / rv - 1) > 5 * gold["max_relative_density_deviation"]


@pytest.mark.parametrize("Q,shape", [(9, (1, 1, 128)), (19, (1, 4, 64))])
def test_pseudoforce_keeps_uniform_temperature(Q, shape):
    """Sec. 4: with E = rho c_v T and the energy pseudoforce, a two-phase
    fluid at uniform T (tau_E = tau, no pressure work) keeps T uniform to
    rounding: g_k stays c_v T N_k.  Without the pseudoforce energy leaks
    from the liquid to the vapour and T develops peaks and dips."""
    T0 = 0.8
    f = W.flat_slab_2d(nx=shape[2], ny=shape[1] * shape[0], T=T0, slab=shape[2] // 2)
    rho = f.rho.reshape(shape)
    d = 2 if Q == 9 else 3
    u = np.zeros((d,) + shape)
    for pf, check in ((True, lambda dev: dev < 1e-13), (False, lambda dev: dev > 1e-4)):
        p = oracle.Params(Q=Q, nx=shape[2], ny=shape[1], nz=shape[0], tau=0.8, tau_E=0.8,
                          pressure_work=False, conduction=True, pseudoforce=pf)
        s = oracle.State(p, rho, u, p.c_v * np.full(shape, T0))
        s.step(400)
        dev = np.abs(s.moments()["T"] - T0).max()
        assert check(dev), (pf, dev)


def _gaussian_width2(profile):
    x = np.arange(profile.size, dtype=float)
    w = profile / profile.sum()
    mu = (w * x).sum()
    return (w * (x - mu) ** 2).sum()


@pytest.mark.parametrize("tau_E,lam", [(0.503, 0.0), (1.0, 0.0), (0.8, 0.05), (0.51, 0.06)])
def test_gaussian_heat_diffusion(tau_E, lam):
    """Resting uniform gas (barotropic EOS, so no flow), Gaussian temperature
    bump: the energy spreads with D = theta (tau_E - 1/2) (scheme diffusion,
    Sec. 6.1) + lambda/(rho c_v) (conduction, Sec. 4), so sigma^2 grows by
    2 D t.  At tau_E = 0.503, lambda = 0 this is the paper's D_E = 0.001."""
    rho0, T0, nx = 0.1, 0.8, 256
    p = oracle.Params(Q=9, nx=nx, ny=1, barotropic=True, T0=T0, tau_E=tau_E, lam=lam,
                      pressure_work=False)
    x = np.arange(nx, dtype=float)
    s0 = 8.0
    T = T0 + 0.05 * np.exp(-(x - nx / 2) ** 2 / (2 * s0 ** 2))
    s = oracle.State(p, np.full(p.shape, rho0), np.zeros((2,) + p.shape), p.c_v * T.reshape(p.shape))
    E0 = rho0 * p.c_v * T0

    def width2():
        return _gaussian_width2(s.moments()["T"].ravel() * rho0 * p.c_v - E0)

    # the BGK random walk starts with a transient (the velocity
    # autocorrelation (1 - 1/tau_E)^n): measure the slope after it
    D = (tau_E - 0.5) / 3.0 + lam / (rho0 * p.c_v)
    s.step(400)
    w0 = width2()
    t = int(round(min(4000, 60.0 / D)))
    s.step(t)
    D_meas = (width2() - w0) / (2 * t)
    assert abs(D_meas / D - 1) < 0.02, (D_meas, D)
    if tau_E == GOLD["scheme_diffusion"]["tau_E"] and lam == 0:
        assert abs(D_meas - GOLD["scheme_diffusion"]["D_E"]) < 2e-5


def _standing_wave_c2(p, rho0, T0, L, amp=1e-4, periods=2.0, c2_guess=None):
    """Squared sound speed from the frequency of a standing wave of wavelength L."""
    x = np.arange(L, dtype=float)
    mode = np.cos(2 * np.pi * x / L)
    rho = rho0 * (1 + amp * mode)
    s = oracle.State(p, rho.reshape(p.shape), np.zeros((2,) + p.shape), p.c_v * np.full(p.shape, T0))
    k = 2 * np.pi / L
    period = 2 * np.pi / (k * math.sqrt(c2_guess))
    nsteps = int(periods * period)
    a = np.empty(nsteps)
    for i in range(nsteps):
        a[i] = (s.moments()["rho"].ravel() - rho0) @ mode
        s.step(1)
    # A density bump at uniform T is a sound wave plus a non-propagating
    # entropy mode (when pressure work is on); fit a damped cosine plus a
    # slowly decaying offset and take w_0^2 = w^2 + g^2.
    t = np.arange(nsteps, dtype=float)
    fit = lambda t, a0, g, w, ph, b, beta: a0 * np.exp(-g * t) * np.cos(w * t + ph) + b * np.exp(-beta * t)
    popt, _ = optimize.curve_fit(fit, t, a, p0=[a[0], 1e-4, 2 * np.pi / period, 0.0, 0.0, 1e-4])
    w = abs(popt[2])
    return (w * w + popt[1] ** 2) / (k * k)


def test_sound_speed_isothermal_and_adiabatic():
    """Sec. 6.2: without pressure work the sound is isothermal,
    c_T^2 = kappa (dp~/drho)_T; with it the sound is adiabatic.  For the
    model E = rho c_v T the adiabatic value is
    c_S^2 = c_T^2 + kappa (dp~/dT)_rho p/(rho^2 c_v), which grows linearly
    in 1/c_v (the paper's Eq. (sspeed) with gamma = C_P/C_V)."""
    g = GOLD["sound_speed"]
    rho0, T0, L = g["rho"], g["T"], 128
    kappa = 0.01
    cT2 = kappa * maxwell.dp_drho(rho0, T0)
    p_iso = oracle.Params(Q=9, nx=L, ny=1, kappa=kappa, pressure_work=False, conduction=False)
    c2 = _standing_wave_c2(p_iso, rho0, T0, L, c2_guess=cT2)
    assert abs(c2 / cT2 - 1) < 0.01, (c2, cT2)
    excess = []
    for c_v in (0.02, 0.05, 0.1):
        p = oracle.Params(Q=9, nx=L, ny=1, kappa=kappa, c_v=c_v, tau_E=0.51, pressure_work=True,
                          conduction=False)
        pr = kappa * maxwell.p_red(rho0, T0)
        cS2 = cT2 + kappa * 8 * rho0 / (3 - rho0) * pr / (rho0 ** 2 * c_v)
        c2 = _standing_wave_c2(p, rho0, T0, L, c2_guess=cS2)
        assert abs(c2 / cS2 - 1) < 0.01, (c_v, c2, cS2)
        excess.append((c2 - cT2) * c_v)
    # linear in 1/c_v: (c_S^2 - c_T^2) c_v is the same for every c_v
    assert max(excess) / min(excess) - 1 < 0.06


# ---------------------------------------------------------------------------
# walls (not in the paper: halfway bounce-back and a fixed-temperature wall)

def test_walls_conserve_mass_and_keep_rest_state():
    p = oracle.Params(Q=19, nx=6, ny=5, nz=8, wall=True, T_fixed_lo=False)
    shape = p.shape
    s = oracle.State(p, np.full(shape, 0.2), np.zeros((3,) + shape), p.c_v * np.full(shape, 0.8))
    s.step(50)
    m = s.moments()
    np.testing.assert_allclose(m["rho"], 0.2, rtol=1e-14)
    np.testing.assert_allclose(m["u"], 0, atol=1e-16)
    np.testing.assert_allclose(m["T"], 0.8, rtol=1e-14)
    # two-phase content under gravity: mass exact, energy bounded
    f = W.pool_boiling_3d(nx=6, ny=5, nz=16, depth=6, noise=1e-3, seed=3)
    q = oracle.Params(Q=19, nx=6, ny=5, nz=16, wall=True, g=(0, 0, -1e-4))
    s = oracle.State(q, f.rho, f.u, q.c_v * f.T)
    m0 = s.N.sum()
    s.step(100)
    assert abs(s.N.sum() - m0) < 1e-12 * m0
    assert s.clamps == 0


@pytest.mark.parametrize("Q", [9, 19])
def test_heated_wall_steady_conduction(Q):
    """Single-phase gas between a wall held at T_w (bottom) and an adiabatic
    wall (top): the steady state is uniform T = T_w; with both walls fixed
    at different T it is the linear profile between the wall values.  Only
    the finite-difference conduction sees the wall temperature (the energy
    populations bounce back), so tau_E is kept near 1/2 where the scheme
    diffusion, which carries no heat through a wall, is small."""
    n = 24
    if Q == 9:
        p = oracle.Params(Q=9, nx=4, ny=n, wall=True, barotropic=True, T0=0.8, lam=0.02,
                          tau_E=0.51, T_fixed_lo=True, T_lo=0.85, pressure_work=False)
    else:
        p = oracle.Params(Q=19, nx=3, ny=3, nz=n, wall=True, barotropic=True, T0=0.8, lam=0.02,
                          tau_E=0.51, T_fixed_lo=True, T_lo=0.85, pressure_work=False)
    rho0 = 0.1
    s = oracle.State(p, np.full(p.shape, rho0), np.zeros((p.d,) + p.shape), p.c_v * np.full(p.shape, 0.8))
    s.step(20000)
    T = s.moments()["T"]
    np.testing.assert_allclose(T, 0.85, atol=2e-4)
    # two fixed walls: linear profile through the wall values at z = -1/2 and n - 1/2
    p.T_fixed_hi, p.T_hi = True, 0.75
    s = oracle.State(p, np.full(p.shape, rho0), np.zeros((p.d,) + p.shape), p.c_v * np.full(p.shape, 0.8))
    s.step(20000)
    T = s.moments()["T"]
    prof = T.reshape(n, -1).mean(1) if Q == 19 else T[0].mean(1)
    z = np.arange(n) + 0.5
    want = 0.85 + (0.75 - 0.85) * z / n
    np.testing.assert_allclose(prof, want, atol=3e-4)


def test_laplace_law_pressure_jump_scales_as_one_over_radius():
    """Resting drops of radius 24 and 32 (128x128, T = 0.7, barotropic): the
    bulk pressure jump times R is the same within 5 % (Laplace law).  The
    paper prints no surface tension, so its absolute value is unpinned."""
    n, prods = 128, []
    for R in (24.0, 32.0):
        f = W.moving_droplet_2d(n=n, T=0.7, radius=R, ux=0.0, noise=0.0, hot_dT=0.0)
        p = oracle.Params(Q=9, nx=n, ny=n, barotropic=True, T0=0.7, lam=0.02)
        s = oracle.State(p, f.rho, f.u, p.c_v * f.T).step(4000)
        P = s.moments()["P"].reshape(n, n)
        dP = P[n // 2, n // 2] - P[0, 0]
        assert dP > 0
        prods.append(dP * R)
    assert max(prods) / min(prods) - 1 < 0.05, prods
