"""Maxwell equal-area construction for the reduced van der Waals equation of state.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3 compares the simulated phase densities with the coexistence curve given
by the Maxwell rule for p~ = 8 rho T/(3 - rho) - 3 rho^2 (critical point
rho = T = p = 1).  At coexistence the vapour (rho_v) and liquid (rho_l) share

  * the pressure:            p~(rho_v) = p~(rho_l) = p_s
  * the chemical potential:  integral_{v_l}^{v_v} p~ dv = p_s (v_v - v_l),  v = 1/rho

The integral of the vdW isotherm in specific volume has the closed form
    int p~ dv = (8T/3) ln(3v - 1) + 3/v.
The saturation pressure is found by bracketed root finding between the two
spinodal pressures (where dp/drho = 0), with the vapour and liquid volumes
bracketed on their own branches, so the trivial solution v_l = v_v of the
two conditions cannot be reached.  The result is independent of the lattice
pressure scale.
"""
from __future__ import annotations

import math

from scipy import optimize


def p_red(rho: float, T: float) -> float:
    return 8.0 * rho * T / (3.0 - rho) - 3.0 * rho * rho


def dp_drho(rho: float, T: float) -> float:
    return 24.0 * T / (3.0 - rho) ** 2 - 6.0 * rho


def _int_p_dv(v: float, T: float) -> float:
    # antiderivative of p~(v) = 8T/(3v - 1) - 3/v^2 in v
    return 8.0 * T / 3.0 * math.log(3.0 * v - 1.0) + 3.0 / v


def spinodals(T: float) -> tuple[float, float]:
    """Densities where dp/drho = 0 on the isotherm T < 1 (vapour, liquid):
    24T/(3 - rho)^2 = 6 rho, i.e. rho (3 - rho)^2 = 4T."""
    f = lambda r: r * (3.0 - r) ** 2 - 4.0 * T
    return optimize.brentq(f, 0.0, 1.0, xtol=1e-15), optimize.brentq(f, 1.0, 3.0, xtol=1e-15)


def _branches(ps: float, T: float, s_v: float, s_l: float) -> tuple[float, float]:
    """Vapour and liquid volumes where p~ = ps (outside the spinodal region)."""
    g = lambda r: p_red(r, T) - ps
    rv = optimize.brentq(g, 0.0, s_v, xtol=1e-16, rtol=1e-15)
    rl = optimize.brentq(g, s_l, 3.0 - 1e-12, xtol=1e-16, rtol=1e-15)
    return 1.0 / rv, 1.0 / rl


def coexistence(T: float) -> tuple[float, float, float]:
    """Return (rho_v, rho_l, p_s) on the Maxwell coexistence curve at 0.3 <= T < 1.

    The saturation pressure p_s is the root, between the two spinodal
    pressures, of the equal-area residual
        integral_{v_l}^{v_v} p~ dv - p_s (v_v - v_l),
    where v_v, v_l are the outer roots of p~(v) = p_s; each root is bracketed."""
    if not (0.3 <= T < 1.0):
        raise ValueError("T must lie in [0.3, 1)")
    s_v, s_l = spinodals(T)
    hi = p_red(s_v, T)
    lo = max(p_red(s_l, T), 1e-10 * hi)

    def area(ps):
        vv, vl = _branches(ps, T, s_v, s_l)
        return (_int_p_dv(vv, T) - _int_p_dv(vl, T)) - ps * (vv - vl)

    ps = optimize.brentq(area, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    vv, vl = _branches(ps, T, s_v, s_l)
    return 1.0 / vv, 1.0 / vl, ps


if __name__ == "__main__":
    for T in (0.7, 0.8, 0.85, 0.9, 0.95):
        print(T, coexistence(T))
