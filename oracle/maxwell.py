"""Maxwell equal-area construction for the reduced van der Waals equation of state.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3 compares the simulated phase densities with the coexistence curve given
by the Maxwell rule for p~ = 8 rho T/(3 - rho) - 3 rho^2 (critical point
rho = T = p = 1).  At coexistence the vapour (rho_v) and liquid (rho_l) share

  * the pressure:            p~(rho_v) = p~(rho_l) = p_s
  * the chemical potential:  integral_{v_l}^{v_v} p~ dv = p_s (v_v - v_l),  v = 1/rho

The integral of the vdW isotherm in specific volume has the closed form
    int p~ dv = (8T/3) ln(3v - 1) + 3/v.
The two conditions are solved by Newton iteration in float64 starting from
the spinodal bracket.  The result is independent of the lattice pressure scale.
"""
from __future__ import annotations

import math


def p_red(rho: float, T: float) -> float:
    return 8.0 * rho * T / (3.0 - rho) - 3.0 * rho * rho


def dp_drho(rho: float, T: float) -> float:
    return 24.0 * T / (3.0 - rho) ** 2 - 6.0 * rho


def _int_p_dv(v: float, T: float) -> float:
    # antiderivative of p~(v) = 8T/(3v - 1) - 3/v^2 in v
    return 8.0 * T / 3.0 * math.log(3.0 * v - 1.0) + 3.0 / v


def coexistence(T: float, tol: float = 1e-14) -> tuple[float, float, float]:
    """Return (rho_v, rho_l, p_s) on the Maxwell coexistence curve at 0.3 <= T < 1."""
    if not (0.3 <= T < 1.0):
        raise ValueError("T must lie in [0.3, 1)")
    # start from a symmetric guess around the critical density, then Newton
    # on the two equations in (v_l, v_v)
    eps = math.sqrt(max(1.0 - T, 1e-12))
    rl, rv = 1.0 + 2.0 * eps, max(1.0 - 2.0 * eps, 1e-3)
    if T < 0.85:
        # low temperature: better guesses from the ideal-gas/liquid limits
        rl = min(2.9, 1.0 + 2.0 * eps)
        rv = 0.5 * (1.0 - eps) ** 2
    vl, vv = 1.0 / rl, 1.0 / rv
    for _ in range(200):
        pl = 8.0 * T / (3.0 * vl - 1.0) - 3.0 / vl ** 2
        pv = 8.0 * T / (3.0 * vv - 1.0) - 3.0 / vv ** 2
        f1 = pl - pv
        f2 = (_int_p_dv(vv, T) - _int_p_dv(vl, T)) - 0.5 * (pl + pv) * (vv - vl)
        dpl = -24.0 * T / (3.0 * vl - 1.0) ** 2 + 6.0 / vl ** 3
        dpv = -24.0 * T / (3.0 * vv - 1.0) ** 2 + 6.0 / vv ** 3
        # partial derivatives of f2: d/dvl = -pl - 0.5 dpl (vv-vl) + 0.5 (pl+pv)
        j11, j12 = dpl, -dpv
        j21 = -pl - 0.5 * dpl * (vv - vl) + 0.5 * (pl + pv)
        j22 = pv - 0.5 * dpv * (vv - vl) - 0.5 * (pl + pv)
        det = j11 * j22 - j12 * j21
        dvl = (f1 * j22 - f2 * j12) / det
        dvv = (j11 * f2 - j21 * f1) / det
        # damp the step so that both volumes stay on their branches
        lam = 1.0
        while (vl - lam * dvl <= 1.0 / 3.0 + 1e-12 or vv - lam * dvv <= vl - lam * dvl) and lam > 1e-6:
            lam *= 0.5
        vl -= lam * dvl
        vv -= lam * dvv
        if abs(dvl) < tol * vl and abs(dvv) < tol * vv:
            break
    rl, rv = 1.0 / vl, 1.0 / vv
    return rv, rl, p_red(rl, T)


if __name__ == "__main__":
    for T in (0.7, 0.8, 0.85, 0.9, 0.95):
        print(T, coexistence(T))
