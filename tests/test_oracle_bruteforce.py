"""The C oracle against an independent plain-Python statement of the step on
tiny grids (periodic, walls, heated walls, gravity, chi mode, switches off),
and the explicit-conduction stability threshold of Sec. 6.1.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from brute_force import Tiny

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

CASES = [
    # (Q, (nx, ny, nz), overrides)
    (9, (5, 4, 1), {}),
    (9, (4, 6, 1), {"wall": True, "T_fixed_lo": True, "T_lo": 0.9, "g": (0.0, -1e-3, 0.0)}),
    (9, (4, 5, 1), {"wall": True, "T_fixed_hi": True, "T_hi": 0.7, "chi_mode": True, "chi": 0.05,
                    "tau": 0.7, "tau_E": 0.6}),
    (9, (3, 4, 1), {"pseudoforce": False, "pressure_work": False, "barotropic": True, "T0": 0.85}),
    (19, (3, 4, 3), {}),
    (19, (3, 3, 5), {"wall": True, "T_fixed_lo": True, "T_lo": 0.95, "g": (0.0, 0.0, -1e-3), "tau": 0.8}),
    (19, (4, 3, 4), {"conduction": False, "A": 0.1, "g": (1e-3, 2e-3, 0.0)}),
]


def _fields(Q, dims, seed):
    from paper_1705_10045_gb300 import workloads as W
    rv, rl = W.coexistence(0.8)
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    d = 2 if Q == 9 else 3
    shape = (nz, ny, nx)
    rho = rng.uniform(rv, rl, size=shape)
    u = rng.uniform(-0.03, 0.03, size=(d,) + shape)
    T = rng.uniform(0.75, 0.85, size=shape)
    return rho, u, T


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_matches_plain_python_statement(case):
    Q, (nx, ny, nz), over = CASES[case]
    p = oracle.Params(Q=Q, nx=nx, ny=ny, nz=nz, **over)
    rho, u, T = _fields(Q, (nx, ny, nz), seed=case)
    d = p.d
    s = oracle.State(p, rho, u, p.c_v * T)

    prm = {k: getattr(p, k) for k in ("kappa", "A", "barotropic", "T0", "tau", "tau_E", "c_v", "chi_mode",
                                      "lam", "chi", "g", "wall", "T_fixed_lo", "T_fixed_hi", "T_lo", "T_hi",
                                      "pressure_work", "conduction", "pseudoforce")}
    dims = (nx, ny) if Q == 9 else (nx, ny, nz)

    def to_dict(a):
        a = a.reshape(nz, ny, nx)
        return {(x, y) if Q == 9 else (x, y, z): float(a[z, y, x])
                for z in range(nz) for y in range(ny) for x in range(nx)}

    tiny = Tiny(dims, prm, to_dict(rho), [to_dict(u[a]) for a in range(d)], to_dict(T))
    for _ in range(3):
        s.step(1)
        tiny.step()
        m = s.moments()
        ref = tiny.outputs()
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    key = (x, y) if Q == 9 else (x, y, z)
                    r = ref[key]
                    assert abs(m["rho"][z, y, x] - r["rho"]) < 1e-13
                    assert abs(m["T"][z, y, x] - r["T"]) < 1e-13
                    assert abs(m["P"][z, y, x] - r["P"]) < 1e-14
                    for a in range(d):
                        assert abs(m["u"][a, z, y, x] - r["u"][a]) < 1e-13


@pytest.mark.parametrize("chi,stable", [(0.49, True), (0.53, False)])
def test_explicit_conduction_stability_threshold(chi, stable):
    """Sec. 6.1: the explicit conduction scheme is stable for chi dt/h^2 < 0.5/d;
    a 1-D run with u = 0.1 at chi = 0.49 stays bounded, above 0.5 it blows up.
    tau_E is the paper's 0.503, where the scheme diffusion adds almost no
    damping of the shortest mode."""
    gold = GOLD["explicit_conduction"]
    nx = 64
    p = oracle.Params(Q=9, nx=nx, ny=1, barotropic=True, T0=0.8, chi_mode=True, chi=chi,
                      pressure_work=False, tau_E=GOLD["scheme_diffusion"]["tau_E"])
    rho0 = 0.1
    x = np.arange(nx)
    T = 0.8 + 0.01 * np.cos(2 * np.pi * x / nx) + 0.001 * np.cos(np.pi * x)  # includes the shortest mode
    u = np.zeros((2,) + p.shape)
    u[0] = gold["u"]
    s = oracle.State(p, np.full(p.shape, rho0), u, p.c_v * T.reshape(p.shape))
    with np.errstate(all="ignore"):
        s.step(3000)
        dev = np.nanmax(np.abs(s.moments()["T"] - 0.8)) if np.all(np.isfinite(s.N)) else np.inf
    if stable:
        assert dev < 0.011
    else:
        assert not dev < 1.0
