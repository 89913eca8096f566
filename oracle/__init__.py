"""FP64 CPU oracle of the thermal multiphase lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports it and shares no code
with it.

The arithmetic lives in plain C (``lbm_oracle.c``, built with
``-O2 -ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with ``ctypes`` and numpy arrays.  ``maxwell.py`` holds the
equal-area construction of the reduced van der Waals equation of state.

Array conventions (same as the C file): scalar fields have shape
``(nz, ny, nx)`` (``nz = 1`` for D2Q9), vector fields ``(d, nz, ny, nx)``,
population sets ``(Q, nz, ny, nx)``; all float64, C-contiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("Q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("kappa", ctypes.c_double), ("A", ctypes.c_double),
        ("barotropic", ctypes.c_int), ("T0", ctypes.c_double),
        ("tau", ctypes.c_double), ("tau_E", ctypes.c_double), ("c_v", ctypes.c_double),
        ("chi_mode", ctypes.c_int), ("lam", ctypes.c_double), ("chi", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("wall", ctypes.c_int), ("T_fixed_lo", ctypes.c_int), ("T_fixed_hi", ctypes.c_int),
        ("T_lo", ctypes.c_double), ("T_hi", ctypes.c_double),
        ("wall_x", ctypes.c_int), ("wall_y", ctypes.c_int),
        ("T_fixed_x", ctypes.c_int * 2), ("T_fixed_y", ctypes.c_int * 2),
        ("T_x", ctypes.c_double * 2), ("T_y", ctypes.c_double * 2),
        ("pressure_work", ctypes.c_int), ("conduction", ctypes.c_int), ("pseudoforce", ctypes.c_int),
        ("latent", ctypes.c_double), ("coex", ctypes.POINTER(ctypes.c_double)),
    ]


@dataclass
class Params:
    """Parameters of one simulation (lattice units h = dt = 1)."""
    Q: int = 9
    nx: int = 64
    ny: int = 64
    nz: int = 1
    kappa: float = 0.01
    A: float = -0.152
    barotropic: bool = False
    T0: float = 0.8
    tau: float = 1.0
    tau_E: float = 1.0
    c_v: float = 1.5
    chi_mode: bool = False
    lam: float = 0.05
    chi: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)
    wall: bool = False
    T_fixed_lo: bool = False
    T_fixed_hi: bool = False
    T_lo: float = 0.0
    T_hi: float = 0.0
    wall_x: bool = False          # bounce-back walls at both ends of x
    wall_y: bool = False          # ... of y (D3Q19; for D2Q9 y is the last axis, `wall`)
    T_fixed_x: tuple = (False, False)   # per x wall (low, high end): held at T_x[i]
    T_fixed_y: tuple = (False, False)
    T_x: tuple = (0.0, 0.0)
    T_y: tuple = (0.0, 0.0)
    pressure_work: bool = True
    conduction: bool = True
    pseudoforce: bool = True
    latent: float = 0.0      # rho_liq Q of Sec. 5; 0 switches the latent heat off

    @property
    def d(self) -> int:
        return 2 if self.Q == 9 else 3

    @property
    def shape(self) -> tuple:
        return (self.nz, self.ny, self.nx)

    def to_c(self) -> _Params:
        if self.Q == 9 and self.wall_y:
            raise ValueError("D2Q9: y is the last axis; its walls are `wall`")
        c = _Params()
        for name, _ in _Params._fields_:
            if name == "g":
                c.g = (ctypes.c_double * 3)(*[float(v) for v in self.g])
            elif name in ("T_fixed_x", "T_fixed_y"):
                setattr(c, name, (ctypes.c_int * 2)(*[int(v) for v in getattr(self, name)]))
            elif name in ("T_x", "T_y"):
                setattr(c, name, (ctypes.c_double * 2)(*[float(v) for v in getattr(self, name)]))
            elif name == "coex":
                c.coex = _ptr(coexistence_table())
            else:
                setattr(c, name, type(getattr(c, name))(getattr(self, name)))
        return c


_COEX = None


def coexistence_table() -> np.ndarray:
    """Maxwell densities on the grid T_j = 0.5 + j/1024, j = 0..512, as one
    array [rho_v(T_0..T_512), rho_l(T_0..T_512)] (the table the C oracle
    interpolates in for the latent-heat source of Sec. 5)."""
    global _COEX
    if _COEX is None:
        from . import maxwell
        n = 512
        tab = np.ones(2 * (n + 1))
        for j in range(n):
            rv, rl, _ = maxwell.coexistence(0.5 + j / 1024.0)
            tab[j], tab[n + 1 + j] = rv, rl
        _COEX = tab
    return _COEX


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        _lib.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        _lib.orc_feq.restype = None
        _lib.orc_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp,
                                     ctypes.POINTER(ctypes.c_int), dp]
        _lib.orc_pressure.argtypes = [pp, ctypes.c_double, ctypes.c_double]
        _lib.orc_pressure.restype = ctypes.c_double
        _lib.orc_macros.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_macros.restype = ctypes.c_long
        _lib.orc_force.argtypes = [pp, dp, dp, dp]
        _lib.orc_force.restype = None
        _lib.orc_energy_source.argtypes = [pp, dp, dp, dp, dp, dp]
        _lib.orc_energy_source.restype = None
        _lib.orc_step.argtypes = [pp, dp, dp, ctypes.c_int]
        _lib.orc_step.restype = ctypes.c_long
        _lib.orc_init.argtypes = [pp, dp, dp, dp, dp, dp]
        _lib.orc_init.restype = None
        _lib.orc_moments.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        _lib.orc_moments.restype = ctypes.c_long
        _lib.orc_sources.argtypes = [pp, dp, dp, dp, dp]
        _lib.orc_sources.restype = ctypes.c_long
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def feq(Q: int, rho: float, u) -> np.ndarray:
    """Equilibrium populations of one node, Eq. (feq)."""
    out = np.zeros(Q)
    uu = np.zeros(3)
    uu[: len(u)] = u
    lib().orc_feq(Q, float(rho), _ptr(uu), _ptr(out))
    return out


def lattice(Q: int) -> dict:
    """Velocity set, weights, force-stencil coefficients, opposites and alpha."""
    c = (ctypes.c_int * (3 * Q))()
    w = np.zeros(Q)
    G = np.zeros(Q)
    opp = (ctypes.c_int * Q)()
    alpha = ctypes.c_double()
    if lib().orc_lattice(Q, c, _ptr(w), _ptr(G), opp, ctypes.byref(alpha)) != 0:
        raise ValueError(f"unknown lattice Q={Q}")
    return {"c": np.array(list(c), dtype=np.int64).reshape(Q, 3), "w": w, "G": G,
            "opp": np.array(list(opp)), "alpha": alpha.value}


def pressure(p: Params, rho: float, T: float) -> float:
    cp = p.to_c()
    return lib().orc_pressure(ctypes.byref(cp), float(rho), float(T))


class State:
    """Population sets N and g of one domain, advanced by the oracle."""

    def __init__(self, p: Params, rho, u, eps):
        self.p = p
        self._cp = p.to_c()
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(p.shape)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape((p.d,) + p.shape)
        eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(p.shape)
        self.N = np.zeros((p.Q,) + p.shape)
        self.g = np.zeros((p.Q,) + p.shape)
        lib().orc_init(ctypes.byref(self._cp), _ptr(rho), _ptr(u), _ptr(eps), _ptr(self.N), _ptr(self.g))
        self.clamps = 0

    @classmethod
    def from_populations(cls, p: Params, N, g):
        s = cls.__new__(cls)
        s.p = p
        s._cp = p.to_c()
        s.N = np.ascontiguousarray(N, dtype=np.float64).reshape((p.Q,) + p.shape).copy()
        s.g = np.ascontiguousarray(g, dtype=np.float64).reshape((p.Q,) + p.shape).copy()
        s.clamps = 0
        return s

    def step(self, n: int = 1) -> "State":
        r = lib().orc_step(ctypes.byref(self._cp), _ptr(self.N), _ptr(self.g), int(n))
        if r < 0:
            raise MemoryError("oracle scratch allocation failed")
        self.clamps += r
        return self

    def moments(self) -> dict:
        """rho, u* (physical velocity), T and P of the current state."""
        p = self.p
        rho = np.zeros(p.shape)
        us = np.zeros((p.d,) + p.shape)
        T = np.zeros(p.shape)
        P = np.zeros(p.shape)
        r = lib().orc_moments(ctypes.byref(self._cp), _ptr(self.N), _ptr(self.g),
                              _ptr(rho), _ptr(us), _ptr(T), _ptr(P))
        if r < 0:
            raise MemoryError("oracle scratch allocation failed")
        return {"rho": rho, "u": us, "T": T, "P": P, "clamps": r}

    def fields(self) -> dict:
        """Pre-collision fields of the current state: rho, u (lattice velocity,
        Eq. (hydro)), E, T, P, Phi, plus du and dE of the next step."""
        p = self.p
        rho = np.zeros(p.shape)
        u = np.zeros((p.d,) + p.shape)
        E = np.zeros(p.shape)
        T = np.zeros(p.shape)
        P = np.zeros(p.shape)
        Phi = np.zeros(p.shape)
        clamps = lib().orc_macros(ctypes.byref(self._cp), _ptr(self.N), _ptr(self.g), _ptr(rho), _ptr(u),
                                  _ptr(E), _ptr(T), _ptr(P), _ptr(Phi))
        du = np.zeros((p.d,) + p.shape)
        dE = np.zeros(p.shape)
        lib().orc_sources(ctypes.byref(self._cp), _ptr(self.N), _ptr(self.g), _ptr(du), _ptr(dE))
        return {"rho": rho, "u": u, "E": E, "T": T, "P": P, "Phi": Phi, "du": du, "dE": dE,
                "clamps": clamps}


def force(p: Params, Phi, rho) -> np.ndarray:
    """Interparticle force plus gravity for given Phi and rho fields (Sec. 3)."""
    cp = p.to_c()
    Phi = np.ascontiguousarray(Phi, dtype=np.float64).reshape(p.shape)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(p.shape)
    F = np.zeros((p.d,) + p.shape)
    lib().orc_force(ctypes.byref(cp), _ptr(Phi), _ptr(rho), _ptr(F))
    return F


def energy_source(p: Params, rho, ustar, T, P) -> np.ndarray:
    """Finite-difference energy change of one step (Sec. 4) for given fields."""
    cp = p.to_c()
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ustar, T, P)]
    dE = np.zeros(p.shape)
    lib().orc_energy_source(ctypes.byref(cp), *[_ptr(a) for a in arrs], _ptr(dE))
    return dE
