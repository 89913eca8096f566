"""Shared helpers of the GPU tests: run the same seeded inputs through the CUDA
library (via its C-ABI binding) and through the FP64 oracle."""
import numpy as np

import oracle
from paper_1705_10045_gb300 import lbm

ORACLE_KEYS = ("Q", "nx", "ny", "nz", "kappa", "A", "barotropic", "T0", "tau", "tau_E", "c_v", "chi_mode",
               "chi", "wall", "T_fixed_lo", "T_fixed_hi", "T_lo", "T_hi", "pressure_work", "conduction",
               "pseudoforce")


def oracle_params(**kw) -> oracle.Params:
    """Oracle parameters from the same keywords the GPU run takes."""
    kw = dict(kw)
    if "lattice" in kw:
        kw["Q"] = kw.pop("lattice")
    if "lambda_" in kw:
        kw["lam"] = kw.pop("lambda_")
    if "gravity" in kw:
        kw["g"] = tuple(kw.pop("gravity"))
    for k in ("storage", "rho_ref", "E_ref", "stream", "device"):
        kw.pop(k, None)
    return oracle.Params(**kw)


def gpu_params(**kw) -> dict:
    kw = dict(kw)
    if "lam" in kw:
        kw["lambda_"] = kw.pop("lam")
    if "g" in kw:
        kw["gravity"] = kw.pop("g")
    if "Q" in kw:
        kw["lattice"] = kw.pop("Q")
    return kw


def run_gpu(fields, steps, **kw) -> dict:
    sim = lbm.Lbm(**gpu_params(**kw))
    try:
        c_v = sim.params.c_v
        sim.init(np.ascontiguousarray(fields.rho), np.ascontiguousarray(fields.u[: sim.d]),
                 np.ascontiguousarray(c_v * fields.T))
        sim.step(steps)
        out = sim.moments()
        out["diag"] = sim.diagnostics()
        return out
    finally:
        sim.close()


def run_oracle(fields, steps, **kw) -> dict:
    p = oracle_params(**kw)
    s = oracle.State(p, fields.rho, fields.u[: p.d], p.c_v * fields.T)
    s.step(steps)
    out = s.moments()
    out["state"] = s
    return out


def max_abs(a, b) -> float:
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
