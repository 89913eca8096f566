"""Python binding of liblbm (include/lbm.h): argument marshalling only.

Every step of the lattice update runs in the CUDA library; this module loads
``_build/liblbm.so`` (built by ``paper_1705_10045_gb300.build``), mirrors the
C structures with ctypes and passes host numpy arrays or device torch
tensors by pointer.  There is no fallback: if the library is missing or no
GPU is present, the calls raise.

The functions carry the C names (``lbm_create``, ``lbm_init``, ...).  ``Lbm``
is a small convenience wrapper around one handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK = 0
LBM_ERR_INVALID_ARG = -1
LBM_ERR_UNSTABLE_PARAMS = -2
LBM_ERR_OOM = -3
LBM_ERR_CUDA = -4
LBM_ERR_NONPHYSICAL = -5
LBM_ERR_TIMEOUT = -6

LBM_D2Q9 = 9
LBM_D3Q19 = 19
LBM_STORE_FP64 = 0
LBM_STORE_FP32 = 1
LBM_STORE_FP16 = 2
LBM_MEM_HOST = 0
LBM_MEM_DEVICE = 1
LBM_STEP_FUSED = 0
LBM_STEP_THREE_LAUNCH = 1

EXPORTED = ("lbm_default_params", "lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_diagnostics",
            "lbm_state_bytes", "lbm_get_state", "lbm_set_state", "lbm_sync", "lbm_launches_per_step",
            "lbm_profile_step", "lbm_launch_name", "lbm_destroy", "lbm_last_error", "lbm_domain_bytes",
            "lbm_batch_create", "lbm_batch_add", "lbm_batch_remove", "lbm_batch_step", "lbm_batch_status",
            "lbm_batch_set_budget", "lbm_batch_domain", "lbm_batch_size", "lbm_batch_variants",
            "lbm_batch_variant_name", "lbm_batch_set_variant", "lbm_batch_tune", "lbm_batch_sync",
            "lbm_batch_destroy", "lbm_conservation_sums_noalloc", "lbm_coexistence", "lbm_slab_plan",
            "lbm_slabs_create", "lbm_slabs_count", "lbm_slabs_domain", "lbm_slabs_init", "lbm_slabs_step",
            "lbm_slabs_moments", "lbm_slabs_diagnostics", "lbm_slabs_sync", "lbm_slabs_destroy", "lbm_plane_bytes",
            "lbm_get_planes", "lbm_set_planes", "lbm_moments_f", "lbm_set_step_planes", "lbm_crossing_bytes",
            "lbm_get_crossing", "lbm_set_crossing", "lbm_step_begin", "lbm_step_end")
LBM_SLAB_HALO = 2


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("kappa", ctypes.c_double), ("A", ctypes.c_double), ("barotropic", ctypes.c_int), ("T0", ctypes.c_double),
        ("tau", ctypes.c_double), ("tau_E", ctypes.c_double), ("c_v", ctypes.c_double),
        ("chi_mode", ctypes.c_int), ("lambda_", ctypes.c_double), ("chi", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("wall", ctypes.c_int), ("T_fixed_lo", ctypes.c_int), ("T_fixed_hi", ctypes.c_int),
        ("T_lo", ctypes.c_double), ("T_hi", ctypes.c_double),
        ("wall_x", ctypes.c_int), ("wall_y", ctypes.c_int),
        ("T_fixed_x", ctypes.c_int * 2), ("T_fixed_y", ctypes.c_int * 2),
        ("T_x", ctypes.c_double * 2), ("T_y", ctypes.c_double * 2),
        ("pressure_work", ctypes.c_int), ("conduction", ctypes.c_int), ("pseudoforce", ctypes.c_int),
        ("latent", ctypes.c_double),
        ("storage", ctypes.c_int), ("rho_ref", ctypes.c_double), ("E_ref", ctypes.c_double),
        ("step_kernel", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("device", ctypes.c_int),
    ]


class lbm_slab(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int), ("own", ctypes.c_int), ("lo", ctypes.c_int), ("hi", ctypes.c_int),
                ("below", ctypes.c_int), ("above", ctypes.c_int), ("p", lbm_params)]


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbm.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1705_10045_gb300.build`")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    P = ctypes.POINTER(lbm_params)
    dp = ctypes.c_void_p   # host or device double*, passed as an address
    lib.lbm_default_params.argtypes = [P]
    lib.lbm_default_params.restype = None
    lib.lbm_create.argtypes = [P, ctypes.POINTER(H)]
    lib.lbm_init.argtypes = [H, dp, dp, dp, ctypes.c_int]
    lib.lbm_step.argtypes = [H, ctypes.c_int]
    lib.lbm_moments.argtypes = [H, dp, dp, dp, dp, ctypes.c_int]
    lib.lbm_moments_f.argtypes = [H, dp, dp, dp, dp, ctypes.c_int]
    lib.lbm_moments_f.restype = ctypes.c_int
    lib.lbm_diagnostics.argtypes = [H, ctypes.POINTER(ctypes.c_double)]
    lib.lbm_state_bytes.argtypes = [H]
    lib.lbm_state_bytes.restype = ctypes.c_size_t
    lib.lbm_get_state.argtypes = [H, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_set_state.argtypes = [H, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_sync.argtypes = [H]
    lib.lbm_launches_per_step.argtypes = [H]
    lib.lbm_profile_step.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.lbm_profile_step.restype = ctypes.c_int
    lib.lbm_launch_name.argtypes = [H, ctypes.c_int]
    lib.lbm_launch_name.restype = ctypes.c_char_p
    lib.lbm_destroy.argtypes = [H]
    lib.lbm_destroy.restype = None
    lib.lbm_conservation_sums_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.lbm_conservation_sums_noalloc.restype = ctypes.c_int
    lib.lbm_coexistence.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
    lib.lbm_coexistence.restype = ctypes.c_int
    lib.lbm_test_drop_handoff.argtypes = [H, ctypes.c_int]
    lib.lbm_test_drop_handoff.restype = ctypes.c_int
    lib.lbm_last_error.argtypes = []
    lib.lbm_last_error.restype = ctypes.c_char_p
    for name in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_diagnostics", "lbm_get_state",
                 "lbm_set_state", "lbm_sync", "lbm_launches_per_step"):
        getattr(lib, name).restype = ctypes.c_int
    B = ctypes.c_void_p
    LL = ctypes.c_longlong
    lib.lbm_domain_bytes.argtypes = [P]
    lib.lbm_domain_bytes.restype = ctypes.c_size_t
    lib.lbm_batch_create.argtypes = [P, ctypes.POINTER(B)]
    lib.lbm_batch_add.argtypes = [B, P, dp, dp, dp, ctypes.c_int, LL, ctypes.POINTER(ctypes.c_int)]
    lib.lbm_batch_remove.argtypes = [B, ctypes.c_int]
    lib.lbm_batch_step.argtypes = [B, ctypes.c_int]
    lib.lbm_batch_status.argtypes = [B, ctypes.c_int, ctypes.POINTER(LL), ctypes.POINTER(LL)]
    lib.lbm_batch_set_budget.argtypes = [B, ctypes.c_int, LL]
    lib.lbm_batch_domain.argtypes = [B, ctypes.c_int]
    lib.lbm_batch_domain.restype = H
    lib.lbm_batch_size.argtypes = [B]
    lib.lbm_batch_variants.argtypes = [B]
    lib.lbm_batch_variant_name.argtypes = [B, ctypes.c_int]
    lib.lbm_batch_variant_name.restype = ctypes.c_char_p
    lib.lbm_batch_set_variant.argtypes = [B, ctypes.c_int]
    lib.lbm_batch_tune.argtypes = [B, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.lbm_batch_sync.argtypes = [B]
    lib.lbm_batch_test_drop_item.argtypes = [B, ctypes.c_int]
    lib.lbm_batch_test_drop_item.restype = ctypes.c_int
    lib.lbm_batch_destroy.argtypes = [B]
    lib.lbm_batch_destroy.restype = None
    S = ctypes.c_void_p
    lib.lbm_slab_plan.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(lbm_slab)]
    lib.lbm_slabs_create.argtypes = [P, ctypes.c_int, ctypes.POINTER(S)]
    lib.lbm_slabs_count.argtypes = [S]
    lib.lbm_slabs_domain.argtypes = [S, ctypes.c_int]
    lib.lbm_slabs_domain.restype = H
    lib.lbm_slabs_init.argtypes = [S, dp, dp, dp, ctypes.c_int]
    lib.lbm_slabs_step.argtypes = [S, ctypes.c_int]
    lib.lbm_slabs_moments.argtypes = [S, dp, dp, dp, dp, ctypes.c_int]
    lib.lbm_slabs_diagnostics.argtypes = [S, ctypes.POINTER(ctypes.c_double)]
    lib.lbm_slabs_sync.argtypes = [S]
    lib.lbm_slabs_destroy.argtypes = [S]
    lib.lbm_slabs_destroy.restype = None
    lib.lbm_plane_bytes.argtypes = [H]
    lib.lbm_plane_bytes.restype = ctypes.c_size_t
    lib.lbm_get_planes.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_set_planes.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_set_step_planes.argtypes = [H, ctypes.c_int, ctypes.c_int]
    lib.lbm_step_begin.argtypes = [H, ctypes.c_int, ctypes.c_int]
    lib.lbm_step_end.argtypes = [H]
    lib.lbm_crossing_bytes.argtypes = [H]
    lib.lbm_crossing_bytes.restype = ctypes.c_size_t
    lib.lbm_get_crossing.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_set_crossing.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    for name in ("lbm_slab_plan", "lbm_slabs_create", "lbm_slabs_count", "lbm_slabs_init", "lbm_slabs_step",
                 "lbm_slabs_moments", "lbm_slabs_diagnostics", "lbm_slabs_sync", "lbm_get_planes",
                 "lbm_set_planes", "lbm_set_step_planes", "lbm_get_crossing", "lbm_set_crossing", "lbm_step_begin",
                 "lbm_step_end"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("lbm_batch_create", "lbm_batch_add", "lbm_batch_remove", "lbm_batch_step", "lbm_batch_status",
                 "lbm_batch_set_budget", "lbm_batch_size", "lbm_batch_variants", "lbm_batch_set_variant",
                 "lbm_batch_tune", "lbm_batch_sync"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_last_error().decode())
    return rc


def _addr(a):
    """(address, mem flag) of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float64")
        return a.ctypes.data, LBM_MEM_HOST
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), (LBM_MEM_DEVICE if a.is_cuda else LBM_MEM_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _byte_addr(buf):
    """(address, mem flag, bytes) of a contiguous uint8 numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.uint8 or not buf.flags.c_contiguous:
            raise TypeError("plane buffers must be C-contiguous uint8")
        return buf.ctypes.data, LBM_MEM_HOST, buf.nbytes
    import torch
    if isinstance(buf, torch.Tensor):
        if buf.dtype != torch.uint8 or not buf.is_contiguous():
            raise TypeError("plane buffers must be contiguous uint8")
        return buf.data_ptr(), (LBM_MEM_DEVICE if buf.is_cuda else LBM_MEM_HOST), buf.numel()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def lbm_default_params() -> lbm_params:
    p = lbm_params()
    load().lbm_default_params(ctypes.byref(p))
    return p


def make_params(**kw) -> lbm_params:
    """Default parameters with keyword overrides (``lambda_`` for lambda)."""
    p = lbm_default_params()
    for k, v in kw.items():
        if k == "lambda":
            k = "lambda_"
        if k == "gravity":
            p.gravity = (ctypes.c_double * 3)(*[float(x) for x in v])
        elif k in ("T_fixed_x", "T_fixed_y"):
            setattr(p, k, (ctypes.c_int * 2)(*[int(x) for x in v]))
        elif k in ("T_x", "T_y"):
            setattr(p, k, (ctypes.c_double * 2)(*[float(x) for x in v]))
        elif k == "stream":
            p.stream = ctypes.c_void_p(int(v) if v is not None else 0)
        else:
            if not hasattr(p, k):
                raise AttributeError(f"lbm_params has no field {k}")
            setattr(p, k, int(v) if isinstance(v, bool) else v)
    return p


def lbm_coexistence(T: float) -> tuple:
    """(rho_v, rho_l) on the Maxwell coexistence curve of the reduced vdW fluid."""
    rv, rl = ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_coexistence(float(T), ctypes.byref(rv), ctypes.byref(rl)))
    return rv.value, rl.value


def lbm_create(params: lbm_params):
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def lbm_init(h, rho, u, eps):
    (r, m1), (uu, m2), (e, m3) = _addr(rho), _addr(u), _addr(eps)
    if not (m1 == m2 == m3):
        raise ValueError("rho, u and eps must all live on the host or all on the device")
    return _check(load().lbm_init(h, r, uu, e, m1))


def lbm_step(h, n: int = 1):
    return _check(load().lbm_step(h, int(n)))


def lbm_moments(h, rho=None, u=None, T=None, P=None):
    addrs = [_addr(a) for a in (rho, u, T, P)]
    mems = {m for _, m in addrs if m is not None}
    if len(mems) > 1:
        raise ValueError("outputs must all live on the host or all on the device")
    mem = mems.pop() if mems else LBM_MEM_HOST
    return _check(load().lbm_moments(h, *[a for a, _ in addrs], mem))


def _addr_f32(a):
    """(address, mem flag) of a float32 numpy array or torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float32")
        return a.ctypes.data, LBM_MEM_HOST
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float32")
        return a.data_ptr(), (LBM_MEM_DEVICE if a.is_cuda else LBM_MEM_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def lbm_moments_f(h, rho=None, u=None, T=None, P=None):
    """FP32 twin of lbm_moments (float32 outputs, host or device)."""
    addrs = [_addr_f32(a) for a in (rho, u, T, P)]
    mems = {m for _, m in addrs if m is not None}
    if len(mems) > 1:
        raise ValueError("outputs must all live on the host or all on the device")
    mem = mems.pop() if mems else LBM_MEM_HOST
    return _check(load().lbm_moments_f(h, *[a for a, _ in addrs], mem))


def lbm_diagnostics(h) -> np.ndarray:
    out = (ctypes.c_double * 8)()
    rc = load().lbm_diagnostics(h, out)
    if rc not in (LBM_OK, LBM_ERR_NONPHYSICAL):
        _check(rc)
    return np.array(list(out))


def lbm_state_bytes(h) -> int:
    return int(load().lbm_state_bytes(h))


def lbm_get_state(h, buf=None) -> np.ndarray:
    if buf is None:
        buf = np.empty(lbm_state_bytes(h), dtype=np.uint8)
    _check(load().lbm_get_state(h, buf.ctypes.data, LBM_MEM_HOST))
    return buf


def lbm_set_state(h, buf: np.ndarray):
    return _check(load().lbm_set_state(h, buf.ctypes.data, LBM_MEM_HOST))


def lbm_sync(h):
    return _check(load().lbm_sync(h))


def lbm_launches_per_step(h) -> int:
    return int(load().lbm_launches_per_step(h))


def lbm_profile_step(h, n: int) -> dict:
    """Run n steps with events around every launch; {kernel name: mean ms}."""
    ms = (ctypes.c_double * 16)()
    r = load().lbm_profile_step(h, int(n), ms, 16)
    if r < 0:
        _check(r)
    return {load().lbm_launch_name(h, j).decode(): ms[j] for j in range(r)}


def lbm_launch_name(h, j: int) -> str:
    return load().lbm_launch_name(h, int(j)).decode()


def lbm_test_drop_handoff(h, plane: int):
    """Test hook: the first CTA of every fused step withholds the hand-off of
    `plane` (plane < 0: off), so that a bounded wait runs out."""
    _check(load().lbm_test_drop_handoff(h, int(plane)))


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


def lbm_conservation_sums_noalloc(lattice: int, storage: int, nx: int, ny: int, nz: int, rho_ref: float,
                                  E_ref: float, populations_ptr: int, sums_ptr: int, stream: int = 0):
    """Conservation sums of a caller-owned device population buffer, for callers
    that cannot allocate device memory (the library uses a static scratch
    array instead).  Pointers are device addresses; the call is asynchronous
    on `stream`."""
    return _check(load().lbm_conservation_sums_noalloc(int(lattice), int(storage), int(nx), int(ny), int(nz),
                                                       float(rho_ref), float(E_ref), ctypes.c_void_p(populations_ptr),
                                                       ctypes.c_void_p(sums_ptr), ctypes.c_void_p(stream)))


def lbm_slab_plan(params: lbm_params, count: int, i: int) -> lbm_slab:
    """Plan of slab i of `count` along the last axis (host only, no device)."""
    out = lbm_slab()
    _check(load().lbm_slab_plan(ctypes.byref(params), int(count), int(i), ctypes.byref(out)))
    return out


def lbm_plane_bytes(h) -> int:
    return int(load().lbm_plane_bytes(h))


def lbm_get_planes(h, first: int, count: int, buf):
    """Planes [first, first + count) of the populations into buf (Q rows of
    `count` planes of (N_k, g_k) pairs, storage format); device buffers are
    filled asynchronously on the handle's stream."""
    a, mem, n = _byte_addr(buf)
    if n < count * lbm_plane_bytes(h):
        raise ValueError("plane buffer too small")
    return _check(load().lbm_get_planes(h, int(first), int(count), a, mem))


def lbm_set_planes(h, first: int, count: int, buf):
    a, mem, n = _byte_addr(buf)
    if n < count * lbm_plane_bytes(h):
        raise ValueError("plane buffer too small")
    return _check(load().lbm_set_planes(h, int(first), int(count), a, mem))


def lbm_set_step_planes(h, first: int, count: int):
    """Collide only planes [first, first + count) of the last axis (0: all)."""
    return _check(load().lbm_set_step_planes(h, int(first), int(count)))


def lbm_step_begin(h, first: int, count: int):
    """Collide planes [first, first + count) of the last axis as part of the
    step the first call opens (its output becomes the current state)."""
    return _check(load().lbm_step_begin(h, int(first), int(count)))


def lbm_step_end(h):
    """Close the step lbm_step_begin opened."""
    return _check(load().lbm_step_end(h))


def lbm_crossing_bytes(h) -> int:
    return int(load().lbm_crossing_bytes(h))


def lbm_get_crossing(h, plane: int, sign: int, buf):
    """The pairs of plane `plane` for the directions whose last-axis velocity
    component is `sign` (+1 / -1) into buf (one row per direction)."""
    a, mem, n = _byte_addr(buf)
    if n < lbm_crossing_bytes(h):
        raise ValueError("crossing buffer too small")
    return _check(load().lbm_get_crossing(h, int(plane), int(sign), a, mem))


def lbm_set_crossing(h, plane: int, sign: int, buf):
    a, mem, n = _byte_addr(buf)
    if n < lbm_crossing_bytes(h):
        raise ValueError("crossing buffer too small")
    return _check(load().lbm_set_crossing(h, int(plane), int(sign), a, mem))


class Lbm:
    """One simulation domain on the GPU (owns a liblbm handle)."""

    def __init__(self, **kw):
        self.params = make_params(**kw)
        self.h = lbm_create(self.params)
        self.Q = self.params.lattice
        self.d = 2 if self.Q == LBM_D2Q9 else 3
        self.shape = (self.params.nz, self.params.ny, self.params.nx)

    def init(self, rho, u, eps):
        return lbm_init(self.h, rho, u, eps)

    def step(self, n: int = 1):
        return lbm_step(self.h, n)

    def moments(self) -> dict:
        """Host copies of rho, u* (d planes), T and P."""
        rho = np.empty(self.shape)
        u = np.empty((self.d,) + self.shape)
        T = np.empty(self.shape)
        P = np.empty(self.shape)
        lbm_moments(self.h, rho, u, T, P)
        return {"rho": rho, "u": u, "T": T, "P": P}

    def diagnostics(self) -> dict:
        o = lbm_diagnostics(self.h)
        return {"mass": o[0], "momentum": o[1:4], "energy": o[4], "clamps": int(o[5]), "bad": int(o[6]),
                "steps": int(o[7])}

    def get_state(self) -> np.ndarray:
        return lbm_get_state(self.h)

    def set_state(self, buf):
        return lbm_set_state(self.h, buf)

    def sync(self):
        return lbm_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slabs:
    """One domain as `count` slabs along its last axis on one GPU
    (lbm_slabs_*): same interface as Lbm, with the halo swap after every step."""

    def __init__(self, count: int, **kw):
        self.params = make_params(**kw)
        s = ctypes.c_void_p()
        _check(load().lbm_slabs_create(ctypes.byref(self.params), int(count), ctypes.byref(s)))
        self.s = s
        self.count = int(count)
        self.Q = self.params.lattice
        self.d = 2 if self.Q == LBM_D2Q9 else 3
        self.shape = (self.params.nz, self.params.ny, self.params.nx)

    def plan(self, i: int) -> lbm_slab:
        return lbm_slab_plan(self.params, self.count, i)

    def handle(self, i: int):
        h = load().lbm_slabs_domain(self.s, int(i))
        if not h:
            raise LbmError(LBM_ERR_INVALID_ARG, load().lbm_last_error().decode())
        return ctypes.c_void_p(h)

    def init(self, rho, u, eps):
        (r, m1), (uu, m2), (e, m3) = _addr(rho), _addr(u), _addr(eps)
        if not (m1 == m2 == m3):
            raise ValueError("rho, u and eps must all live on the host or all on the device")
        return _check(load().lbm_slabs_init(self.s, r, uu, e, m1))

    def step(self, n: int = 1):
        return _check(load().lbm_slabs_step(self.s, int(n)))

    def moments(self) -> dict:
        out = {"rho": np.empty(self.shape), "u": np.empty((self.d,) + self.shape), "T": np.empty(self.shape),
               "P": np.empty(self.shape)}
        _check(load().lbm_slabs_moments(self.s, out["rho"].ctypes.data, out["u"].ctypes.data,
                                        out["T"].ctypes.data, out["P"].ctypes.data, LBM_MEM_HOST))
        return out

    def diagnostics(self) -> dict:
        o = (ctypes.c_double * 8)()
        rc = load().lbm_slabs_diagnostics(self.s, o)
        if rc not in (LBM_OK, LBM_ERR_NONPHYSICAL):
            _check(rc)
        return {"mass": o[0], "momentum": np.array(o[1:4]), "energy": o[4], "clamps": int(o[5]),
                "bad": int(o[6]), "steps": int(o[7])}

    def sync(self):
        return _check(load().lbm_slabs_sync(self.s))

    def close(self):
        if getattr(self, "s", None):
            load().lbm_slabs_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_domain_bytes(params: lbm_params) -> int:
    return int(load().lbm_domain_bytes(ctypes.byref(params)))


class LbmBatch:
    """Many domains advanced together by one launch per step (lbm_batch_*)."""

    def __init__(self, **common):
        self.common = make_params(**common)
        b = ctypes.c_void_p()
        _check(load().lbm_batch_create(ctypes.byref(self.common), ctypes.byref(b)))
        self.b = b
        self.shapes = {}

    def add(self, rho, u, eps, steps: int, **kw) -> int:
        """Add a domain (keywords as for Lbm; lattice and storage default to the batch's)."""
        kw.setdefault("lattice", self.common.lattice)
        kw.setdefault("storage", self.common.storage)
        p = make_params(**kw)
        (r, m1), (uu, m2), (e, m3) = _addr(rho), _addr(u), _addr(eps)
        if not (m1 == m2 == m3):
            raise ValueError("rho, u and eps must all live on the host or all on the device")
        i = ctypes.c_int()
        _check(load().lbm_batch_add(self.b, ctypes.byref(p), r, uu, e, m1, int(steps), ctypes.byref(i)))
        self.shapes[i.value] = (p.nz, p.ny, p.nx)
        return i.value

    def remove(self, i: int):
        _check(load().lbm_batch_remove(self.b, int(i)))
        self.shapes.pop(i, None)

    def step(self, n: int):
        return _check(load().lbm_batch_step(self.b, int(n)))

    def status(self, i: int) -> tuple:
        done, left = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().lbm_batch_status(self.b, int(i), ctypes.byref(done), ctypes.byref(left)))
        return done.value, left.value

    def set_budget(self, i: int, steps: int):
        return _check(load().lbm_batch_set_budget(self.b, int(i), int(steps)))

    def handle(self, i: int):
        h = load().lbm_batch_domain(self.b, int(i))
        if not h:
            raise LbmError(LBM_ERR_INVALID_ARG, load().lbm_last_error().decode())
        return ctypes.c_void_p(h)

    def moments(self, i: int) -> dict:
        nz, ny, nx = self.shapes[i]
        d = 2 if self.common.lattice == LBM_D2Q9 else 3
        out = {"rho": np.empty((nz, ny, nx)), "u": np.empty((d, nz, ny, nx)), "T": np.empty((nz, ny, nx)),
               "P": np.empty((nz, ny, nx))}
        lbm_moments(self.handle(i), out["rho"], out["u"], out["T"], out["P"])
        return out

    def diagnostics(self, i: int) -> np.ndarray:
        return lbm_diagnostics(self.handle(i))

    def get_state(self, i: int) -> np.ndarray:
        return lbm_get_state(self.handle(i))

    def size(self) -> int:
        return int(load().lbm_batch_size(self.b))

    def variants(self) -> list:
        return [load().lbm_batch_variant_name(self.b, v).decode() for v in range(load().lbm_batch_variants(self.b))]

    def set_variant(self, v: int):
        return _check(load().lbm_batch_set_variant(self.b, int(v)))

    def tune(self, reps: int = 3) -> tuple:
        """Autotune the CTA shape; returns (best index, ms per launch of every shape)."""
        nv = load().lbm_batch_variants(self.b)
        ms = (ctypes.c_double * nv)()
        best = ctypes.c_int()
        _check(load().lbm_batch_tune(self.b, int(reps), ctypes.byref(best), ms))
        return best.value, list(ms)

    def sync(self):
        return _check(load().lbm_batch_sync(self.b))

    def close(self):
        if getattr(self, "b", None):
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
