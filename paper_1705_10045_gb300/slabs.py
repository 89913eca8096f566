"""One domain over several processes: rank r holds slab r of the cut along
the last axis (``lbm_slab_plan``) and swaps halo planes with its neighbours
through ``torch.distributed`` after every step.

The plan, the halo depth and the reason three planes suffice are the
library's (``lbm_slab_plan`` in include/lbm.h): a step moves information two
planes for the force and finite-difference stencils plus one for streaming,
so a slab whose three halo planes beyond each cut are refreshed after every
step computes every plane it owns exactly as the undivided domain would.

``exchange_halos`` is the swap itself, written against two callables that
read and write planes of a slab, so that it does not care where the planes
live.  ``SlabRank`` binds it to a library handle on this process's GPU: NCCL
moves the device buffers; a gloo group gets them staged through host memory.  Only a process group is needed: the swap is
point-to-point (no collective on the data path).
"""
from __future__ import annotations

import numpy as np

from . import lbm

# tags of the two messages a rank sends per step: its top owned planes
# travelling up and its bottom owned planes travelling down (with two slabs of
# a periodic domain both go to the same peer)
TAG_UP, TAG_DOWN = 0, 1


def exchange_halos(dist, slab, get, put, group=None):
    """Refresh the halo planes of `slab` (an ``lbm_slab``; this rank holds
    slab index == rank) from its neighbours.  ``get(first, count)`` returns a
    contiguous tensor of the local planes [first, first + count);
    ``put(first, count, tensor)`` stores one.  Sends are posted with the
    receives in one batch, so no pair of ranks can wait on each other."""
    H = lbm.LBM_SLAB_HALO
    ops, recvs = [], []
    up = get(slab.lo + slab.own - H, H) if slab.hi else None
    down = get(slab.lo, H) if slab.lo else None
    if up is not None:
        ops.append(dist.P2POp(dist.isend, up, slab.above, group, TAG_UP))
    if down is not None:
        ops.append(dist.P2POp(dist.isend, down, slab.below, group, TAG_DOWN))
    if down is not None:
        buf = down.new_empty(down.shape)
        ops.append(dist.P2POp(dist.irecv, buf, slab.below, group, TAG_UP))
        recvs.append((0, buf))
    if up is not None:
        buf = up.new_empty(up.shape)
        ops.append(dist.P2POp(dist.irecv, buf, slab.above, group, TAG_DOWN))
        recvs.append((slab.lo + slab.own, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for first, buf in recvs:
        put(first, H, buf)


def local_planes(field: np.ndarray, slab, axis: int, nm: int) -> np.ndarray:
    """The slab's local planes (halos included) of a whole-domain field along
    `axis`, wrapping around a periodic last axis."""
    idx = (np.arange(slab.lo + slab.own + slab.hi) + slab.first - slab.lo) % nm
    return np.ascontiguousarray(np.take(field, idx, axis=axis))


class SlabRank:
    """Slab ``rank`` of ``world`` of one domain on this process's GPU."""

    def __init__(self, dist, group=None, **kw):
        import torch
        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        # the plane copies are enqueued on the handle's stream and the sends,
        # receives and buffer lifetimes are ordered on torch's current stream:
        # the two must be the same stream
        current = torch.cuda.current_stream().cuda_stream
        if kw.get("stream") not in (None, current):
            raise ValueError("SlabRank runs on torch's current stream; make the intended stream current instead")
        kw["stream"] = current
        self.params = lbm.make_params(**kw)
        self.slab = lbm.lbm_slab_plan(self.params, self.world, self.rank)
        self.h = lbm.lbm_create(self.slab.p)
        self.d = 2 if self.params.lattice == lbm.LBM_D2Q9 else 3
        self.nm = self.params.ny if self.params.lattice == lbm.LBM_D2Q9 else self.params.nz
        self.plane_bytes = lbm.lbm_plane_bytes(self.h)
        self.device = torch.device("cuda", torch.cuda.current_device())
        # gloo moves host tensors only: stage the planes through host memory
        self.staging = torch.device("cpu") if dist.get_backend(group) == "gloo" else self.device

    def init(self, rho, u, eps):
        """Whole-domain host fields (the same arrays on every rank)."""
        p, sl = self.slab.p, self.slab
        shape = (p.nz, p.ny, p.nx)
        whole = (self.params.nz, self.params.ny, self.params.nx)
        ax = 0 if self.d == 3 else 1
        r = local_planes(np.asarray(rho, dtype=np.float64).reshape(whole), sl, ax, self.nm).reshape(shape)
        uu = local_planes(np.asarray(u, dtype=np.float64).reshape((self.d,) + whole), sl, ax + 1, self.nm)
        e = local_planes(np.asarray(eps, dtype=np.float64).reshape(whole), sl, ax, self.nm).reshape(shape)
        return lbm.lbm_init(self.h, r, uu, e)

    def _get(self, first, count):
        import torch
        buf = torch.empty(count * self.plane_bytes, dtype=torch.uint8, device=self.staging)
        lbm.lbm_get_planes(self.h, first, count, buf)
        return buf

    def _put(self, first, count, buf):
        lbm.lbm_set_planes(self.h, first, count, buf)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            lbm.lbm_step(self.h, 1)
            exchange_halos(self.dist, self.slab, self._get, self._put, self.group)

    def moments(self) -> dict:
        """rho, u*, T, P of the planes this rank owns (host arrays)."""
        p, sl = self.slab.p, self.slab
        shape = (p.nz, p.ny, p.nx)
        out = {"rho": np.empty(shape), "u": np.empty((self.d,) + shape), "T": np.empty(shape),
               "P": np.empty(shape)}
        lbm.lbm_moments(self.h, out["rho"], out["u"], out["T"], out["P"])
        ax = 0 if self.d == 3 else 1
        own = slice(sl.lo, sl.lo + sl.own)
        return {k: v[(slice(None),) * (ax + (k == "u")) + (own,)] for k, v in out.items()}

    def close(self):
        if getattr(self, "h", None):
            lbm.lbm_destroy(self.h)
            self.h = None
