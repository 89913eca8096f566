"""One domain over several processes: rank r holds slab r of the cut along
the last axis (``lbm_slab_plan``) and swaps halos with its neighbours through
``torch.distributed`` after every step.

The plan, the halo depth and the exchange are the library's (``lbm_slab_plan``
and the slab notes in include/lbm.h): the collision of a plane reads the
populations of the two planes beyond it on either side, so a slab with two
halo planes beyond each cut collides every plane it owns exactly and collides
only those.  After a step its edge planes have pushed the populations that
cross a cut into its halo planes; the swap moves them to the neighbour that
owns their plane (round 1), then refreshes the halo planes from the
neighbours' edge planes, which round 1 has completed (round 2).

``exchange_halos`` is the swap itself, written against callables that read
and write planes and crossing populations of a slab, so that it does not care
where they live.  ``SlabRank`` binds it to a library handle on this process's
GPU: NCCL moves the device buffers; a gloo group gets them staged through host
memory.  Only a process group is needed: the swap is point-to-point (no
collective on the data path).
"""
from __future__ import annotations

import numpy as np

from . import lbm

# tags of the messages a rank sends per step: crossing populations and edge
# planes travelling up and down (with two slabs of a periodic domain both
# directions go to the same peer)
TAG_CROSS_UP, TAG_CROSS_DOWN, TAG_UP, TAG_DOWN = 0, 1, 2, 3


def _swap(dist, group, sends, recvs):
    """Post every send with every receive in one batch (no pair of ranks can
    wait on each other) and wait for all of them."""
    ops = [dist.P2POp(dist.isend, t, peer, group, tag) for t, peer, tag in sends]
    ops += [dist.P2POp(dist.irecv, t, peer, group, tag) for t, peer, tag in recvs]
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def exchange_halos(dist, slab, get, put, get_cross, put_cross, group=None):
    """Refresh the halos of `slab` (an ``lbm_slab``; this rank holds slab
    index == rank) from its neighbours after a step.  ``get(first, count)``
    returns a contiguous tensor of the local planes [first, first + count),
    ``put(first, count, tensor)`` stores one; ``get_cross(plane, sign)`` and
    ``put_cross(plane, sign, tensor)`` do the same for the populations of
    one plane whose velocity has last-axis component ``sign``."""
    H = lbm.LBM_SLAB_HALO
    top, bottom = slab.lo + slab.own - 1, slab.lo      # edge planes
    # round 1: what the edge planes pushed into the halo planes goes to its owner
    sends, recvs, puts = [], [], []
    if slab.hi:
        sends.append((get_cross(top + 1, +1), slab.above, TAG_CROSS_UP))
    if slab.lo:
        sends.append((get_cross(bottom - 1, -1), slab.below, TAG_CROSS_DOWN))
    if slab.lo:
        buf = sends[-1][0].new_empty(sends[-1][0].shape)
        recvs.append((buf, slab.below, TAG_CROSS_UP))
        puts.append((bottom, +1, buf))
    if slab.hi:
        buf = sends[0][0].new_empty(sends[0][0].shape)
        recvs.append((buf, slab.above, TAG_CROSS_DOWN))
        puts.append((top, -1, buf))
    _swap(dist, group, sends, recvs)
    for plane, sign, buf in puts:
        put_cross(plane, sign, buf)
    # round 2: the halo planes from the neighbours' edge planes, now complete
    sends, recvs, puts = [], [], []
    if slab.hi:
        sends.append((get(top + 1 - H, H), slab.above, TAG_UP))
    if slab.lo:
        sends.append((get(bottom, H), slab.below, TAG_DOWN))
    if slab.lo:
        buf = sends[-1][0].new_empty(sends[-1][0].shape)
        recvs.append((buf, slab.below, TAG_UP))
        puts.append((0, buf))
    if slab.hi:
        buf = sends[0][0].new_empty(sends[0][0].shape)
        recvs.append((buf, slab.above, TAG_DOWN))
        puts.append((top + 1, buf))
    _swap(dist, group, sends, recvs)
    for first, buf in puts:
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
        if self.world > 1:   # halo planes are refreshed, not collided
            lbm.lbm_set_step_planes(self.h, self.slab.lo, self.slab.own)
        self.d = 2 if self.params.lattice == lbm.LBM_D2Q9 else 3
        self.nm = self.params.ny if self.params.lattice == lbm.LBM_D2Q9 else self.params.nz
        self.plane_bytes = lbm.lbm_plane_bytes(self.h)
        self.cross_bytes = lbm.lbm_crossing_bytes(self.h)
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

    def _get_cross(self, plane, sign):
        import torch
        buf = torch.empty(self.cross_bytes, dtype=torch.uint8, device=self.staging)
        lbm.lbm_get_crossing(self.h, plane, sign, buf)
        return buf

    def _put_cross(self, plane, sign, buf):
        lbm.lbm_set_crossing(self.h, plane, sign, buf)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            lbm.lbm_step(self.h, 1)
            exchange_halos(self.dist, self.slab, self._get, self._put, self._get_cross, self._put_cross,
                           self.group)

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
