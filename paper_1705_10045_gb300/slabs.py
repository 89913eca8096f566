"""One domain over several processes: rank r holds slab r of the cut along
the last axis (``lbm_slab_plan``) and swaps halos with its neighbours through
``torch.distributed`` after every step.

The plan and the halo depth are the library's (``lbm_slab_plan`` and the slab
notes in include/lbm.h): the collision of a plane reads the populations of the
two planes beyond it on either side, so a slab with two halo planes beyond
each cut collides every plane it owns exactly and collides only those.  After
a step its edge planes have pushed the populations that cross a cut into its
halo planes.  The swap is one message per neighbour and direction: the
crossing populations a slab pushed into its halo plane next to the cut, and
its two edge planes.  The receiver

1. writes the neighbour's edge planes into its halo planes;
2. puts back, into the halo plane next to the cut, the crossing populations
   it pushed there itself (the neighbour's copy of that plane lacks exactly
   those; across a wall on x or y the wall column keeps the neighbour's value,
   which ``lbm_set_crossing`` does);
3. completes its own edge plane with the neighbour's crossing populations.

Everything a rank sends comes from the planes next to its cuts, so
``SlabRank`` steps those first (``lbm_step_begin``), posts the swap, steps
its interior while the messages travel, and then applies what it received.

``post_halos`` / ``finish_halos`` (and ``exchange_halos``, both in one call)
are written against callables that read and write planes and crossing
populations of a slab, so that they do not care where those live.
``SlabRank`` binds them to a library handle on this process's GPU: NCCL
moves the device buffers; a gloo group gets them staged through host memory.
Only a process group is needed: the swap is point-to-point (no collective on
the data path).
"""
from __future__ import annotations

import numpy as np

from . import lbm

# tags of the messages a rank sends per step, travelling up and down (with two
# slabs of a periodic domain both directions go to the same peer)
TAG_UP, TAG_DOWN = 2, 3
# planes next to a cut stepped before the interior: the two edge planes the
# swap sends take pushes from up to two planes beyond the cut
EDGE_PLANES = 3


def _pack(cross, planes):
    import torch
    return torch.cat([cross.reshape(-1), planes.reshape(-1)])


def _unpack(buf, like_cross, like_planes):
    n = like_cross.numel()
    return buf[:n].reshape(like_cross.shape), buf[n:].reshape(like_planes.shape)


def post_halos(dist, slab, get, get_cross, group=None):
    """Read what this rank sends (``get(first, count)``: a contiguous tensor
    of local planes [first, first + count); ``get_cross(plane, sign)``: the
    populations of one plane whose velocity has last-axis component sign) and
    post the sends and receives of one swap.  Returns the pending swap for
    ``finish_halos``."""
    H = lbm.LBM_SLAB_HALO
    top, bottom = slab.lo + slab.own - 1, slab.lo      # edge planes
    sends, recvs, todo = [], [], []
    if slab.hi:   # up: my pushes into halo plane top + 1, my top edge planes
        cross, planes = get_cross(top + 1, +1), get(top + 1 - H, H)
        msg = _pack(cross, planes)
        sends.append((msg, slab.above, TAG_UP))
        buf = msg.new_empty(msg.shape)
        recvs.append((buf, slab.above, TAG_DOWN))
        todo.append(("up", buf, cross, planes))
    if slab.lo:   # down: my pushes into halo plane bottom - 1, my bottom edge planes
        cross, planes = get_cross(bottom - 1, -1), get(bottom, H)
        msg = _pack(cross, planes)
        sends.append((msg, slab.below, TAG_DOWN))
        buf = msg.new_empty(msg.shape)
        recvs.append((buf, slab.below, TAG_UP))
        todo.append(("down", buf, cross, planes))
    ops = [dist.P2POp(dist.isend, t, peer, group, tag) for t, peer, tag in sends]
    ops += [dist.P2POp(dist.irecv, t, peer, group, tag) for t, peer, tag in recvs]
    reqs = dist.batch_isend_irecv(ops) if ops else []
    return reqs, todo, sends


def finish_halos(slab, pending, put, put_cross):
    """Wait for the swap ``post_halos`` started and apply it
    (``put(first, count, tensor)``, ``put_cross(plane, sign, tensor)``)."""
    H = lbm.LBM_SLAB_HALO
    reqs, todo, _ = pending
    for req in reqs:
        req.wait()
    top, bottom = slab.lo + slab.own - 1, slab.lo
    for side, buf, mine, like_planes in todo:
        theirs, planes = _unpack(buf, mine, like_planes)
        if side == "up":
            put(top + 1, H, planes)        # the neighbour's lower edge planes
            put_cross(top + 1, +1, mine)   # with my own pushes across the cut
            put_cross(top, -1, theirs)     # its pushes complete my top plane
        else:
            put(0, H, planes)
            put_cross(bottom - 1, -1, mine)
            put_cross(bottom, +1, theirs)


def exchange_halos(dist, slab, get, put, get_cross, put_cross, group=None):
    """Refresh the halos of `slab` (an ``lbm_slab``; this rank holds slab
    index == rank) from its neighbours after a step: ``post_halos`` and
    ``finish_halos`` in one call."""
    finish_halos(slab, post_halos(dist, slab, get, get_cross, group), put, put_cross)


def split_ranges(slab, edge: int = EDGE_PLANES):
    """(planes next to the cuts, interior planes) of the planes `slab` owns,
    as lists of (first, count) local plane ranges: `edge` planes beside each
    cut (a slab ending at a wall has no cut there), the rest in one range.
    A slab too thin to split steps all its owned planes in the first list."""
    sl, E = slab, edge
    if sl.own < 2 * E:
        return [(sl.lo, sl.own)], []
    edges = ([(sl.lo, E)] if sl.lo else []) + ([(sl.lo + sl.own - E, E)] if sl.hi else [])
    lo, hi = sl.lo + (E if sl.lo else 0), sl.lo + sl.own - (E if sl.hi else 0)
    return edges, ([(lo, hi - lo)] if hi > lo else [])


def local_planes(field: np.ndarray, slab, axis: int, nm: int) -> np.ndarray:
    """The slab's local planes (halos included) of a whole-domain field along
    `axis`, wrapping around a periodic last axis."""
    idx = (np.arange(slab.lo + slab.own + slab.hi) + slab.first - slab.lo) % nm
    return np.ascontiguousarray(np.take(field, idx, axis=axis))


class SlabRank:
    """Slab ``rank`` of ``world`` of one domain on this process's GPU."""

    def __init__(self, dist, group=None, overlap: bool = True, **kw):
        import torch
        self.dist, self.group, self.overlap = dist, group, overlap
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

    def _ranges(self):
        return split_ranges(self.slab)

    def step(self, n: int = 1):
        """n steps, each: the planes next to the cuts, the swap posted, the
        interior planes while it travels, the swap applied (``overlap``);
        otherwise, and with the three-launch step form, a whole step and
        then the swap."""
        if self.world == 1:
            lbm.lbm_step(self.h, int(n))
            return
        if not self.overlap or self.params.step_kernel == lbm.LBM_STEP_THREE_LAUNCH:
            for _ in range(int(n)):
                lbm.lbm_step(self.h, 1)
                exchange_halos(self.dist, self.slab, self._get, self._put, self._get_cross, self._put_cross,
                               self.group)
            return
        edges, interior = self._ranges()
        for _ in range(int(n)):
            for first, count in edges:
                lbm.lbm_step_begin(self.h, first, count)
            pending = post_halos(self.dist, self.slab, self._get, self._get_cross, self.group)
            for first, count in interior:
                lbm.lbm_step_begin(self.h, first, count)
            finish_halos(self.slab, pending, self._put, self._put_cross)
            lbm.lbm_step_end(self.h)

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
