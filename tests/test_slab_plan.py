"""The slab plan of lbm_slab_plan (host only, no GPU): the owned ranges tile
the last axis, the halos sit at the cuts (and wrap on a periodic axis), the
neighbours are the adjacent slabs, a slab's own domain is its owned planes
plus its halos, and fixed wall temperatures stay at the domain's ends."""
import pytest

from paper_1705_10045_gb300 import build as B
from paper_1705_10045_gb300 import lbm

H = lbm.LBM_SLAB_HALO


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()


def _plans(count, **kw):
    p = lbm.make_params(**kw)
    return p, [lbm.lbm_slab_plan(p, count, i) for i in range(count)]


@pytest.mark.parametrize("count", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("wall", [0, 1])
def test_owned_ranges_tile_the_last_axis(count, wall):
    p, plans = _plans(count, lattice=19, nx=8, ny=6, nz=43, wall=wall, T_fixed_lo=1, T_lo=0.9, T_fixed_hi=1,
                      T_hi=0.7)
    assert [s.first for s in plans] == [sum(t.own for t in plans[:i]) for i in range(count)]
    assert sum(s.own for s in plans) == 43
    assert max(s.own for s in plans) - min(s.own for s in plans) <= 1
    for i, s in enumerate(plans):
        cut_lo = count > 1 and (not wall or i > 0)
        cut_hi = count > 1 and (not wall or i < count - 1)
        assert (s.lo, s.hi) == (H if cut_lo else 0, H if cut_hi else 0)
        assert s.below == ((i - 1) % count if cut_lo else -1)
        assert s.above == ((i + 1) % count if cut_hi else -1)
        assert (s.p.nx, s.p.ny, s.p.nz) == (8, 6, s.lo + s.own + s.hi)
        assert s.p.wall == wall
        # the fixed temperatures belong to the domain's ends only
        assert s.p.T_fixed_lo == (0 if cut_lo else 1)
        assert s.p.T_fixed_hi == (0 if cut_hi else 1)
        assert (s.p.T_lo, s.p.T_hi) == (0.9, 0.7)


def test_d2q9_cuts_along_y_and_keeps_the_physics():
    p, plans = _plans(3, lattice=9, nx=17, ny=30, latent=0.02, tau=0.8, chi_mode=1, chi=0.05)
    for s in plans:
        assert (s.p.nx, s.p.nz) == (17, 1) and s.p.ny == s.own + 2 * H
        assert (s.p.latent, s.p.tau, s.p.chi_mode, s.p.chi) == (0.02, 0.8, 1, 0.05)
    # the neighbours' owned planes next to a cut are the planes a halo copies
    for i, s in enumerate(plans):
        up = plans[s.above]
        assert (s.first + s.own) % 30 == up.first


def test_one_slab_is_the_whole_domain():
    p, (s,) = _plans(1, lattice=19, nx=4, ny=4, nz=9, wall=1, T_fixed_lo=1)
    assert (s.first, s.own, s.lo, s.hi, s.below, s.above) == (0, 9, 0, 0, -1, -1)
    assert s.p.nz == 9 and s.p.T_fixed_lo == 1


@pytest.mark.parametrize("count, i", [(0, 0), (2, 2), (2, -1), (4, 0)])
def test_plan_rejects_bad_counts_and_thin_slabs(count, i):
    # 8 planes into 4 slabs leaves slabs of 2 planes, as many as the halo
    # (a neighbour's halo copies both): allowed; 7 planes into 4 would leave
    # 1-plane slabs, thinner than the halo
    assert H == 2
    p = lbm.make_params(lattice=19, nx=4, ny=4, nz=7)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_slab_plan(p, count, i)
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lbm_slab_plan(lbm.make_params(lattice=19, nx=4, ny=4, nz=8), 4, 3).own == 2


@pytest.mark.parametrize("count", [0, -1, 5])
def test_slabs_create_rejects_bad_counts_before_touching_a_device(count):
    import ctypes
    p = lbm.make_params(lattice=19, nx=4, ny=4, nz=9)
    s = ctypes.c_void_p()
    assert lbm.load().lbm_slabs_create(ctypes.byref(p), count, ctypes.byref(s)) == lbm.LBM_ERR_INVALID_ARG
    assert not s.value


@pytest.mark.parametrize("lattice,nm,wall", [(19, 256, 1), (19, 17, 0), (9, 60, 0), (19, 40, 1), (9, 33, 1)])
@pytest.mark.parametrize("count", [1, 2, 3, 4, 5])
def test_split_ranges_cover_the_owned_planes_once_with_the_cut_planes_first(lattice, nm, wall, count):
    """The planes a slab process steps before posting its swap and those it
    steps while the swap travels: disjoint, covering its owned planes, and
    the first list holds the three planes beside every cut (which give the
    two edge planes the swap sends all their pushes)."""
    from paper_1705_10045_gb300.slabs import EDGE_PLANES, split_ranges
    kw = dict(lattice=lattice, nx=8, ny=nm if lattice == 9 else 6, nz=nm if lattice == 19 else 1, wall=wall)
    p = lbm.make_params(**kw)
    if count > 1 and nm // count < lbm.LBM_SLAB_HALO:
        return
    for i in range(count):
        sl = lbm.lbm_slab_plan(p, count, i)
        edges, interior = split_ranges(sl)
        planes = [q for f, c in edges + interior for q in range(f, f + c)]
        assert sorted(planes) == list(range(sl.lo, sl.lo + sl.own))
        assert len(planes) == len(set(planes))
        first = {q for f, c in edges for q in range(f, f + c)}
        need = set()
        if sl.lo:
            need |= set(range(sl.lo, min(sl.lo + EDGE_PLANES, sl.lo + sl.own)))
        if sl.hi:
            need |= set(range(max(sl.lo, sl.lo + sl.own - EDGE_PLANES), sl.lo + sl.own))
        assert need <= first
        assert all(c >= 1 for _, c in edges + interior)
