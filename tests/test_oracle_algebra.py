"""Pins of the FP64 oracle against what the paper and the algebra fix.

Tables (Sec. 2-3), equilibrium moments (Eq. (feq)), exact conservation of the
collision and the EDM (Eq. (edm)), the force stencil (Sec. 3) and the
second moment after a tau = 1 step.  CPU only.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("Q,name", [(9, "D2Q9"), (19, "D3Q19")])
def test_lattice_tables_match_paper(Q, name):
    L = oracle.lattice(Q)
    c, w, G = L["c"], L["w"], L["G"]
    norm2 = (c ** 2).sum(1)
    gw = GOLD["weights"][name]
    np.testing.assert_allclose(w[norm2 == 0], gw["rest"], rtol=0, atol=1e-16)
    np.testing.assert_allclose(w[norm2 == 1], gw["nearest"], rtol=0, atol=1e-16)
    np.testing.assert_allclose(w[norm2 == 2], gw["next_nearest"], rtol=0, atol=1e-16)
    gs = GOLD["force_stencil"]
    np.testing.assert_allclose(G[norm2 == 1], gs["G_nearest"])
    np.testing.assert_allclose(G[norm2 == 2], gs["G_next_nearest"][name])
    assert L["alpha"] == gs["alpha"][name]
    d = 2 if Q == 9 else 3
    # velocity counts of Sec. 2: |c| = 0, 1, sqrt(2)
    assert (norm2 == 0).sum() == 1 and (norm2 == 1).sum() == 2 * d
    assert (norm2 == 2).sum() == (4 if d == 2 else 12)
    assert np.all(c[:, d:] == 0)
    # opposite directions
    assert np.all(c[L["opp"]] == -c)


@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_isotropy(Q):
    """Weight moments up to fourth order and the force-stencil sums:
    sum G e e = 2 alpha I makes the discrete force tend to grad(Phi^2)."""
    L = oracle.lattice(Q)
    d = 2 if Q == 9 else 3
    c = L["c"][:, :d].astype(float)
    w, G = L["w"], L["G"]
    th = GOLD["kinetic_temperature"]["theta"]
    I = np.eye(d)
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("k,ka->a", w, c), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("k,ka,kb->ab", w, c, c), th * I, atol=1e-15)
    np.testing.assert_allclose(np.einsum("k,ka,kb,kc->abc", w, c, c, c), 0, atol=1e-16)
    iso4 = th * th * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) +
                      np.einsum("ad,bc->abcd", I, I))
    np.testing.assert_allclose(np.einsum("k,ka,kb,kc,kd->abcd", w, c, c, c, c), iso4, atol=1e-15)
    np.testing.assert_allclose(np.einsum("k,ka->a", G, c), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("k,ka,kb->ab", G, c, c), 2 * L["alpha"] * I, atol=1e-15)


@pytest.mark.parametrize("Q", [9, 19])
def test_equilibrium_moments(Q):
    """Eq. (feq): sum f = rho, sum c f = rho u, sum c c f = rho theta I + rho u u."""
    rng = np.random.default_rng(1)
    L = oracle.lattice(Q)
    d = 2 if Q == 9 else 3
    c = L["c"][:, :d].astype(float)
    th = 1.0 / 3.0
    for _ in range(20):
        rho = rng.uniform(0.05, 2.5)
        u = rng.uniform(-0.2, 0.2, size=d)
        f = oracle.feq(Q, rho, u)
        assert abs(f.sum() - rho) < 1e-14 * rho
        np.testing.assert_allclose(c.T @ f, rho * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("k,ka,kb->ab", f, c, c),
                                   rho * th * np.eye(d) + rho * np.outer(u, u), atol=1e-14)


def _random_two_phase(Q, shape, seed, T=0.8):
    from paper_1705_10045_gb300 import workloads as W
    rv, rl = W.coexistence(T)
    rng = np.random.default_rng(seed)
    d = 2 if Q == 9 else 3
    rho = rng.uniform(rv, rl, size=shape)
    u = rng.uniform(-0.02, 0.02, size=(d,) + shape)
    Tf = T + rng.uniform(-0.02, 0.02, size=shape)
    return rho, u, Tf


@pytest.mark.parametrize("Q,shape", [(9, (1, 12, 10)), (19, (6, 5, 7))])
def test_force_sums_to_zero_periodic(Q, shape):
    """Both terms of the discrete force telescope on a periodic lattice
    (sum_k G_k e_k = 0 and the +e/-e pairs cancel), so sum_x F = 0."""
    p = oracle.Params(Q=Q, nx=shape[2], ny=shape[1], nz=shape[0])
    rng = np.random.default_rng(3)
    Phi = rng.uniform(0.1, 0.9, size=shape)
    rho = rng.uniform(0.1, 2.0, size=shape)
    F = oracle.force(p, Phi, rho)
    scale = np.abs(F).sum()
    assert scale > 1.0
    np.testing.assert_allclose(F.reshape(p.d, -1).sum(1), 0, atol=1e-13 * scale)


@pytest.mark.parametrize("Q", [9, 19])
def test_force_tends_to_gradient_of_phi_squared(Q):
    """For a smooth Phi the stencil of Sec. 3 approximates 2A grad Phi^2 +
    (1-2A) 2 Phi grad Phi = grad Phi^2 = -grad U with second-order error."""
    errs = []
    for L in (16, 32, 64):
        nz = 1 if Q == 9 else 2
        p = oracle.Params(Q=Q, nx=L, ny=2, nz=nz)
        x = np.arange(L, dtype=float)
        phi1 = 0.6 + 0.2 * np.sin(2 * np.pi * x / L)
        Phi = np.broadcast_to(phi1, p.shape).copy()
        F = oracle.force(p, Phi, np.ones(p.shape))
        exact = 2 * phi1 * 0.2 * np.cos(2 * np.pi * x / L) * 2 * np.pi / L
        errs.append(np.abs(F[0].reshape(-1, L)[0] - exact).max() / np.abs(exact).max())
        np.testing.assert_allclose(F[1:], 0, atol=1e-15)
    assert errs[-1] < 3e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("Q,shape", [(9, (1, 6, 8)), (19, (4, 5, 6))])
def test_collision_and_edm_conserve_mass_and_add_force(Q, shape):
    """Uniform fluid under gravity: the interparticle force vanishes and one
    step adds exactly rho g to every node's momentum (Eq. (edm)); mass and
    energy are unchanged; with tau = 1 the momentum flux becomes that of
    N^eq(rho, u + du): rho theta I + rho (u+du)(u+du)."""
    d = 2 if Q == 9 else 3
    g = (1e-3, -2e-3, 5e-4)[:d] + (0.0,) * (3 - d)
    for tau in (0.7, 1.0):
        p = oracle.Params(Q=Q, nx=shape[2], ny=shape[1], nz=shape[0], g=g, tau=tau, tau_E=tau)
        u0 = np.array([0.01, -0.02, 0.005][:d])
        rho0, T0 = 0.3, 0.8
        u = np.broadcast_to(u0[:, None, None, None], (d,) + shape).copy()
        s = oracle.State(p, np.full(shape, rho0), u, np.full(shape, p.c_v * T0))
        s.step(1)
        L = oracle.lattice(Q)
        c = L["c"][:, :d].astype(float)
        N = s.N.reshape(Q, -1)
        rho = N.sum(0)
        j = c.T @ N
        np.testing.assert_allclose(rho, rho0, rtol=1e-15)
        want_j = (rho0 * u0 + rho0 * np.array(g[:d]))[:, None]
        np.testing.assert_allclose(j, np.broadcast_to(want_j, j.shape), atol=1e-16)
        np.testing.assert_allclose(s.g.reshape(Q, -1).sum(0), rho0 * p.c_v * T0, rtol=1e-15)
        if tau == 1.0:
            v = u0 + np.array(g[:d])
            Pi = np.einsum("kn,ka,kb->abn", N, c, c)
            want = rho0 / 3.0 * np.eye(d) + rho0 * np.outer(v, v)
            np.testing.assert_allclose(Pi, np.broadcast_to(want[:, :, None], Pi.shape), atol=1e-15)


@pytest.mark.parametrize("Q,shape", [(9, (1, 24, 32)), (19, (8, 8, 10))])
def test_two_phase_conservation_periodic(Q, shape):
    """Periodic two-phase flow without gravity: total mass and momentum are
    conserved to rounding over many steps; with pressure work off the total
    internal energy is conserved too (conduction is in conservative form)."""
    rho, u, T = _random_two_phase(Q, shape, seed=7)
    p = oracle.Params(Q=Q, nx=shape[2], ny=shape[1], nz=shape[0], pressure_work=False)
    s = oracle.State(p, rho, u, p.c_v * T)
    L = oracle.lattice(Q)
    d = p.d
    c = L["c"][:, :d].astype(float)

    def totals():
        N = s.N.reshape(Q, -1)
        return N.sum(), (c.T @ N).sum(1), s.g.sum()

    m0, j0, e0 = totals()
    s.step(200)
    m1, j1, e1 = totals()
    assert s.clamps == 0
    assert abs(m1 - m0) < 1e-12 * m0
    np.testing.assert_allclose(j1, j0, atol=1e-12 * m0)
    assert abs(e1 - e0) < 1e-12 * e0
