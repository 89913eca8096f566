"""Second, independent statement of the step in plain Python (tiny grids only).

Test helper.  It is written apart from the C oracle on purpose: its own
velocity ordering (all vectors of {-1,0,1}^d with |c|^2 <= 2, in
lexicographic order), weights and stencil coefficients chosen from |c|^2,
node storage in dicts, and pull-form streaming.  Comparing the two on
macroscopic fields after a few steps catches index, wrap-around and sign
slips in either.  Physics readings are the same as the oracle's (Sec. 2-4).
"""
import itertools
import math

THETA = 1.0 / 3.0


def lattice(d):
    vecs = [v for v in itertools.product((-1, 0, 1), repeat=d) if sum(c * c for c in v) <= 2]
    if d == 2:
        w = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
        G = {1: 1.0, 2: 0.25}
        alpha = 1.5
    else:
        w = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}
        G = {1: 1.0, 2: 0.5}
        alpha = 3.0
    ws = [w[sum(c * c for c in v)] for v in vecs]
    Gs = [G.get(sum(c * c for c in v), 0.0) for v in vecs]
    opp = [vecs.index(tuple(-c for c in v)) for v in vecs]
    return vecs, ws, Gs, opp, alpha


def equilibrium(vecs, ws, dens, u):
    usq = sum(a * a for a in u)
    out = []
    for v, w in zip(vecs, ws):
        cu = sum(c * a for c, a in zip(v, u))
        out.append(dens * w * (1 + cu / THETA + cu * cu / (2 * THETA ** 2) - usq / (2 * THETA)))
    return out


class Tiny:
    """Tiny domain: dims = (nx, ny) or (nx, ny, nz); the last axis may carry walls."""

    def __init__(self, dims, prm, rho, u, T):
        self.dims = tuple(dims)
        self.d = len(dims)
        self.prm = prm
        self.vecs, self.w, self.G, self.opp, self.alpha = lattice(self.d)
        self.N, self.g = {}, {}
        for x in self.nodes():
            ux = [u[a][x] for a in range(self.d)]
            self.N[x] = equilibrium(self.vecs, self.w, rho[x], ux)
            self.g[x] = equilibrium(self.vecs, self.w, rho[x] * prm["c_v"] * T[x], ux)

    def nodes(self):
        return list(itertools.product(*[range(n) for n in self.dims]))

    def shift(self, x, v):
        """Return (node, crossed_wall) for x + v; ghost nodes map to the mirror node."""
        y = list(x)
        crossed = 0
        for a in range(self.d):
            y[a] = x[a] + v[a]
            n = self.dims[a]
            if a == self.d - 1 and self.prm["wall"]:
                if y[a] < 0:
                    y[a] = -1 - y[a]
                    crossed = -1
                elif y[a] >= n:
                    y[a] = 2 * n - 1 - y[a]
                    crossed = 1
            else:
                y[a] %= n
        return tuple(y), crossed

    def eos(self, dens, T):
        prm = self.prm
        Te = prm["T0"] if prm["barotropic"] else T
        return prm["kappa"] * (8 * dens * Te / (3 - dens) - 3 * dens * dens)

    def macros(self):
        m = {}
        for x in self.nodes():
            dens = sum(self.N[x])
            mom = [sum(v[a] * f for v, f in zip(self.vecs, self.N[x])) for a in range(self.d)]
            E = sum(self.g[x])
            T = E / (dens * self.prm["c_v"])
            p = self.eos(dens, T)
            U = p - dens * THETA
            m[x] = {"rho": dens, "u": [j / dens for j in mom], "E": E, "T": T, "p": p,
                    "Phi": math.sqrt(-U) if U < 0 else 0.0}
        return m

    def force(self, m, x):
        prm = self.prm
        s1 = [0.0] * self.d
        s2 = [0.0] * self.d
        for v, G in zip(self.vecs, self.G):
            if G == 0.0:
                continue
            y, _ = self.shift(x, v)
            ph = m[y]["Phi"]
            for a in range(self.d):
                s1[a] += G * ph * ph * v[a]
                s2[a] += G * ph * v[a]
        A = prm["A"]
        return [(A * s1[a] + (1 - 2 * A) * m[x]["Phi"] * s2[a]) / self.alpha + m[x]["rho"] * prm["g"][a]
                for a in range(self.d)]

    def lam(self, dens):
        prm = self.prm
        return dens * prm["c_v"] * prm["chi"] if prm["chi_mode"] else prm["lam"]

    def step(self):
        prm = self.prm
        m = self.macros()
        F = {x: self.force(m, x) for x in self.nodes()}
        us = {x: [m[x]["u"][a] + 0.5 * F[x][a] / m[x]["rho"] for a in range(self.d)] for x in self.nodes()}
        post_N, post_g = {}, {}
        for x in self.nodes():
            dE = 0.0
            for a in range(self.d):
                e = [0] * self.d
                e[a] = 1
                yp, cp = self.shift(x, e)
                ym, cm = self.shift(x, [-c for c in e])
                up = -us[yp][a] if cp else us[yp][a]
                um = -us[ym][a] if cm else us[ym][a]
                Tp, Tm = m[yp]["T"], m[ym]["T"]
                if cp and prm["T_fixed_hi"]:
                    Tp = 2 * prm["T_hi"] - Tp
                if cm and prm["T_fixed_lo"]:
                    Tm = 2 * prm["T_lo"] - Tm
                if prm["pressure_work"]:
                    dE -= m[x]["p"] * (up - um) / 2
                if prm["conduction"]:
                    lp = 0.5 * (self.lam(m[x]["rho"]) + self.lam(m[yp]["rho"]))
                    lm = 0.5 * (self.lam(m[x]["rho"]) + self.lam(m[ym]["rho"]))
                    dE += lp * (Tp - m[x]["T"]) - lm * (m[x]["T"] - Tm)
            u = m[x]["u"]
            du = [F[x][a] / m[x]["rho"] for a in range(self.d)]
            u2 = [u[a] + du[a] for a in range(self.d)]
            n0 = equilibrium(self.vecs, self.w, m[x]["rho"], u)
            n1 = equilibrium(self.vecs, self.w, m[x]["rho"], u2)
            e0 = equilibrium(self.vecs, self.w, m[x]["E"], u)
            e1 = equilibrium(self.vecs, self.w, m[x]["E"], u2)
            post_N[x] = [f + (a0 - f) / prm["tau"] + (a1 - a0) for f, a0, a1 in zip(self.N[x], n0, n1)]
            post_g[x] = [h + (b0 - h) / prm["tau_E"] + h * dE / m[x]["E"] +
                         ((b1 - b0) if prm["pseudoforce"] else 0.0)
                         for h, b0, b1 in zip(self.g[x], e0, e1)]
        # pull: population k arriving at x left x - c_k, or bounced at x
        for x in self.nodes():
            newN, newg = [], []
            for k, v in enumerate(self.vecs):
                src, crossed = self.shift(x, [-c for c in v])
                if crossed:
                    newN.append(post_N[x][self.opp[k]])
                    newg.append(post_g[x][self.opp[k]])
                else:
                    newN.append(post_N[src][k])
                    newg.append(post_g[src][k])
            self.N[x], self.g[x] = newN, newg

    def outputs(self):
        """rho, u* (physical velocity), T and P per node."""
        m = self.macros()
        out = {}
        for x in self.nodes():
            F = self.force(m, x)
            out[x] = {"rho": m[x]["rho"], "T": m[x]["T"], "P": m[x]["p"],
                      "u": [m[x]["u"][a] + 0.5 * F[a] / m[x]["rho"] for a in range(self.d)]}
        return out
