/*
 * Plain FP64 CPU oracle of one time step of the thermal multiphase lattice
 * Boltzmann method of Kupershtokh, Medvedev and Gribanov, "Thermal lattice
 * Boltzmann method for multiphase flows" (arXiv:1705.10045).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * table or header with the CUDA library.
 *
 * Conventions (lattice units h = dt = 1, so theta = 1/3, Sec. 2):
 *   - nodes are indexed  n = (z*ny + y)*nx + x  (x fastest); D2Q9 has nz = 1;
 *   - populations are stored as Q planes of nn nodes: f[k*nn + n];
 *   - vector fields (u, F, du, u*) are d planes of nn nodes: v[a*nn + n];
 *   - every sum over k runs k = 0..Q-1 in order, every loop over nodes in
 *     index order, two population arrays (push streaming), no fused
 *     multiply-add (built with -ffp-contract=off).
 *
 * Readings of points on which the paper is silent (walls, order of the
 * sources inside a step, the multi-D finite-difference formulas, the EOS
 * scale kappa) are listed where they are used.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int Q;               /* 9 (D2Q9) or 19 (D3Q19) */
    int nx, ny, nz;      /* nz = 1 for D2Q9 */
    double kappa;        /* p = kappa * p~(rho, T): lattice pressure scale */
    double A;            /* mixing parameter of the force, Sec. 3 */
    int barotropic;      /* 1: EOS evaluated at T0 instead of T (Sec. 4) */
    double T0;
    double tau, tau_E;   /* relaxation times, Eq. (lbe) and Eq. (gk) */
    double c_v;          /* specific heat, E = rho c_v T (Sec. 4) */
    int chi_mode;        /* 0: constant lambda; 1: lambda = rho c_v chi */
    double lambda, chi;
    double g[3];         /* body force per unit mass (gravity) */
    int wall;            /* last axis: 0 periodic, 1 bounce-back walls at both ends */
    int T_fixed_lo, T_fixed_hi;   /* wall temperature mode: 0 adiabatic, 1 fixed */
    double T_lo, T_hi;
    int wall_x;          /* x axis: 0 periodic, 1 bounce-back walls at both ends */
    int wall_y;          /* y axis of D3Q19 (for D2Q9 y is the last axis: `wall`) */
    int T_fixed_x[2], T_fixed_y[2];   /* per wall (low, high end): 0 adiabatic, 1 fixed */
    double T_x[2], T_y[2];
    int pressure_work, conduction, pseudoforce;   /* physics switches */
    double latent;       /* rho_liq Q of Sec. 5 (energy per volume); 0: no latent heat */
    const double* coex;  /* Maxwell densities on the temperature grid below:
                            coex[j] = rho_v(T_j), coex[LH_N + 1 + j] = rho_l(T_j) */
} orc_params;

/* Temperature grid of the coexistence table used by the latent-heat source:
 * T_j = LH_T0 + j / LH_PER_T, j = 0..LH_N (the last point is the critical
 * point, where rho_v = rho_l = 1). */
#define LH_T0 0.5
#define LH_PER_T 1024.0
#define LH_N 512

/* ---------------------------------------------------------------------- */
/* Velocity sets, Sec. 2: rest vector, nearest neighbours, next-nearest.
 * Opposite directions are stored next to each other (k odd <-> k+1).      */

static const int C9[9][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

static const int C19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static const int (*vel(int Q))[3] { return Q == 9 ? C9 : C19; }

/* weights w_k, Sec. 2 (D2Q9: 4/9, 1/9, 1/36; D3Q19: 1/3, 1/18, 1/36) */
static double weight(int Q, int k)
{
    if (Q == 9) return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

/* force-stencil coefficients G_k, Sec. 3 (1 for nearest neighbours; 1/4 for
 * D2Q9 and 1/2 for D3Q19 next-nearest neighbours), G_0 unused */
static double stencil_G(int Q, int k)
{
    if (k == 0) return 0.0;
    if (Q == 9) return k <= 4 ? 1.0 : 0.25;
    return k <= 6 ? 1.0 : 0.5;
}

/* alpha of the force approximation, Sec. 3: 3/2 (D2Q9), 3 (D3Q19) */
static double stencil_alpha(int Q) { return Q == 9 ? 1.5 : 3.0; }

static int opposite(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

static int dims(const orc_params* p) { return p->Q == 9 ? 2 : 3; }

static const double THETA = 1.0 / 3.0;   /* kinetic temperature (h/dt)^2/3 */

/* ---------------------------------------------------------------------- */
/* Equilibrium, Eq. (feq):
 *   f_k^eq(rho,u) = rho w_k (1 + (c.u)/theta + (c.u)^2/(2 theta^2) - u^2/(2 theta)) */
void orc_feq(int Q, double rho, const double* u, double* out)
{
    const int (*c)[3] = vel(Q);
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < Q; ++k) {
        double cu = c[k][0] * u[0] + c[k][1] * u[1] + c[k][2] * u[2];
        out[k] = rho * weight(Q, k) *
                 (1.0 + cu / THETA + cu * cu / (2.0 * THETA * THETA) - uu / (2.0 * THETA));
    }
}

/* Lattice tables, exposed so that the tests can check them. */
int orc_lattice(int Q, int* c, double* w, double* G, int* opp, double* alpha)
{
    if (Q != 9 && Q != 19) return -1;
    const int (*cv)[3] = vel(Q);
    for (int k = 0; k < Q; ++k) {
        for (int a = 0; a < 3; ++a) c[3 * k + a] = cv[k][a];
        w[k] = weight(Q, k);
        G[k] = stencil_G(Q, k);
        opp[k] = opposite(k);
    }
    *alpha = stencil_alpha(Q);
    return 0;
}

/* Reduced van der Waals equation of state, Sec. 3: p~ = 8 rho T/(3-rho) - 3 rho^2,
 * scaled to lattice units by kappa (the paper gives only reduced variables). */
double orc_pressure(const orc_params* p, double rho, double T)
{
    double Te = p->barotropic ? p->T0 : T;
    return p->kappa * (8.0 * rho * Te / (3.0 - rho) - 3.0 * rho * rho);
}

/* ---------------------------------------------------------------------- */
/* Neighbour lookup.  Each axis is periodic or closed by walls half a node
 * outside its first and last layer (the last axis through `wall`, x through
 * `wall_x`, y of D3Q19 through `wall_y`).  Outside a wall the stencils read
 * the mirror node (a node at distance m beyond the wall mirrors the node at
 * distance m-1 inside); g[a] is -1 / +1 when the step crosses the low / high
 * wall of axis a, and ghost is nonzero when it crosses any wall. */

typedef struct { long n; int ghost; int g[3]; } nb_t;

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* coordinate i + d along an axis of n nodes, periodic or walled */
static int axis_step(int i, int n, int walled, int* g)
{
    *g = 0;
    if (!walled) return wrap(i, n);
    if (i < 0) { *g = -1; return -1 - i; }
    if (i >= n) { *g = 1; return 2 * n - 1 - i; }
    return i;
}

static nb_t neighbour(const orc_params* p, int x, int y, int z, int dx, int dy, int dz)
{
    nb_t r;
    int X = axis_step(x + dx, p->nx, p->wall_x, &r.g[0]);
    int Y, Z;
    if (p->Q == 9) {
        Y = axis_step(y + dy, p->ny, p->wall, &r.g[1]);
        Z = 0;
        r.g[2] = 0;
    } else {
        Y = axis_step(y + dy, p->ny, p->wall_y, &r.g[1]);
        Z = axis_step(z + dz, p->nz, p->wall, &r.g[2]);
    }
    r.ghost = r.g[0] != 0 || r.g[1] != 0 || r.g[2] != 0;
    r.n = ((long)Z * p->ny + Y) * p->nx + X;
    return r;
}

/* Temperature mode of the wall at end `hi` (0 low, 1 high) of axis a:
 * returns 1 and the wall temperature when that wall is held at a fixed T. */
static int wall_T(const orc_params* p, int a, int hi, double* Tw)
{
    const int last = p->Q == 9 ? 1 : 2;
    if (a == last) {
        *Tw = hi ? p->T_hi : p->T_lo;
        return hi ? p->T_fixed_hi : p->T_fixed_lo;
    }
    if (a == 0) {
        *Tw = p->T_x[hi];
        return p->T_fixed_x[hi];
    }
    *Tw = p->T_y[hi];
    return p->T_fixed_y[hi];
}

static long nnodes(const orc_params* p) { return (long)p->nx * p->ny * p->nz; }

/* ---------------------------------------------------------------------- */
/* Step part 1: macroscopic fields of every node, Eq. (hydro), E = sum g_k
 * (Sec. 4), T = E/(rho c_v), p from the EOS, U = p - rho theta and
 * Phi = sqrt(-U) (Eq. (force) and Sec. 3).  Where U >= 0 the square root
 * is undefined; Phi is set to 0 there and the node is counted. */
long orc_macros(const orc_params* p, const double* N, const double* g,
                double* rho, double* u, double* E, double* T, double* P, double* Phi)
{
    const int (*c)[3] = vel(p->Q);
    const int d = dims(p);
    const long nn = nnodes(p);
    long clamps = 0;
    for (long n = 0; n < nn; ++n) {
        double r = 0.0, e = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < p->Q; ++k) {
            double f = N[k * nn + n];
            r += f;
            for (int a = 0; a < d; ++a) j[a] += c[k][a] * f;
            e += g[k * nn + n];
        }
        rho[n] = r;
        for (int a = 0; a < d; ++a) u[a * nn + n] = j[a] / r;
        E[n] = e;
        T[n] = e / (r * p->c_v);
        P[n] = orc_pressure(p, r, T[n]);
        double U = P[n] - r * THETA;
        if (U < 0.0) {
            Phi[n] = sqrt(-U);
        } else {
            Phi[n] = 0.0;
            ++clamps;
        }
    }
    return clamps;
}

/* Step part 2: the force of Sec. 3 in its isotropic discrete form
 *   F(x) = (1/alpha) [ A sum_k G_k Phi^2(x+e_k) e_k
 *                      + (1-2A) Phi(x) sum_k G_k Phi(x+e_k) e_k ]
 * plus gravity rho g (the EDM takes any total force, Sec. 2).
 * Outside a wall Phi is read at the mirror node (neutral wetting). */
void orc_force(const orc_params* p, const double* Phi, const double* rho, double* F)
{
    const int (*c)[3] = vel(p->Q);
    const int d = dims(p);
    const long nn = nnodes(p);
    const double alpha = stencil_alpha(p->Q);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = ((long)z * p->ny + y) * p->nx + x;
                double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
                for (int k = 1; k < p->Q; ++k) {
                    nb_t m = neighbour(p, x, y, z, c[k][0], c[k][1], c[k][2]);
                    double ph = Phi[m.n];
                    double G = stencil_G(p->Q, k);
                    for (int a = 0; a < d; ++a) {
                        s1[a] += G * ph * ph * c[k][a];
                        s2[a] += G * ph * c[k][a];
                    }
                }
                for (int a = 0; a < d; ++a)
                    F[a * nn + n] = (p->A * s1[a] + (1.0 - 2.0 * p->A) * Phi[n] * s2[a]) / alpha
                                    + rho[n] * p->g[a];
            }
}

/* heat conductivity of a node: constant lambda, or lambda = rho c_v chi (Sec. 4) */
static double conductivity(const orc_params* p, double rho)
{
    return p->chi_mode ? rho * p->c_v * p->chi : p->lambda;
}

/* Vapour and liquid densities on the coexistence curve at temperature T, by
 * linear interpolation in the table (T below the grid takes its first
 * point).  Returns 0 at or above the critical temperature (no two-phase
 * band), 1 otherwise. */
static int coexistence_at(const orc_params* p, double T, double* rv, double* rl)
{
    if (!(T < 1.0)) return 0;
    double s = (T - LH_T0) * LH_PER_T;
    if (s < 0.0) s = 0.0;
    int j = (int)floor(s);
    if (j > LH_N - 1) j = LH_N - 1;
    double f = s - (double)j;
    const double* v = p->coex;
    const double* l = p->coex + LH_N + 1;
    *rv = v[j] + f * (v[j + 1] - v[j]);
    *rl = l[j] + f * (l[j + 1] - l[j]);
    return 1;
}

/* Step part 3: change of internal energy by finite differences (Sec. 4):
 *   pressure work  -p div(u*) dt, with the centred difference of Sec. 6.2
 *   applied along every axis;
 *   conduction     div(lambda grad T) dt, conservative form with the face
 *   conductivity the mean of the two nodes.
 * Across a wall of axis a: u*_a(ghost) = -u*_a(mirror) (no-slip; only the
 * component normal to the wall enters the difference along a),
 * T(ghost) = T(mirror) for an adiabatic wall and 2 T_w - T(mirror) for a wall
 * held at T_w.
 * Latent heat of the phase transition (Sec. 5), when p->latent = rho_liq Q
 * is nonzero: inside the transition layer rho_v(T) < rho < rho_l(T) the
 * energy changes by  (rho_liq Q / (rho_l - rho_v)) d(rho)/dt  with
 * d(rho)/dt = -rho div(u*), the divergence being the same centred
 * difference as in the pressure work. */
void orc_energy_source(const orc_params* p, const double* rho, const double* ustar,
                       const double* T, const double* P, double* dE)
{
    const int d = dims(p);
    const long nn = nnodes(p);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = ((long)z * p->ny + y) * p->nx + x;
                double div = 0.0, cond = 0.0;
                for (int a = 0; a < d; ++a) {
                    int e[3] = {0, 0, 0};
                    e[a] = 1;
                    nb_t up = neighbour(p, x, y, z, e[0], e[1], e[2]);
                    nb_t dn = neighbour(p, x, y, z, -e[0], -e[1], -e[2]);
                    double uu = up.g[a] ? -ustar[a * nn + up.n] : ustar[a * nn + up.n];
                    double ud = dn.g[a] ? -ustar[a * nn + dn.n] : ustar[a * nn + dn.n];
                    div += (uu - ud) / 2.0;

                    double Tu = T[up.n], Td = T[dn.n], Tw;
                    if (up.g[a] && wall_T(p, a, 1, &Tw)) Tu = 2.0 * Tw - T[up.n];
                    if (dn.g[a] && wall_T(p, a, 0, &Tw)) Td = 2.0 * Tw - T[dn.n];
                    double lc = conductivity(p, rho[n]);
                    double lu = (lc + conductivity(p, rho[up.n])) / 2.0;
                    double ld = (lc + conductivity(p, rho[dn.n])) / 2.0;
                    cond += lu * (Tu - T[n]) - ld * (T[n] - Td);
                }
                double s = 0.0;
                if (p->pressure_work) s += -P[n] * div;
                if (p->conduction) s += cond;
                if (p->latent != 0.0) {
                    double rv, rl;
                    if (coexistence_at(p, T[n], &rv, &rl) && rho[n] > rv && rho[n] < rl)
                        s += -p->latent * rho[n] * div / (rl - rv);
                }
                dE[n] = s;
            }
}

/* Step part 4: BGK collision with the EDM source for N (Eq. (lbe), Eq. (edm)),
 * and for g (Eq. (gk)) with Delta g^(1) = g_k dE/E and the energy pseudoforce
 * Delta g^(2) = g^eq(E, u+du) - g^eq(E, u) (Sec. 4), followed by push
 * streaming to x + c_k.  All sources use the fields of time t.  A population
 * that would cross a wall returns to its node in the opposite direction
 * (halfway bounce-back, for N and g alike). */
void orc_collide_stream(const orc_params* p, const double* N, const double* g,
                        const double* rho, const double* u, const double* E,
                        const double* du, const double* dE, double* Nout, double* gout)
{
    const int (*c)[3] = vel(p->Q);
    const int Q = p->Q, d = dims(p);
    const long nn = nnodes(p);
    double feq0[19], feq1[19], geq0[19], geq1[19];
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long n = ((long)z * p->ny + y) * p->nx + x;
                double uv[3] = {0.0, 0.0, 0.0}, us[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < d; ++a) {
                    uv[a] = u[a * nn + n];
                    us[a] = uv[a] + du[a * nn + n];
                }
                orc_feq(Q, rho[n], uv, feq0);
                orc_feq(Q, rho[n], us, feq1);
                orc_feq(Q, E[n], uv, geq0);
                orc_feq(Q, E[n], us, geq1);
                for (int k = 0; k < Q; ++k) {
                    double f = N[k * nn + n];
                    double h = g[k * nn + n];
                    double fs = f + (feq0[k] - f) / p->tau + (feq1[k] - feq0[k]);
                    double hs = h + (geq0[k] - h) / p->tau_E + h * dE[n] / E[n];
                    if (p->pseudoforce) hs += geq1[k] - geq0[k];
                    nb_t m = neighbour(p, x, y, z, c[k][0], c[k][1], c[k][2]);
                    if (m.ghost) {
                        int kb = opposite(k);
                        Nout[kb * nn + n] = fs;
                        gout[kb * nn + n] = hs;
                    } else {
                        Nout[k * nn + m.n] = fs;
                        gout[k * nn + m.n] = hs;
                    }
                }
            }
}

/* ---------------------------------------------------------------------- */
/* Scratch for one step. */
typedef struct {
    double *rho, *u, *E, *T, *P, *Phi, *F, *du, *us, *dE, *N2, *g2;
} work_t;

static int work_alloc(const orc_params* p, work_t* w)
{
    const long nn = nnodes(p);
    const int d = dims(p);
    memset(w, 0, sizeof(*w));
    w->rho = malloc(sizeof(double) * nn);
    w->u = malloc(sizeof(double) * nn * d);
    w->E = malloc(sizeof(double) * nn);
    w->T = malloc(sizeof(double) * nn);
    w->P = malloc(sizeof(double) * nn);
    w->Phi = malloc(sizeof(double) * nn);
    w->F = malloc(sizeof(double) * nn * d);
    w->du = malloc(sizeof(double) * nn * d);
    w->us = malloc(sizeof(double) * nn * d);
    w->dE = malloc(sizeof(double) * nn);
    w->N2 = malloc(sizeof(double) * nn * p->Q);
    w->g2 = malloc(sizeof(double) * nn * p->Q);
    return (w->rho && w->u && w->E && w->T && w->P && w->Phi && w->F && w->du && w->us &&
            w->dE && w->N2 && w->g2) ? 0 : -1;
}

static void work_free(work_t* w)
{
    free(w->rho); free(w->u); free(w->E); free(w->T); free(w->P); free(w->Phi);
    free(w->F); free(w->du); free(w->us); free(w->dE); free(w->N2); free(w->g2);
}

/* velocity change and physical velocity: du = F dt/rho (Eq. (edm)),
 * u* = u + F dt/(2 rho) (Eq. (ustar)) */
static void velocities(const orc_params* p, const double* rho, const double* u,
                       const double* F, double* du, double* us)
{
    const int d = dims(p);
    const long nn = nnodes(p);
    for (int a = 0; a < d; ++a)
        for (long n = 0; n < nn; ++n) {
            du[a * nn + n] = F[a * nn + n] / rho[n];
            us[a * nn + n] = u[a * nn + n] + du[a * nn + n] / 2.0;
        }
}

/* Advance N, g (Q planes each, in place) by nsteps time steps.
 * Returns the number of (node, step) pairs where U >= 0 was clamped, or -1
 * when scratch memory could not be allocated. */
long orc_step(const orc_params* p, double* N, double* g, int nsteps)
{
    work_t w;
    const long nn = nnodes(p);
    if (work_alloc(p, &w)) { work_free(&w); return -1; }
    long clamps = 0;
    for (int s = 0; s < nsteps; ++s) {
        clamps += orc_macros(p, N, g, w.rho, w.u, w.E, w.T, w.P, w.Phi);
        orc_force(p, w.Phi, w.rho, w.F);
        velocities(p, w.rho, w.u, w.F, w.du, w.us);
        orc_energy_source(p, w.rho, w.us, w.T, w.P, w.dE);
        orc_collide_stream(p, N, g, w.rho, w.u, w.E, w.du, w.dE, w.N2, w.g2);
        memcpy(N, w.N2, sizeof(double) * nn * p->Q);
        memcpy(g, w.g2, sizeof(double) * nn * p->Q);
    }
    work_free(&w);
    return clamps;
}

/* Initial state: N = N^eq(rho, u), g = g^eq(rho eps, u) with eps = c_v T the
 * specific internal energy; u is taken as the lattice velocity of Eq. (hydro). */
void orc_init(const orc_params* p, const double* rho, const double* u, const double* eps,
              double* N, double* g)
{
    const int d = dims(p);
    const long nn = nnodes(p);
    double f[19];
    for (long n = 0; n < nn; ++n) {
        double uv[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < d; ++a) uv[a] = u[a * nn + n];
        orc_feq(p->Q, rho[n], uv, f);
        for (int k = 0; k < p->Q; ++k) N[k * nn + n] = f[k];
        orc_feq(p->Q, rho[n] * eps[n], uv, f);
        for (int k = 0; k < p->Q; ++k) g[k * nn + n] = f[k];
    }
}

/* Output fields of the current state: rho, the physical velocity u*
 * (Eq. (ustar)), T = E/(rho c_v) and the pressure P (EOS).  Any output may
 * be NULL.  Returns the clamp count of the state, or -1 on allocation failure. */
long orc_moments(const orc_params* p, const double* N, const double* g,
                 double* rho, double* ustar, double* T, double* P)
{
    work_t w;
    const long nn = nnodes(p);
    const int d = dims(p);
    if (work_alloc(p, &w)) { work_free(&w); return -1; }
    long clamps = orc_macros(p, N, g, w.rho, w.u, w.E, w.T, w.P, w.Phi);
    orc_force(p, w.Phi, w.rho, w.F);
    velocities(p, w.rho, w.u, w.F, w.du, w.us);
    if (rho) memcpy(rho, w.rho, sizeof(double) * nn);
    if (ustar) memcpy(ustar, w.us, sizeof(double) * nn * d);
    if (T) memcpy(T, w.T, sizeof(double) * nn);
    if (P) memcpy(P, w.P, sizeof(double) * nn);
    work_free(&w);
    return clamps;
}

/* Intermediate fields of one step, exposed for the tests: du (d planes) and
 * dE (one plane) from the current state. */
long orc_sources(const orc_params* p, const double* N, const double* g, double* du, double* dE)
{
    work_t w;
    const long nn = nnodes(p);
    const int d = dims(p);
    if (work_alloc(p, &w)) { work_free(&w); return -1; }
    long clamps = orc_macros(p, N, g, w.rho, w.u, w.E, w.T, w.P, w.Phi);
    orc_force(p, w.Phi, w.rho, w.F);
    velocities(p, w.rho, w.u, w.F, w.du, w.us);
    orc_energy_source(p, w.rho, w.us, w.T, w.P, w.dE);
    if (du) memcpy(du, w.du, sizeof(double) * nn * d);
    if (dE) memcpy(dE, w.dE, sizeof(double) * nn);
    work_free(&w);
    return clamps;
}
