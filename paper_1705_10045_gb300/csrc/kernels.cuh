// Kernels of liblbm: the per-time-step lattice update of the thermal
// multiphase LB method (arXiv:1705.10045), split into three launches:
//   fields_kernel   moments -> rho, u, T, Phi               (Eq. (hydro), Sec. 3-4)
//   force_kernel    Phi stencil + gravity -> du = F/rho     (Sec. 3, Eq. (edm))
//   collide_kernel  dE by finite differences, BGK + EDM for N, BGK + g dE/E +
//                   pseudoforce for g, push streaming with walls (Eq. (lbe), (gk))
// plus initialisation, output moments and the conservation reductions.
//
// Populations: Q arrays of nn node pairs (N_k, g_k), nn = nx*ny*nz, x fastest
// (lattice.cuh); checkpoints use 2Q set-major planes.  Fields: planes of nn
// values of the arithmetic type R.
#pragma once

#include "lattice.cuh"

namespace lbm {

// field planes (R): 0 rho, 1..3 u, 4 T, 5 Phi, 6..8 du
enum { F_RHO = 0, F_UX = 1, F_UY = 2, F_UZ = 3, F_T = 4, F_PHI = 5, F_DUX = 6, F_DUY = 7, F_DUZ = 8,
       F_COUNT = 9 };

// device counters: clamped U >= 0, non-finite / non-positive nodes, and nodes
// failing the stability pre-flight of lbm_init
struct Counters {
    unsigned long long clamps;
    unsigned long long bad;
    unsigned long long unstable;
    unsigned long long timeouts;   // fused step: a hand-off wait gave up (never expected)
};

template <typename R> __device__ __forceinline__ bool finite_pos(R v) { return v > R(0) && isfinite(v); }

// moments of one node from its 2Q populations, each sum in fixed k order.
// PAIRS: the library's pair layout; false: the set-major checkpoint layout.
template <int Q, typename S, typename R, bool PAIRS = true>
__device__ __forceinline__ void node_moments(const S* __restrict__ pop, long long nn, long long i,
                                             const KParams<R>& p, R& rho, R& jx, R& jy, R& jz, R& E) {
    using V = Vel<Q>;
    rho = R(0); jx = R(0); jy = R(0); jz = R(0); E = R(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const R sN = R(V::w(k)) * p.rho_ref, sG = R(V::w(k)) * p.E_ref;
        R f, h;
        if (PAIRS) {
            Store<S, R>::load2(pop, pair_index(k, nn, i), sN, sG, f, h);
        } else {
            f = Store<S, R>::load(pop, (size_t)k * nn + i, sN);
            h = Store<S, R>::load(pop, (size_t)(Q + k) * nn + i, sG);
        }
        rho += f;
        if (V::cx(k) == 1) jx += f; else if (V::cx(k) == -1) jx -= f;
        if (V::cy(k) == 1) jy += f; else if (V::cy(k) == -1) jy -= f;
        if (V::D == 3) { if (V::cz(k) == 1) jz += f; else if (V::cz(k) == -1) jz -= f; }
        E += h;
    }
}

// Layout conversion between the 2Q set-major checkpoint planes and the pair
// layout: element (s, k, n) moves between s Q nn + k nn + n and
// 2 (k nn + n) + s.  W is an unsigned word of the storage element's size.
template <typename W>
__global__ void __launch_bounds__(256) sets_to_pairs_kernel(const W* __restrict__ sets, W* __restrict__ pairs,
                                                            long long qnn) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < qnn; j += stride) {
        pairs[2 * j] = sets[j];
        pairs[2 * j + 1] = sets[qnn + j];
    }
}
template <typename W>
__global__ void __launch_bounds__(256) pairs_to_sets_kernel(const W* __restrict__ pairs, W* __restrict__ sets,
                                                            long long qnn) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < qnn; j += stride) {
        sets[j] = pairs[2 * j];
        sets[qnn + j] = pairs[2 * j + 1];
    }
}

// Step part 1: rho, u = j/rho, T = E/(rho c_v), Phi = sqrt(-(p - rho/3)).
// count != 0 adds clamped and non-physical nodes to the device counters.
template <int Q, typename S, typename R>
__global__ void __launch_bounds__(256) fields_kernel(const S* __restrict__ pop, R* __restrict__ fld,
                                                     KParams<R> p, Counters* cnt, int count) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nn) return;
    const long long nn = p.nn;
    R rho, jx, jy, jz, E;
    node_moments<Q, S, R>(pop, nn, i, p, rho, jx, jy, jz, E);
    R T = E / (rho * p.c_v);
    R U = fma(-rho, R(1.0 / 3.0), eos_pressure(p, rho, T));
    R Phi;
    if (U < R(0)) {
        Phi = sqrt(-U);
    } else {
        Phi = R(0);
        if (count) atomicAdd(&cnt->clamps, 1ull);
    }
    if (count && !(finite_pos(rho) && finite_pos(E))) atomicAdd(&cnt->bad, 1ull);
    fld[F_RHO * nn + i] = rho;
    fld[F_UX * nn + i] = jx / rho;
    fld[F_UY * nn + i] = jy / rho;
    if (Vel<Q>::D == 3) fld[F_UZ * nn + i] = jz / rho;
    fld[F_T * nn + i] = T;
    fld[F_PHI * nn + i] = Phi;
}

// node coordinates in 32-bit arithmetic (lbm_create keeps nn below 2^31)
__device__ __forceinline__ void node_xyz(long long i, int nx, int ny, int& x, int& y, int& z) {
    const unsigned ui = (unsigned)i;
    const unsigned r = ui / (unsigned)nx;
    x = (int)(ui - r * (unsigned)nx);
    y = (int)(r % (unsigned)ny);
    z = (int)(r / (unsigned)ny);
}

// Step part 2: F = (1/alpha)[A sum G Phi^2(x+e) e + (1-2A) Phi sum G Phi(x+e) e] + rho g,
// du = F/rho (Sec. 3, Eq. (edm)).  Beyond a wall Phi is read at the mirror node.
template <int Q, typename R>
__global__ void __launch_bounds__(256) force_kernel(R* __restrict__ fld, KParams<R> p) {
    using V = Vel<Q>;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nn) return;
    const long long nn = p.nn;
    int x, y, z;
    node_xyz(i, p.nx, p.ny, x, y, z);
    const R* Phi = fld + F_PHI * nn;
    R s1x = 0, s1y = 0, s1z = 0, s2x = 0, s2y = 0, s2z = 0;
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        Nb m = neighbour<V::D>(x, y, z, V::cx(k), V::cy(k), V::cz(k), p);
        R ph = Phi[m.n];
        R t1 = R(V::G(k)) * ph * ph;
        R t2 = R(V::G(k)) * ph;
        if (V::cx(k) == 1) { s1x += t1; s2x += t2; } else if (V::cx(k) == -1) { s1x -= t1; s2x -= t2; }
        if (V::cy(k) == 1) { s1y += t1; s2y += t2; } else if (V::cy(k) == -1) { s1y -= t1; s2y -= t2; }
        if (V::D == 3) {
            if (V::cz(k) == 1) { s1z += t1; s2z += t2; } else if (V::cz(k) == -1) { s1z -= t1; s2z -= t2; }
        }
    }
    const R rho = fld[F_RHO * nn + i];
    const R ph0 = Phi[i];
    const R a = p.A, b = R(1) - R(2) * p.A, inv_alpha = R(1.0 / V::alpha);
    fld[F_DUX * nn + i] = ((a * s1x + b * ph0 * s2x) * inv_alpha + rho * p.g[0]) / rho;
    fld[F_DUY * nn + i] = ((a * s1y + b * ph0 * s2y) * inv_alpha + rho * p.g[1]) / rho;
    if (V::D == 3) fld[F_DUZ * nn + i] = ((a * s1z + b * ph0 * s2z) * inv_alpha + rho * p.g[2]) / rho;
}

// Step part 3: dE (pressure work + conduction, Sec. 4 and Sec. 6.2), collision
// of both sets with the EDM and pseudoforce sources, push streaming.
template <int Q, typename S, typename R>
__global__ void __launch_bounds__(256) collide_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                      const R* __restrict__ fld, KParams<R> p) {
    using V = Vel<Q>;
    constexpr int D = V::D;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nn) return;
    const long long nn = p.nn;
    int x, y, z;
    node_xyz(i, p.nx, p.ny, x, y, z);

    const R rho = fld[F_RHO * nn + i];
    const R T = fld[F_T * nn + i];
    R u[3] = {fld[F_UX * nn + i], fld[F_UY * nn + i], D == 3 ? fld[F_UZ * nn + i] : R(0)};
    R du[3] = {fld[F_DUX * nn + i], fld[F_DUY * nn + i], D == 3 ? fld[F_DUZ * nn + i] : R(0)};

    // finite-difference energy change along every axis
    R div = R(0), cond = R(0);
    const R lc = conductivity(p, rho);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int ex = a == 0, ey = a == 1, ez = a == 2;
        Nb up = neighbour<D>(x, y, z, ex, ey, ez, p);
        Nb dn = neighbour<D>(x, y, z, -ex, -ey, -ez, p);
        R uu = fld[(F_UX + a) * nn + up.n] + fld[(F_DUX + a) * nn + up.n] / R(2);
        R ud = fld[(F_UX + a) * nn + dn.n] + fld[(F_DUX + a) * nn + dn.n] / R(2);
        if (up.g[a]) uu = -uu;   // across a wall of axis a the normal velocity flips
        if (dn.g[a]) ud = -ud;
        div += (uu - ud) / R(2);
        R Tu = fld[F_T * nn + up.n], Td = fld[F_T * nn + dn.n], Tw;
        if (up.g[a] && wall_T<D>(p, a, 1, Tw)) Tu = R(2) * Tw - Tu;
        if (dn.g[a] && wall_T<D>(p, a, 0, Tw)) Td = R(2) * Tw - Td;
        R lu = (lc + conductivity(p, fld[F_RHO * nn + up.n])) / R(2);
        R ld = (lc + conductivity(p, fld[F_RHO * nn + dn.n])) / R(2);
        cond += lu * (Tu - T) - ld * (T - Td);
    }
    R dE = R(0);
    if (p.pressure_work) dE += -eos_pressure(p, rho, T) * div;
    if (p.conduction) dE += cond;
    if (p.latent != R(0)) dE += latent_heat(p, rho, T, div);

    // the node's populations; its energy in the summation order of fields_kernel
    R fv[Q], hv[Q];
    R E = R(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        Store<S, R>::load2(src, pair_index(k, nn, i), R(V::w(k)) * p.rho_ref, R(V::w(k)) * p.E_ref, fv[k], hv[k]);
        E += hv[k];
    }
    const R dEoverE = dE / E;

    const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const R dsq = du[0] * (R(2) * u[0] + du[0]) + du[1] * (R(2) * u[1] + du[1]) + du[2] * (R(2) * u[2] + du[2]);
    const unsigned nbits = Store<S, R>::kStochastic ? node_bits(p.step, (unsigned)i) : 0u;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const R wk = R(V::w(k));
        const R cu = cdot<Q, R>(k, u[0], u[1], u[2]);
        const R cd = cdot<Q, R>(k, du[0], du[1], du[2]);
        const R e0 = wk * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
        const R de = wk * (R(3) * cd + R(4.5) * cd * (R(2) * cu + cd) - R(1.5) * dsq);
        const R f = fv[k], h = hv[k];
        const R fs = f + p.omega * (rho * e0 - f) + rho * de;
        R hs = h + p.omega_E * (E * e0 - h) + h * dEoverE;
        if (p.pseudoforce) hs += E * de;
        Nb m = neighbour<D>(x, y, z, V::cx(k), V::cy(k), V::cz(k), p);
        const int ko = m.ghost ? opposite(k) : k;
        const long long to = m.ghost ? i : m.n;
        Store<S, R>::store2(dst, pair_index(ko, nn, to), fs, hs, R(V::w(ko)) * p.rho_ref, R(V::w(ko)) * p.E_ref,
                            pair_word(nbits, k));
    }
}

// Initial state: N = rho e(u), g = rho eps e(u) (Eq. (feq)); counts nodes
// with rho <= 0, eps <= 0, non-finite input or U >= 0.
template <int Q, typename S, typename R>
__global__ void __launch_bounds__(256) init_kernel(S* __restrict__ pop, const double* __restrict__ rho_in,
                                                   const double* __restrict__ u_in,
                                                   const double* __restrict__ eps_in, KParams<R> p,
                                                   Counters* cnt) {
    using V = Vel<Q>;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nn) return;
    const long long nn = p.nn;
    const R rho = (R)rho_in[i];
    const R eps = (R)eps_in[i];
    R u[3] = {(R)u_in[i], (R)u_in[nn + i], V::D == 3 ? (R)u_in[2 * nn + i] : R(0)};
    const R E = rho * eps;
    const R T = eps / p.c_v;
    bool ok = finite_pos(rho) && finite_pos(eps) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
    if (ok) ok = fma(-rho, R(1.0 / 3.0), eos_pressure(p, rho, T)) < R(0);
    if (!ok) atomicAdd(&cnt->bad, 1ull);
    // stability pre-flight: (dp/drho)_T <= (h/dt)^2 + theta (Sec. 3) and the
    // explicit conduction limit chi dt/h^2 < 0.5/d (Sec. 6.1)
    if (ok) {
        const R Te = p.barotropic ? p.T0 : T;
        const R dpdrho = p.kappa * (R(24) * Te / ((R(3) - rho) * (R(3) - rho)) - R(6) * rho);
        const R chi = p.conduction ? conductivity(p, rho) / (rho * p.c_v) : R(0);
        if (dpdrho > R(4.0 / 3.0) || chi >= R(0.5) / R(V::D)) atomicAdd(&cnt->unstable, 1ull);
    }
    const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const unsigned nbits = Store<S, R>::kStochastic ? node_bits(p.step, (unsigned)i) : 0u;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const R wk = R(V::w(k));
        const R cu = cdot<Q, R>(k, u[0], u[1], u[2]);
        const R e0 = wk * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
        Store<S, R>::store2(pop, pair_index(k, nn, i), rho * e0, E * e0, wk * p.rho_ref, wk * p.E_ref,
                            pair_word(nbits, k));
    }
}

// Output fields after fields_kernel + force_kernel: rho, u* = u + du/2
// (Eq. (ustar)), T and P (EOS).
template <int Q, typename R>
__global__ void __launch_bounds__(256) output_kernel(const R* __restrict__ fld, KParams<R> p, double* rho,
                                                     double* u, double* T, double* P) {
    constexpr int D = Vel<Q>::D;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nn) return;
    const long long nn = p.nn;
    const R r = fld[F_RHO * nn + i], t = fld[F_T * nn + i];
    if (rho) rho[i] = (double)r;
    if (T) T[i] = (double)t;
    if (P) P[i] = (double)eos_pressure(p, r, t);
    if (u)
        for (int a = 0; a < D; ++a)
            u[a * nn + i] = (double)(fld[(F_UX + a) * nn + i] + fld[(F_DUX + a) * nn + i] / R(2));
}

// ---------------------------------------------------------------------------
// Conservation sums in FP64 with Kahan compensation.  Each thread walks a
// fixed strided set of nodes, blocks combine in a fixed shuffle tree and a
// single block sums the block partials in index order: bitwise reproducible
// for a fixed grid.

constexpr int kReduceBlocks = 1024;
constexpr int kReduceThreads = 256;
constexpr int kSums = 5;   // mass, momentum x, y, z, energy

// compensated (Kahan) summation in type T; the sum is s - c
template <typename T> struct KahanT {
    T s = T(0), c = T(0);
    __device__ void add(T v) {
        T y = v - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
using Kahan = KahanT<double>;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// PAIRS: populations in the library's pair layout; false: set-major planes
// (a checkpoint buffer, lbm_conservation_sums_noalloc)
template <int Q, typename S, typename R, bool PAIRS = true>
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const S* __restrict__ pop, KParams<R> p,
                                                                double* __restrict__ partials) {
    // Each thread sums the moments of its nodes (about nn / 262144 of them,
    // each formed in the arithmetic type as the step forms it) in FP64 with
    // Kahan compensation; the partials are combined in FP64 from here on, in
    // a fixed order, so the sums are FP64 and bitwise reproducible.
    Kahan acc[kSums];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.nn; i += stride) {
        R rho, jx, jy, jz, E;
        node_moments<Q, S, R, PAIRS>(pop, p.nn, i, p, rho, jx, jy, jz, E);
        acc[0].add((double)rho);
        acc[1].add((double)jx);
        acc[2].add((double)jy);
        acc[3].add((double)jz);
        acc[4].add((double)E);
    }
    __shared__ double sh[kSums][kReduceThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kSums; ++q) {
        double v = warp_sum(acc[q].s - acc[q].c);
        if (lane == 0) sh[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        Kahan b;
        for (int w = 0; w < kReduceThreads / 32; ++w) b.add(sh[threadIdx.x][w]);
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = b.s;
    }
}

static __global__ void __launch_bounds__(32) reduce_final_kernel(const double* __restrict__ partials, int nblocks,
                                                          double* __restrict__ out) {
    if (threadIdx.x < kSums) {
        Kahan b;
        for (int j = 0; j < nblocks; ++j) b.add(partials[(size_t)threadIdx.x * nblocks + j]);
        out[threadIdx.x] = b.s;
    }
}

}  // namespace lbm
