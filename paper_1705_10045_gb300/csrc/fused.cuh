// Fused one-launch time step of the thermal multiphase LB method
// (arXiv:1705.10045): every node's 2Q populations are read from HBM and its
// 2Q post-collision populations written once per step.
//
// Why a march: the energy change dE at x needs u* at x +- e_a, u* needs the
// force there, and the force needs Phi one node further out, so one step of a
// node depends on the moments of a 2-ring around it.  A CTA owns a TX x TY
// tile of the plane normal to the last lattice axis (z for D3Q19, y for D2Q9)
// and marches along that axis through a chunk of planes.  Per plane m it
//   M: loads the populations of the (TX+4) x (TY+4) ring region of plane m and
//      keeps rho, u, T, Phi in a 5-plane shared-memory ring buffer;
//   F: computes du = F/rho (Sec. 3 force + gravity) on the (TX+2) x (TY+2)
//      region of plane m-1 into a 3-plane buffer;
//   C: for the TX x TY nodes of plane m-2 forms dE by finite differences,
//      reloads the node's populations (an L2 hit: plane m-2 was read two
//      iterations earlier), collides N and g and pushes them to x + c_k.
// Ring nodes are recomputed by neighbouring CTAs from L2 rather than
// exchanged.  D2Q9 runs the same code as a lattice with one y node: its
// lattice y axis is the march axis and its tile is TX x 1.
//
// Index arithmetic is kept out of the inner loops: the wrapped ring
// coordinates of a CTA are tabulated once in shared memory, and each thread
// precomputes the +-1 node offsets of its own node along every axis.
#pragma once

#include "kernels.cuh"

namespace lbm {

// Velocity of direction k in march coordinates: (a, b) across the tile,
// m along the march axis.
template <int Q> struct MVel;
template <> struct MVel<9> {
    __host__ __device__ static constexpr int a(int k) { return Vel<9>::cx(k); }
    __host__ __device__ static constexpr int b(int) { return 0; }
    __host__ __device__ static constexpr int m(int k) { return Vel<9>::cy(k); }
};
template <> struct MVel<19> {
    __host__ __device__ static constexpr int a(int k) { return Vel<19>::cx(k); }
    __host__ __device__ static constexpr int b(int k) { return Vel<19>::cy(k); }
    __host__ __device__ static constexpr int m(int k) { return Vel<19>::cz(k); }
};

// Geometry of the march: na x nb tile plane (nb = 1 for D2Q9), nm planes.
struct MarchGeom {
    int na, nb, nm;
    int chunk;   // planes per CTA along the march axis
};

template <int TX, int TY> struct FusedShape {
    static constexpr int RB = TY > 1 ? 2 : 0;           // ring width across b (none for D2Q9)
    static constexpr int RW = TX + 4;                   // ring region width (a)
    static constexpr int RH = TY + 2 * RB;              // ring region height (b)
    static constexpr int R = RW * RH;
    static constexpr int FW = TX + 2;                   // force region
    static constexpr int FB = RB / 2;
    static constexpr int FH = TY + 2 * FB;
    static constexpr int F = FW * FH;
    static constexpr int kFields = 6;                   // Phi, rho, ua, ub, um, T
    template <typename R_> static constexpr size_t smem_bytes() {
        return sizeof(R_) * ((size_t)5 * kFields * R + (size_t)3 * 3 * F) + sizeof(int) * (RW + RH);
    }
};

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

template <int Q, typename S, typename R, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) fused_step_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                            KParams<R> p, MarchGeom G, Counters* cnt) {
    using V = Vel<Q>;
    using M = MVel<Q>;
    using Sh = FusedShape<TX, TY>;
    constexpr int NT = TX * TY;
    constexpr int RB = Sh::RB, RW = Sh::RW, RH = Sh::RH, R_ = Sh::R, FW = Sh::FW, FB = Sh::FB, F_ = Sh::F;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* fs = reinterpret_cast<R*>(smem_raw);               // [5][kFields][R_]
    R* dus = fs + 5 * Sh::kFields * R_;                    // [3][3][F_]
    int* ring_a = reinterpret_cast<int*>(dus + 3 * 3 * F_);   // wrapped a of ring column
    int* ring_b = ring_a + RW;                                // wrapped b * na of ring row

    const size_t nn = (size_t)p.nn;
    const int na = G.na, nb = G.nb, nm = G.nm;
    const int plane_n = na * nb;
    const int tid = threadIdx.x;
    const int a0 = blockIdx.x * TX, b0 = blockIdx.y * TY;
    const int zb = blockIdx.z * G.chunk;
    const int ze = min(zb + G.chunk, nm);
    const bool walls = p.wall;
    const R third = R(1.0 / 3.0);

    for (int i = tid; i < RW; i += NT) ring_a[i] = wrapi(a0 + i - 2, na);
    for (int i = tid; i < RH; i += NT) ring_b[i] = wrapi(b0 + i - RB, nb) * na;

    auto fld = [&](int slot, int f, int r) -> R& { return fs[((slot * Sh::kFields) + f) * R_ + r]; };
    auto du = [&](int slot, int c, int r) -> R& { return dus[(slot * 3 + c) * F_ + r]; };
    // Buffer slots are keyed by the unwrapped plane index the M stage loaded
    // (a periodic plane -1 holds the data of plane nm-1); across a wall a
    // stencil read goes to the mirror plane instead.
    auto mplane = [&](int m) -> int {
        if (!walls) return m;
        return m < 0 ? -1 - m : (m >= nm ? 2 * nm - 1 - m : m);
    };
    auto slot5 = [](int m) { return ((m % 5) + 5) % 5; };
    auto slot3 = [](int m) { return ((m % 3) + 3) % 3; };

    // this thread's node in the tile and its +-1 offsets along a and b
    const int ta = tid % TX, tb = tid / TX;
    const int ga = a0 + ta, gb = b0 + tb;
    const bool owns = ga < na && gb < nb;
    const int base_ab = gb * na + ga;
    const int dA_m = ga == 0 ? na - 1 : -1, dA_p = ga == na - 1 ? 1 - na : 1;
    const int dB_m = (gb == 0 ? nb - 1 : -1) * na, dB_p = (gb == nb - 1 ? 1 - nb : 1) * na;

    __syncthreads();

    for (int m = zb - 2; m < ze + 2; ++m) {
        // ---- M: moments of plane m on the ring region -------------------
        const bool m_real = walls ? (m >= 0 && m < nm) : true;
        if (m_real) {
            const int plane_off = wrapi(m, nm) * plane_n;
            const int sl = slot5(m);
            for (int r = tid; r < R_; r += NT) {
                const int ra = r % RW, rb = r / RW;
                const size_t n = (size_t)(plane_off + ring_b[rb] + ring_a[ra]);
                R fN[Q], fG[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    fN[k] = Store<S, R>::load(src, (size_t)k * nn + n, R(V::w(k)) * p.rho_ref);
                    fG[k] = Store<S, R>::load(src, (size_t)(Q + k) * nn + n, R(V::w(k)) * p.E_ref);
                }
                R rho = 0, ja = 0, jb = 0, jm = 0, E = 0;
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const R f = fN[k];
                    rho += f;
                    if (M::a(k) == 1) ja += f; else if (M::a(k) == -1) ja -= f;
                    if (M::b(k) == 1) jb += f; else if (M::b(k) == -1) jb -= f;
                    if (M::m(k) == 1) jm += f; else if (M::m(k) == -1) jm -= f;
                }
#pragma unroll
                for (int k = 0; k < Q; ++k) E += fG[k];
                const R T = E / (rho * p.c_v);
                const R U = eos_pressure(p, rho, T) - rho * third;
                fld(sl, 0, r) = U < R(0) ? sqrt(-U) : R(0);
                fld(sl, 1, r) = rho;
                fld(sl, 2, r) = ja / rho;
                fld(sl, 3, r) = jb / rho;
                fld(sl, 4, r) = jm / rho;
                fld(sl, 5, r) = T;
            }
        }
        __syncthreads();

        // ---- F: du = F/rho on the force region of plane f = m - 1 --------
        const int f = m - 1;
        const bool f_need = f >= zb - 1 && f <= ze && (walls ? (f >= 0 && f < nm) : true);
        if (f_need) {
            const int sl = slot5(f), sd = slot3(f);
            const int slm = slot5(mplane(f - 1)), slp = slot5(mplane(f + 1));
            const R A = p.A, B = R(1) - R(2) * p.A, inv_alpha = R(1.0 / V::alpha);
            const R g_a = p.g[0], g_b = Q == 9 ? R(0) : p.g[1], g_m = Q == 9 ? p.g[1] : p.g[2];
            for (int r = tid; r < F_; r += NT) {
                const int fa = r % FW, fb = r / FW;
                const int ra = fa + 1, rb = fb + (RB - FB);
                R s1a = 0, s1b = 0, s1m = 0, s2a = 0, s2b = 0, s2m = 0;
#pragma unroll
                for (int k = 1; k < Q; ++k) {
                    const int s = M::m(k) == 0 ? sl : (M::m(k) > 0 ? slp : slm);
                    const R ph = fld(s, 0, (rb + M::b(k)) * RW + ra + M::a(k));
                    const R t1 = R(V::G(k)) * ph * ph;
                    const R t2 = R(V::G(k)) * ph;
                    if (M::a(k) == 1) { s1a += t1; s2a += t2; } else if (M::a(k) == -1) { s1a -= t1; s2a -= t2; }
                    if (M::b(k) == 1) { s1b += t1; s2b += t2; } else if (M::b(k) == -1) { s1b -= t1; s2b -= t2; }
                    if (M::m(k) == 1) { s1m += t1; s2m += t2; } else if (M::m(k) == -1) { s1m -= t1; s2m -= t2; }
                }
                const int rc = rb * RW + ra;
                const R rho = fld(sl, 1, rc), ph0 = fld(sl, 0, rc);
                du(sd, 0, r) = ((A * s1a + B * ph0 * s2a) * inv_alpha + rho * g_a) / rho;
                du(sd, 1, r) = ((A * s1b + B * ph0 * s2b) * inv_alpha + rho * g_b) / rho;
                du(sd, 2, r) = ((A * s1m + B * ph0 * s2m) * inv_alpha + rho * g_m) / rho;
            }
        }
        __syncthreads();

        // ---- C: energy change, collision and push of plane c = m - 2 -----
        const int c = m - 2;
        if (c >= zb && c < ze && owns) {
            const int sl = slot5(c), sd = slot3(c);
            const int rc = (tb + RB) * RW + ta + 2;        // ring index of the node
            const int fc = (tb + FB) * FW + ta + 1;        // force-region index
            const R rho = fld(sl, 1, rc), T = fld(sl, 5, rc);
            const R u[3] = {fld(sl, 2, rc), fld(sl, 3, rc), fld(sl, 4, rc)};
            const R dv[3] = {du(sd, 0, fc), du(sd, 1, fc), du(sd, 2, fc)};

            // finite-difference dE along a, b and the march axis
            R div = 0, cond = 0;
            const R lc = conductivity(p, rho);
            {   // a: same plane, ring neighbours
                const R uu = fld(sl, 2, rc + 1) + du(sd, 0, fc + 1) / R(2);
                const R ud = fld(sl, 2, rc - 1) + du(sd, 0, fc - 1) / R(2);
                div += (uu - ud) / R(2);
                const R Tu = fld(sl, 5, rc + 1), Td = fld(sl, 5, rc - 1);
                const R lu = (lc + conductivity(p, fld(sl, 1, rc + 1))) / R(2);
                const R ld = (lc + conductivity(p, fld(sl, 1, rc - 1))) / R(2);
                cond += lu * (Tu - T) - ld * (T - Td);
            }
            if (Q == 19) {   // b: same plane
                const R uu = fld(sl, 3, rc + RW) + du(sd, 1, fc + FW) / R(2);
                const R ud = fld(sl, 3, rc - RW) + du(sd, 1, fc - FW) / R(2);
                div += (uu - ud) / R(2);
                const R Tu = fld(sl, 5, rc + RW), Td = fld(sl, 5, rc - RW);
                const R lu = (lc + conductivity(p, fld(sl, 1, rc + RW))) / R(2);
                const R ld = (lc + conductivity(p, fld(sl, 1, rc - RW))) / R(2);
                cond += lu * (Tu - T) - ld * (T - Td);
            }
            {   // march axis: neighbouring planes, or the node itself mirrored across a wall
                const bool gu = walls && c + 1 >= nm, gd = walls && c - 1 < 0;
                const int su = slot5(c + 1), sdn = slot5(c - 1), du_u = slot3(c + 1), du_d = slot3(c - 1);
                R uu, ud, Tu, Td, ru, rd;
                if (gu) {
                    uu = -(u[2] + dv[2] / R(2));
                    Tu = p.T_fixed_hi ? R(2) * p.T_hi - T : T;
                    ru = rho;
                } else {
                    uu = fld(su, 4, rc) + du(du_u, 2, fc) / R(2);
                    Tu = fld(su, 5, rc);
                    ru = fld(su, 1, rc);
                }
                if (gd) {
                    ud = -(u[2] + dv[2] / R(2));
                    Td = p.T_fixed_lo ? R(2) * p.T_lo - T : T;
                    rd = rho;
                } else {
                    ud = fld(sdn, 4, rc) + du(du_d, 2, fc) / R(2);
                    Td = fld(sdn, 5, rc);
                    rd = fld(sdn, 1, rc);
                }
                div += (uu - ud) / R(2);
                const R lu = (lc + conductivity(p, ru)) / R(2);
                const R ld = (lc + conductivity(p, rd)) / R(2);
                cond += lu * (Tu - T) - ld * (T - Td);
            }
            const R P = eos_pressure(p, rho, T);
            R dE = 0;
            if (p.pressure_work) dE += -P * div;
            if (p.conduction) dE += cond;
            if (P - rho * third >= R(0)) atomicAdd(&cnt->clamps, 1ull);

            const int n = c * plane_n + base_ab;
            R hv[Q];
            R E = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                hv[k] = Store<S, R>::load(src, (size_t)(Q + k) * nn + n, R(V::w(k)) * p.E_ref);
                E += hv[k];
            }
            if (!(finite_pos(rho) && finite_pos(E))) atomicAdd(&cnt->bad, 1ull);
            const R dEoverE = dE / E;

            // node offsets of x + c_k: +-1 along a and b (periodic), along the
            // march axis periodic or bounced at a wall
            const int dM_m = (c == 0 ? nm - 1 : -1) * plane_n, dM_p = (c == nm - 1 ? 1 - nm : 1) * plane_n;
            const bool wall_lo = walls && c == 0, wall_hi = walls && c == nm - 1;

            const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const R dsq = dv[0] * (R(2) * u[0] + dv[0]) + dv[1] * (R(2) * u[1] + dv[1]) +
                          dv[2] * (R(2) * u[2] + dv[2]);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const R wk = R(V::w(k));
                R cu = 0, cd = 0;
                if (M::a(k) == 1) { cu += u[0]; cd += dv[0]; } else if (M::a(k) == -1) { cu -= u[0]; cd -= dv[0]; }
                if (M::b(k) == 1) { cu += u[1]; cd += dv[1]; } else if (M::b(k) == -1) { cu -= u[1]; cd -= dv[1]; }
                if (M::m(k) == 1) { cu += u[2]; cd += dv[2]; } else if (M::m(k) == -1) { cu -= u[2]; cd -= dv[2]; }
                const R e0 = wk * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
                const R de = wk * (R(3) * cd + R(4.5) * cd * (R(2) * cu + cd) - R(1.5) * dsq);
                const R fv = Store<S, R>::load(src, (size_t)k * nn + n, wk * p.rho_ref);
                const R fo = fv + p.omega * (rho * e0 - fv) + rho * de;
                R ho = hv[k] + p.omega_E * (E * e0 - hv[k]) + hv[k] * dEoverE;
                if (p.pseudoforce) ho += E * de;
                // push to x + c_k, or bounce back at a wall on the march axis
                const bool bounce = (M::m(k) == -1 && wall_lo) || (M::m(k) == 1 && wall_hi);
                const int ko = bounce ? opposite(k) : k;
                int to = n;
                if (!bounce) {
                    if (M::a(k) == 1) to += dA_p; else if (M::a(k) == -1) to += dA_m;
                    if (M::b(k) == 1) to += dB_p; else if (M::b(k) == -1) to += dB_m;
                    if (M::m(k) == 1) to += dM_p; else if (M::m(k) == -1) to += dM_m;
                }
                // opposite directions share a weight, so the FP16 shift of slot ko is w_k ref
                Store<S, R>::store(dst, (size_t)ko * nn + to, fo, wk * p.rho_ref);
                Store<S, R>::store(dst, (size_t)(Q + ko) * nn + to, ho, wk * p.E_ref);
            }
        }
    }
}

}  // namespace lbm
