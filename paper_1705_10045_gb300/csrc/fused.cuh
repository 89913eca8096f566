// Fused one-launch time step of the thermal multiphase LB method
// (arXiv:1705.10045): every node's 2Q populations are read from HBM and its
// 2Q post-collision populations written once per step.
//
// Why a march: the energy change dE at x needs u* at x +- e_a, u* needs the
// force there, and the force needs Phi one node further out, so one step of a
// node depends on the moments of a 2-ring around it.  A CTA owns a TX x TY
// tile of the plane normal to the last lattice axis (z for D3Q19, y for D2Q9)
// and marches along that axis through a chunk of planes.  Three stages work
// on a plane each:
//   M: loads the populations of the (TX+4) x (TY+4) ring region of a plane,
//      keeps Phi on that region and rho, u, T on the (TX+2) x (TY+2) 1-ring
//      region in shared-memory plane buffers;
//   F: computes du = F/rho (Sec. 3 force + gravity) on the 1-ring region;
//   C: for the TX x TY nodes of a plane forms dE by finite differences,
//      reloads the node's populations (an L2 hit: the M stage read them a few
//      planes earlier), collides N and g and pushes them to x + c_k.
// The CTA is warp-specialised: producer warps run M on plane i and F on
// plane i-1 while consumer warps (one thread per tile node) run C on plane
// i-3 or later, so population loads overlap the collision arithmetic.  The
// two roles hand planes over through mbarriers in shared memory: producers
// release iteration i when M(i) and F(i-1) are done, and consumers release
// plane c when C(c) has read its buffers, which the producers wait for before
// overwriting them.  Neither role waits for the other's whole iteration, so a
// slow plane on one side does not stall the other.  A named barrier orders M
// before F, and F before the next M, inside the producer warps.  Ring nodes are recomputed by neighbouring
// CTAs from L2 rather than exchanged.  D2Q9 runs the same code as a lattice
// with one y node: its lattice y axis is the march axis and its tile is
// TX x 1.
//
// Index arithmetic is kept out of the inner loops: the wrapped ring
// coordinates of a CTA are tabulated once in shared memory, and each
// consumer thread precomputes the +-1 node offsets of its node along every
// axis.  The force stencil and the collision work on opposite-direction pairs
// (c_{k+1} = -c_k), which share the even part of every term.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace lbm {

// mbarrier helpers of the producer/consumer hand-off (shared memory, CTA scope)
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// Wait until the phase of parity `parity` of *b has completed, for at most
// about half a second (1e9 clock cycles); false when the wait gave up.  Each
// try_wait may suspend the warp for up to kWaitHintNs nanoseconds; it resumes
// as soon as the phase completes, so the hint bounds how often a waiting warp
// polls (and takes issue slots from the working warps), not its latency.
#ifndef LBM_WAIT_HINT_NS
#define LBM_WAIT_HINT_NS 20000
#endif
constexpr unsigned kWaitHintNs = LBM_WAIT_HINT_NS;

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned done;
    if (kWaitHintNs > 0) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(b)), "r"(parity), "n"(kWaitHintNs)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(b)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
    if (mbar_try_wait(b, parity)) return true;
    const long long t0 = clock64();
    do {
        if (mbar_try_wait(b, parity)) return true;
    } while (clock64() - t0 < 1000000000ll);
    return false;
}

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
    int chunk;        // planes per CTA along the march axis
    int m_lo, m_hi;   // planes whose collision the launch runs (the moment and
                      // force stages reach two and one planes beyond them)
};

// Plane buffers: Phi for 3 planes, rho/u/T for 5 planes, du for 4 planes
// (the consumer trails the producer by three planes).  SPLIT: the consumers
// form the moments of their own nodes three planes ahead, which takes one
// more rho/u/T plane and a third mbarrier ring.
template <int TX, int TY, bool SPLIT = false> struct FusedShape {
    static constexpr int RB = TY > 1 ? 2 : 0;           // ring width across b (none for D2Q9)
    static constexpr int RW = TX + 4;                   // 2-ring region (Phi)
    static constexpr int RH = TY + 2 * RB;
    static constexpr int R = RW * RH;
    static constexpr int FB = RB / 2;                   // 1-ring region (rho, u, T, du)
    static constexpr int FW = TX + 2;
    static constexpr int FH = TY + 2 * FB;
    static constexpr int F = FW * FH;
    static constexpr int kRut = 5;                      // rho, ua, ub, um, T
    static constexpr int kPhiSlots = 3, kRutSlots = SPLIT ? 6 : 5, kDuSlots = 4;
    static constexpr int kHandSlots = 8;   // mbarrier ring of the producer/consumer hand-off
    static constexpr int kRings = SPLIT ? 3 : 2;
    // ring nodes outside the tile: RB full rows above and below, 2 columns
    // left and right of each tile row
    static constexpr int kBorder = 2 * RB * RW + 4 * TY;
    template <typename R_> static constexpr size_t table_offset() {
        return sizeof(R_) * ((size_t)kPhiSlots * R + (size_t)kRutSlots * kRut * F + (size_t)kDuSlots * 3 * F);
    }
    template <typename R_> static constexpr size_t barrier_offset() {
        return (table_offset<R_>() + sizeof(int) * (RW + RH) + 7) & ~(size_t)7;
    }
    // plane buffers, ring tables, kRings x kHandSlots mbarriers and an abort flag
    template <typename R_> static constexpr size_t smem_bytes() {
        return barrier_offset<R_>() + 8 * (kRings * kHandSlots + 1);
    }
    // ring index of border node q < kBorder
    __device__ static int border_ring(int q) {
        if (q < 2 * RB * RW) {
            const int row = q / RW;
            return (row < RB ? row : row + TY) * RW + q % RW;
        }
        const int q2 = q - 2 * RB * RW, c = q2 & 3;
        return (RB + (q2 >> 2)) * RW + (c < 2 ? c : c + TX);
    }
};

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ int slotn(int m, int n) { return ((m % n) + n) % n; }

// Coordinate of a ring row or column: wrapped on a periodic axis, the mirror
// node across a wall (clamped into the axis for ring nodes of a ragged tile
// that lie further out; their values are never used).
__device__ __forceinline__ int ring_coord(int i, int n, int walled) {
    if (!walled) return wrapi(i, n);
    if (i < 0) i = -1 - i;
    if (i >= n) i = 2 * n - 1 - i;
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Walls beside tile-plane node (ga, gb): bit 0 / 1 the low / high wall of axis
// a (x), bit 2 / 3 of axis b (y of D3Q19).
template <typename R>
__device__ __forceinline__ int wall_edges(const KParams<R>& p, int Q, int ga, int gb, int na, int nb) {
    int e = 0;
    if (p.wall_x) e |= (ga == 0 ? 1 : 0) | (ga == na - 1 ? 2 : 0);
    if (Q == 19 && p.wall_y) e |= (gb == 0 ? 4 : 0) | (gb == nb - 1 ? 8 : 0);
    return e;
}

// COH: read the populations through coherent loads (the persistent batch
// kernel reads, in one launch, buffers that other CTAs wrote earlier in it).
template <int Q, typename S, typename R, int TX, int TY, bool COH = false, bool SPLIT = false> struct FusedStages {
    using V = Vel<Q>;
    using M = MVel<Q>;
    using Sh = FusedShape<TX, TY, SPLIT>;
    static constexpr int RB = Sh::RB, RW = Sh::RW, RH = Sh::RH, R_ = Sh::R, FW = Sh::FW, FB = Sh::FB, F_ = Sh::F;

    R* phis;     // [kPhiSlots][R_]
    R* ruts;     // [kRutSlots][kRut][F_]
    R* dus;      // [kDuSlots][3][F_]
    int* ring_a; // wrapped a of ring column
    int* ring_b; // wrapped b * na of ring row
    const S* __restrict__ src;
    S* __restrict__ dst;
    const KParams<R>* p;
    MarchGeom G;
    size_t nn;
    int plane_n;
    unsigned step;   // step counter of this launch (seeds FP16 stochastic rounding)

    // the pair (N_k, g_k) at pair index i of q.  With shifted storage (FP16)
    // the stages work on the stored values N_k - w_k rho_ref, g_k - w_k E_ref
    // themselves: the moments add rho_ref and E_ref once, and the collision
    // writes shifted values (see c_stage), so no value is shifted on its own.
    static constexpr bool kSh = Store<S, R>::kShifted;
    __device__ static void ld2(const S* q, size_t i, R sN, R sG, R& a, R& b) {
        if constexpr (kSh) {
            if (COH) Store<S, R>::load2_coh_raw(q, i, a, b);
            else Store<S, R>::load2_raw(q, i, a, b);
        } else {
            if (COH) Store<S, R>::load2_coh(q, i, sN, sG, a, b);
            else Store<S, R>::load2(q, i, sN, sG, a, b);
        }
    }
    __device__ static void ld2_last(const S* q, size_t i, R sN, R sG, R& a, R& b) {
        if constexpr (kSh) {
            if (COH) Store<S, R>::load2_last_coh_raw(q, i, a, b);
            else Store<S, R>::load2_last_raw(q, i, a, b);
        } else {
            if (COH) Store<S, R>::load2_last_coh(q, i, sN, sG, a, b);
            else Store<S, R>::load2_last(q, i, sN, sG, a, b);
        }
    }
    __device__ R& phi(int slot, int r) const { return phis[slot * R_ + r]; }
    __device__ R& rut(int slot, int f, int r) const { return ruts[(slot * Sh::kRut + f) * F_ + r]; }
    __device__ R& du(int slot, int c, int r) const { return dus[(slot * 3 + c) * F_ + r]; }
    // Buffer slots are keyed by the unwrapped plane index the M stage loaded
    // (a periodic plane -1 holds the data of plane nm-1); across a wall a
    // stencil read goes to the mirror plane instead.
    __device__ int mplane(int m) const {
        if (!p->wall) return m;
        return m < 0 ? -1 - m : (m >= G.nm ? 2 * G.nm - 1 - m : m);
    }

    // M: moments of plane m on the ring region, ring nodes t, t + nt, ...
    __device__ void m_stage(int m, int t, int nt) const {
        const int plane_off = wrapi(m, G.nm) * plane_n;
        const int sp = slotn(m, Sh::kPhiSlots), sr = slotn(m, Sh::kRutSlots);
        for (int r = t; r < R_; r += nt) m_node(plane_off, sp, sr, r);
    }
    // the same for the border nodes only (SPLIT: the consumers take the tile)
    __device__ void m_border(int m, int t, int nt) const {
        const int plane_off = wrapi(m, G.nm) * plane_n;
        const int sp = slotn(m, Sh::kPhiSlots), sr = slotn(m, Sh::kRutSlots);
        for (int q = t; q < Sh::kBorder; q += nt) m_node(plane_off, sp, sr, Sh::border_ring(q));
    }
    // the moments of tile node (ta, tb) of plane m
    __device__ void m_interior(int m, int ta, int tb) const {
        m_node<true>(wrapi(m, G.nm) * plane_n, slotn(m, Sh::kPhiSlots), slotn(m, Sh::kRutSlots),
                     (tb + RB) * RW + ta + 2);
    }
    // Phi of ring node r, and rho, u, T if r lies in the 1-ring region.
    // KEEP: the node is the caller's own, reloaded by its C stage three
    // planes later, so its lines get the L2 evict-last hint.
    template <bool KEEP = false>
    __device__ __forceinline__ void m_node(int plane_off, int sp, int sr, int r) const {
        {
            const int ra = r % RW, rb = r / RW;
            const size_t n = (size_t)(plane_off + ring_b[rb] + ring_a[ra]);
            if constexpr (kSh) {
                // shifted FP16 storage: the sums take the halves of the pair
                // words directly (the same values as widening them first)
                using H = Store<S, R>;
                unsigned w[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k)
                    w[k] = COH ? H::word_coh(src, pair_index(k, nn, n)) : H::word(src, pair_index(k, nn, n));
                R rho = H::lo(w[0]), ja = R(0), jb = R(0), jm = R(0), E = H::hi(w[0]);
                bool new_a = true, new_b = true, new_m = true;
#pragma unroll
                for (int k = 1; k < Q; k += 2) {
                    const R x = H::lo(w[k]);
                    const R s = H::add_lo(w[k + 1], x), dn = H::sub_lo(w[k + 1], x);   // x + y and y - x
                    rho += s;
                    if (M::a(k) != 0) { const R t = M::a(k) > 0 ? -dn : dn; ja = new_a ? t : ja + t; new_a = false; }
                    if (M::b(k) != 0) { const R t = M::b(k) > 0 ? -dn : dn; jb = new_b ? t : jb + t; new_b = false; }
                    if (M::m(k) != 0) { const R t = M::m(k) > 0 ? -dn : dn; jm = new_m ? t : jm + t; new_m = false; }
                }
#pragma unroll
                for (int k = 1; k < Q; ++k) E = H::add_hi(w[k], E);
                // sums of shifted values: sum_k w_k = 1, sum_k w_k c_k = 0
                rho += p->rho_ref;
                E += p->E_ref;
                m_finish(sp, sr, r, rho, ja, jb, jm, E);
                return;
            } else {
                R fN[Q], fG[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k)
                    if (KEEP && !COH)
                        Store<S, R>::load2_keep(src, pair_index(k, nn, n), R(V::w(k)) * p->rho_ref,
                                                R(V::w(k)) * p->E_ref, fN[k], fG[k]);
                    else
                        ld2(src, pair_index(k, nn, n), R(V::w(k)) * p->rho_ref, R(V::w(k)) * p->E_ref, fN[k], fG[k]);
                // opposite directions k, k+1 pair up: their sum enters rho, their
                // difference the momentum along c_k (each sum starts at its
                // first term)
                R rho = fN[0], ja = R(0), jb = R(0), jm = R(0), E = fG[0];
                bool new_a = true, new_b = true, new_m = true;
#pragma unroll
                for (int k = 1; k < Q; k += 2) {
                    const R s = fN[k] + fN[k + 1], d = fN[k] - fN[k + 1];
                    rho += s;
                    if (M::a(k) != 0) { const R t = M::a(k) > 0 ? d : -d; ja = new_a ? t : ja + t; new_a = false; }
                    if (M::b(k) != 0) { const R t = M::b(k) > 0 ? d : -d; jb = new_b ? t : jb + t; new_b = false; }
                    if (M::m(k) != 0) { const R t = M::m(k) > 0 ? d : -d; jm = new_m ? t : jm + t; new_m = false; }
                }
#pragma unroll
                for (int k = 1; k < Q; ++k) E += fG[k];
                m_finish(sp, sr, r, rho, ja, jb, jm, E);
            }
        }
    }
    // Phi of ring node r from its moments, and rho, u, T if r lies in the
    // 1-ring region
    __device__ __forceinline__ void m_finish(int sp, int sr, int r, R rho, R ja, R jb, R jm, R E) const {
        const R third = R(1.0 / 3.0);
        const int ra = r % RW, rb = r / RW;
        const R T = E / (rho * p->c_v);
        const R U = fma(-rho, third, eos_pressure(*p, rho, T));
        phi(sp, r) = U < R(0) ? sqrt(-U) : R(0);
        const int fa = ra - 1, fb = rb - (RB - FB);
        if (fa >= 0 && fa < FW && fb >= 0 && fb < Sh::FH) {
            const int f = fb * FW + fa;
            const R inv_rho = R(1) / rho;
            rut(sr, 0, f) = rho;
            rut(sr, 1, f) = ja * inv_rho;
            rut(sr, 2, f) = jb * inv_rho;
            rut(sr, 3, f) = jm * inv_rho;
            rut(sr, 4, f) = T;
        }
    }

    // F: du = F/rho on the 1-ring region of plane f, region nodes t, t + nt, ...
    __device__ void f_stage(int f, int t, int nt) const {
        const int sp0 = slotn(f, Sh::kPhiSlots), spm = slotn(mplane(f - 1), Sh::kPhiSlots),
                  spp = slotn(mplane(f + 1), Sh::kPhiSlots);
        const int sr = slotn(f, Sh::kRutSlots), sd = slotn(f, Sh::kDuSlots);
        const R A = p->A, B = R(1) - R(2) * p->A, inv_alpha = R(1.0 / V::alpha);
        const R gv[3] = {p->g[0], Q == 9 ? R(0) : p->g[1], Q == 9 ? p->g[1] : p->g[2]};
        const R G2 = R(V::G(Q - 1));   // next-nearest weight (1/4 or 1/2)
        for (int r = t; r < F_; r += nt) {
            const int ra = r % FW + 1, rb = r / FW + (RB - FB);
            // opposite directions pair up: G Phi(x+e) e + G Phi(x-e)(-e) = G (Phi+ - Phi-) e,
            // and the Phi^2 term is G (Phi+ - Phi-)(Phi+ + Phi-) e
            R n1[3] = {0, 0, 0}, n2[3] = {0, 0, 0}, q1[3] = {0, 0, 0}, q2[3] = {0, 0, 0};
#pragma unroll
            for (int k = 1; k < Q; k += 2) {
                const int s_p = M::m(k) == 0 ? sp0 : (M::m(k) > 0 ? spp : spm);
                const int s_m = M::m(k) == 0 ? sp0 : (M::m(k) > 0 ? spm : spp);
                const R pp = phi(s_p, (rb + M::b(k)) * RW + ra + M::a(k));
                const R pm = phi(s_m, (rb - M::b(k)) * RW + ra - M::a(k));
                const R d = pp - pm, sum = pp + pm;
                const bool nearest = M::a(k) * M::a(k) + M::b(k) * M::b(k) + M::m(k) * M::m(k) == 1;
                R* s1 = nearest ? n1 : q1;
                R* s2 = nearest ? n2 : q2;
                // s1 += +-d (Phi+ + Phi-) as one fused multiply-add per axis
                if (M::a(k) == 1) { s1[0] = fma(d, sum, s1[0]); s2[0] += d; }
                else if (M::a(k) == -1) { s1[0] = fma(-d, sum, s1[0]); s2[0] -= d; }
                if (M::b(k) == 1) { s1[1] = fma(d, sum, s1[1]); s2[1] += d; }
                else if (M::b(k) == -1) { s1[1] = fma(-d, sum, s1[1]); s2[1] -= d; }
                if (M::m(k) == 1) { s1[2] = fma(d, sum, s1[2]); s2[2] += d; }
                else if (M::m(k) == -1) { s1[2] = fma(-d, sum, s1[2]); s2[2] -= d; }
            }
            const R rho = rut(sr, 0, r), ph0 = phi(sp0, rb * RW + ra);
            const R scale = inv_alpha / rho, Bph0 = B * ph0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const R s1 = fma(G2, q1[a], n1[a]), s2 = fma(G2, q2[a], n2[a]);
                du(sd, a, r) = fma(fma(A, s1, Bph0 * s2), scale, gv[a]);
            }
        }
    }

    // C: energy change, collision and push of the node (ta, tb) of plane c.
    // edge: walls next to the node across the tile plane (bit 0 / 1: the low /
    // high wall of axis a, bit 2 / 3: of axis b), from wall_edges().
    // XW: the domain may have walls on the tile-plane axes (false: edge is 0
    // and the wall handling across the tile compiles away).
    template <bool XW>
    __device__ void c_stage(int c, int ta, int tb, int n_ab, int dA_m, int dA_p, int dB_m, int dB_p, int edge_in,
                            Counters* cnt) const {
        const int edge = XW ? edge_in : 0;
        const bool walls = p->wall;
        const int nm = G.nm;
        const R third = R(1.0 / 3.0);
        // the node's populations first: their loads are in flight while the
        // finite differences below read shared memory.  The reload is the last
        // use of these lines on this SM, so it does not allocate them in L1.
        // The pointer walks from one direction's pair array to the next.
        // With shifted FP16 storage the reload stays packed (one 32-bit word
        // per pair, half the registers) and each half is widened where it is
        // used.
        const int n = c * plane_n + n_ab;
        R fv[Q], hv[Q];
        unsigned wv[Q];
        {
            const S* q = src + 2 * (size_t)n;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                if constexpr (kSh) wv[k] = COH ? Store<S, R>::word_last_coh(q, 0) : Store<S, R>::word_last(q, 0);
                else ld2_last(q, 0, R(V::w(k)) * p->rho_ref, R(V::w(k)) * p->E_ref, fv[k], hv[k]);
                q += 2 * nn;
            }
        }
        auto fvk = [&](int k) -> R {   // N_k (stored, shifted value with FP16)
            if constexpr (kSh) return __half2float(__ushort_as_half((unsigned short)(wv[k] & 0xFFFFu)));
            else return fv[k];
        };
        auto hvk = [&](int k) -> R {   // g_k
            if constexpr (kSh) return __half2float(__ushort_as_half((unsigned short)(wv[k] >> 16)));
            else return hv[k];
        };
        const int sr = slotn(c, Sh::kRutSlots), sd = slotn(c, Sh::kDuSlots);
        const int fc = (tb + FB) * FW + ta + 1;        // 1-ring index of the node
        const R rho = rut(sr, 0, fc), T = rut(sr, 4, fc);
        const R u[3] = {rut(sr, 1, fc), rut(sr, 2, fc), rut(sr, 3, fc)};
        const R dv[3] = {du(sd, 0, fc), du(sd, 1, fc), du(sd, 2, fc)};

        // finite-difference dE along a, b and the march axis (Sec. 4, Sec. 6.2)
        R div = 0, cond = 0;
        const R lc = conductivity(*p, rho), half_lc = lc * R(0.5);
        // one axis of the differences; g: bit 0 / 1 the low / high neighbour is
        // the ghost beyond a wall, whose values are then own_u (normal
        // velocity), T_lo / T_hi and the node's own density
        auto axis = [&](R uu, R ud, R Tu, R Td, R ru, R rd, int g = 0, R own_u = R(0), R T_lo = R(0),
                        R T_hi = R(0)) {
            if (g) {
                if (g & 2) { uu = own_u; Tu = T_hi; ru = rho; }
                if (g & 1) { ud = own_u; Td = T_lo; rd = rho; }
            }
            div = fma(uu - ud, R(0.5), div);
            // face conductivities, the mean of the two nodes'
            const R lu = fma(conductivity(*p, ru), R(0.5), half_lc);
            const R ld = fma(conductivity(*p, rd), R(0.5), half_lc);
            cond = fma(-ld, T - Td, fma(lu, Tu - T, cond));
        };
        // axes across the tile: neighbouring ring nodes, or (only for nodes
        // beside a wall) the node itself mirrored across it: normal velocity
        // negated, T mirrored or reflected about the wall temperature
        axis(fma(du(sd, 0, fc + 1), R(0.5), rut(sr, 1, fc + 1)), fma(du(sd, 0, fc - 1), R(0.5), rut(sr, 1, fc - 1)),
             rut(sr, 4, fc + 1), rut(sr, 4, fc - 1), rut(sr, 0, fc + 1), rut(sr, 0, fc - 1), edge & 3,
             -fma(dv[0], R(0.5), u[0]), p->T_fixed_x[0] ? R(2) * p->T_x[0] - T : T,
             p->T_fixed_x[1] ? R(2) * p->T_x[1] - T : T);
        if (Q == 19)
            axis(fma(du(sd, 1, fc + FW), R(0.5), rut(sr, 2, fc + FW)), fma(du(sd, 1, fc - FW), R(0.5), rut(sr, 2, fc - FW)),
                 rut(sr, 4, fc + FW), rut(sr, 4, fc - FW), rut(sr, 0, fc + FW), rut(sr, 0, fc - FW), (edge >> 2) & 3,
                 -fma(dv[1], R(0.5), u[1]), p->T_fixed_y[0] ? R(2) * p->T_y[0] - T : T,
                 p->T_fixed_y[1] ? R(2) * p->T_y[1] - T : T);
        {   // march axis: neighbouring planes, or the node itself mirrored across a wall
            const bool gu = walls && c + 1 >= nm, gd = walls && c - 1 < 0;
            const int su = slotn(c + 1, Sh::kRutSlots), sdn = slotn(c - 1, Sh::kRutSlots);
            const int du_u = slotn(c + 1, Sh::kDuSlots), du_d = slotn(c - 1, Sh::kDuSlots);
            const R own = -fma(dv[2], R(0.5), u[2]);
            const R uu = gu ? own : fma(du(du_u, 2, fc), R(0.5), rut(su, 3, fc));
            const R ud = gd ? own : fma(du(du_d, 2, fc), R(0.5), rut(sdn, 3, fc));
            const R Tu = gu ? (p->T_fixed_hi ? R(2) * p->T_hi - T : T) : rut(su, 4, fc);
            const R Td = gd ? (p->T_fixed_lo ? R(2) * p->T_lo - T : T) : rut(sdn, 4, fc);
            const R ru = gu ? rho : rut(su, 0, fc);
            const R rd = gd ? rho : rut(sdn, 0, fc);
            axis(uu, ud, Tu, Td, ru, rd);
        }
        const R P = eos_pressure(*p, rho, T);
        R dE = 0;
        if (p->pressure_work) dE += -P * div;
        if (p->conduction) dE += cond;
        if (p->latent != R(0)) dE += latent_heat(*p, rho, T, div);
        if (fma(-rho, third, P) >= R(0)) atomicAdd(&cnt->clamps, 1ull);

        R E = hvk(0);
        if constexpr (kSh) {
#pragma unroll
            for (int k = 1; k < Q; ++k) E = Store<S, R>::add_hi(wv[k], E);
            E += p->E_ref;
        } else {
#pragma unroll
            for (int k = 1; k < Q; ++k) E += hvk(k);
        }
        if (!(finite_pos(rho) && finite_pos(E))) atomicAdd(&cnt->bad, 1ull);
        const R dEoverE = dE / E;
        // node offsets of x + c_k: +-1 along a and b (periodic), along the
        // march axis periodic or bounced at a wall
        const int dM_m = (c == 0 ? nm - 1 : -1) * plane_n, dM_p = (c == nm - 1 ? 1 - nm : 1) * plane_n;
        const bool wall_lo = walls && c == 0, wall_hi = walls && c == nm - 1;
        const bool edge_a_lo = edge & 1, edge_a_hi = edge & 2, edge_b_lo = edge & 4, edge_b_hi = edge & 8;

        // Collision, Eq. (lbe)/(edm)/(gk), written per node as
        //   N*_k = (1 - omega) N_k + rho (omega e0_k + de_k)
        //   g*_k = (1 - omega_E + dE/E) g_k + E (omega_E e0_k + [pseudoforce] de_k)
        // with e0 = N^eq(rho,u)/rho and de = (N^eq(rho,u+du) - N^eq(rho,u))/rho.
        // With v = u + du, s = c_k.u and t = c_k.v, Eq. (feq) gives
        //   e0_k = w_k (b0 + 4.5 s^2 + 3 s),   de_k = w_k (db + 4.5 (t^2 - s^2) + 3 (t - s))
        // (b0 = 1 - 1.5 u.u, db = -1.5 (v.v - u.u) = -1.5 du.(2u + du)), so
        //   rho (omega e0_k + de_k) = w_k K + 4.5 w_k [P s^2 + rho t^2] + 3 w_k [P s + rho t]
        // with K = rho omega b0 + rho db and P = rho omega - rho; the same holds
        // for g with (E omega_E, E_pf) in place of (rho omega, rho).  Opposite
        // directions k, k+1 (c -> -c) share the even part and flip the odd one.
        // The factors w K, 4.5 w P, ... are formed once for the nearest
        // directions and scaled by w2/w1 (1/2 on D3Q19, 1/4 on D2Q9: exact) for
        // the next-nearest.  Products that feed a sum are written as explicit
        // fused multiply-adds, so every kernel that runs this code rounds them
        // the same way.
        const R usq = fma(u[0], u[0], fma(u[1], u[1], u[2] * u[2]));
        const R dsq = fma(dv[0], fma(R(2), u[0], dv[0]), fma(dv[1], fma(R(2), u[1], dv[1]), dv[2] * fma(R(2), u[2], dv[2])));
        const R base0 = fma(R(-1.5), usq, R(1)), dbase = R(-1.5) * dsq;
        const R om = p->omega, omE = p->omega_E;
        const R fN = R(1) - om, fG = R(1) - omE + dEoverE;
        const R rho_om = rho * om, E_omE = E * omE, E_pf = p->pseudoforce ? E : R(0);
        // shifted storage: with N_k = N'_k + w_k rho_ref and g_k = g'_k + w_k E_ref
        //   N*'_k = (1 - omega) N'_k + rho (omega e0_k + de_k) - omega w_k rho_ref
        //   g*'_k = fG g'_k + E (omega_E e0_k + [pf] de_k) + (fG - 1) w_k E_ref
        // so the shifts enter K as nsh and gsh
        const R nsh = kSh ? -om * p->rho_ref : R(0), gsh = kSh ? (fG - R(1)) * p->E_ref : R(0);
        const R KN = kSh ? fma(rho_om, base0, fma(rho, dbase, nsh)) : fma(rho_om, base0, rho * dbase);
        const R KG = kSh ? fma(E_omE, base0, fma(E_pf, dbase, gsh)) : fma(E_omE, base0, E_pf * dbase);
        const R PN = rho_om - rho, PG = E_omE - E_pf;
        const R v[3] = {u[0] + dv[0], u[1] + dv[1], u[2] + dv[2]};
        const unsigned nbits = Store<S, R>::kStochastic ? node_bits(step, (unsigned)n) : 0u;
        S* dk = dst + 2 * (size_t)n;        // pair k of the node's slot (walks over k)
        // the collision and push, instantiated once for planes next to a wall
        // (WALL: some directions bounce back) and once for all other planes
        auto collide = [&](auto wall_tag) {
            constexpr bool WALL = decltype(wall_tag)::value;
            // a: rho (omega e0 + de), b: E (omega_E e0 + [pseudoforce] de) of direction k
            auto emit = [&](int k, R a, R b, R fv, R hvk) {
                const R fo = fma(fv, fN, a);
                const R ho = fma(hvk, fG, b);
                // push to x + c_k, or bounce back at a wall on the march axis
                const bool bounce = WALL && ((M::m(k) == -1 && wall_lo) || (M::m(k) == 1 && wall_hi) ||
                                             (M::a(k) == -1 && edge_a_lo) || (M::a(k) == 1 && edge_a_hi) ||
                                             (M::b(k) == -1 && edge_b_lo) || (M::b(k) == 1 && edge_b_hi));
                int to = 0;
                if (M::a(k) == 1) to += dA_p; else if (M::a(k) == -1) to += dA_m;
                if (M::b(k) == 1) to += dB_p; else if (M::b(k) == -1) to += dB_m;
                if (M::m(k) == 1) to += dM_p; else if (M::m(k) == -1) to += dM_m;
                // opposite directions share a weight, so the FP16 shift of slot ko is w_k ref
                const R wk = R(V::w(k));
                const unsigned t = Store<S, R>::kStochastic ? pair_word(nbits, k) : 0u;
                const long long off = bounce ? (long long)(opposite(k) - k) * (long long)nn : (long long)to;
                if constexpr (kSh) Store<S, R>::store2_raw(dk + 2 * off, 0, fo, ho, t);
                else Store<S, R>::store2(dk + 2 * off, 0, fo, ho, wk * p->rho_ref, wk * p->E_ref, t);
                dk += 2 * nn;
            };
            emit(0, R(V::w(0)) * KN, R(V::w(0)) * KG, fvk(0), hvk(0));
            constexpr double w1 = V::w(1);
            R kn = R(w1) * KN, kg = R(w1) * KG;
            R pn = R(4.5 * w1) * PN, qn = R(4.5 * w1) * rho, pg = R(4.5 * w1) * PG, qg = R(4.5 * w1) * E_pf;
            R rn = R(3.0 * w1) * PN, sn = R(3.0 * w1) * rho, rg = R(3.0 * w1) * PG, sg = R(3.0 * w1) * E_pf;
#pragma unroll
            for (int k = 1; k < Q; k += 2) {
                if (k == (Q == 19 ? 7 : 5)) {   // first next-nearest direction
                    const R h = R(V::w(Q - 1) / w1);
                    kn *= h; kg *= h; pn *= h; qn *= h; pg *= h; qg *= h; rn *= h; sn *= h; rg *= h; sg *= h;
                }
                // s = c_k.u and t = c_k.v, each summed from its first term
                R s = R(0), t = R(0);
                bool first = true;
                auto add = [&](int cc, R x, R y) {
                    if (cc == 0) return;
                    const R xs = cc > 0 ? x : -x, ys = cc > 0 ? y : -y;
                    s = first ? xs : s + xs;
                    t = first ? ys : t + ys;
                    first = false;
                };
                add(M::a(k), u[0], v[0]);
                add(M::b(k), u[1], v[1]);
                add(M::m(k), u[2], v[2]);
                const R s2 = s * s, t2 = t * t;
                const R aE = fma(pn, s2, fma(qn, t2, kn)), bE = fma(pg, s2, fma(qg, t2, kg));
                const R aO = fma(rn, s, sn * t), bO = fma(rg, s, sg * t);
                emit(k, aE + aO, bE + bO, fvk(k), hvk(k));
                emit(k + 1, aE - aO, bE - bO, fvk(k + 1), hvk(k + 1));
            }
        };
        if (wall_lo || wall_hi || edge) collide(std::true_type{});
        else collide(std::false_type{});
    }
};

// One CTA of the producer/consumer fused step: the tile (a0, b0) of planes
// [zb, zb + G.chunk) of one domain.  Threads [0, TX*TY) are consumers (one per
// tile node), threads [TX*TY, TX*TY + NP) producers.
// FAULT instantiates the fault-injection form: the first CTA withholds the
// hand-off of plane fault_plane (tests of the bounded waits only).
template <int Q, typename S, typename R, int TX, int TY, int NP, bool FAULT = false, bool COH = false,
          bool XW = true, bool SPLIT = false>
__device__ __forceinline__ void fused_tile(const S* __restrict__ src, S* __restrict__ dst, const KParams<R>* p,
                                           const MarchGeom& G, unsigned step, int a0, int b0, int zb,
                                           Counters* cnt, unsigned char* smem_raw, int fault_plane = -1) {
    using St = FusedStages<Q, S, R, TX, TY, COH, SPLIT>;
    using Sh = typename St::Sh;
    constexpr int NC = TX * TY, NT = NC + NP;
    St st;
    st.phis = reinterpret_cast<R*>(smem_raw);
    st.ruts = st.phis + Sh::kPhiSlots * Sh::R;
    st.dus = st.ruts + Sh::kRutSlots * Sh::kRut * Sh::F;
    st.ring_a = reinterpret_cast<int*>(st.dus + Sh::kDuSlots * 3 * Sh::F);
    st.ring_b = st.ring_a + Sh::RW;
    st.src = src;
    st.dst = dst;
    st.p = p;
    st.G = G;
    st.nn = (size_t)p->nn;
    st.plane_n = G.na * G.nb;
    st.step = step;

    const int tid = threadIdx.x;
    const int ze = min(zb + G.chunk, G.m_hi);
    const bool walls = p->wall;
    const int wa = p->wall_x, wb = Q == 19 ? p->wall_y : 0;
    for (int i = tid; i < Sh::RW; i += NT) st.ring_a[i] = ring_coord(a0 + i - 2, G.na, wa);
    for (int i = tid; i < Sh::RH; i += NT) st.ring_b[i] = ring_coord(b0 + i - Sh::RB, G.nb, wb) * G.na;

    // hand-off ring: full[s] completes when the producers finish iteration u
    // (u = i - zb + 2, s = u mod D); empty[s] when every consumer has finished
    // plane c (u = c - zb).  The k-th use of a slot completes its phase k, so
    // the wait parity is (u / D) & 1; neither side gets two phases ahead of
    // the other's wait (producers run at most 2 iterations ahead of the plane
    // they need released, consumers cannot pass the producers).
    // SPLIT adds mint[s]: every consumer has formed the moments of its node of
    // plane c + 3 (u = c - zb), which the producers' F stage of iteration
    // c + 3 reads.  A consumer forms them right after its wait for iteration
    // c + 2, into buffer slots whose last readers (F(c+1), C(c-2)) that wait
    // has ordered before it; the producers wait on every phase in order.
    constexpr int D = Sh::kHandSlots;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem_raw + Sh::template barrier_offset<R>());
    unsigned long long* empty = full + D;
    unsigned long long* mint = empty + D;
    volatile int* aborted = reinterpret_cast<volatile int*>(full + Sh::kRings * D);
    if (tid == 0) {
        *aborted = 0;
        for (int s = 0; s < D; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, NC);
            if (SPLIT) mbar_init(mint + s, NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto wait = [&](unsigned long long* b, int u) {
        if (*aborted) return;
        if (!mbar_wait(b + (u % D), (unsigned)(u / D) & 1u)) {
            *aborted = 1;
            atomicAdd(&cnt->timeouts, 1ull);
        }
    };

    if (tid >= NC) {
        // producers: iteration i builds M(i) and F(i-1).  M(i) and F(i-1)
        // overwrite the buffers that C(i-4) read last.
        // SPLIT: from plane zb + 3 on the consumers form the tile's moments
        // and the producers the border's.
        const int t = tid - NC;
        for (int i = zb - 2; i < ze + 3; ++i) {
            const int cw = i - 4;
            if (cw >= zb && cw < ze) wait(empty, cw - zb);
            const bool m_need = i <= ze + 1 && (walls ? (i >= 0 && i < G.nm) : true);
            const bool split = SPLIT && i >= zb + 3 && i <= ze + 1;
            if (m_need) {
                if (split) st.m_border(i, t, NP);
                else st.m_stage(i, t, NP);
            }
            if (split) wait(mint, i - zb - 3);
            asm volatile("bar.sync 1, %0;" ::"r"(NP));
            const int f = i - 1;
            const bool f_need = f >= zb - 1 && f <= ze && (walls ? (f >= 0 && f < G.nm) : true);
            if (f_need) st.f_stage(f, t, NP);
            asm volatile("bar.sync 1, %0;" ::"r"(NP));
            bool withhold = false;
            if constexpr (FAULT) withhold = i == fault_plane && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
            if (t == 0 && !withhold) mbar_arrive(full + ((i - zb + 2) % D));
        }
    } else {
        // consumers: C(c) needs M(c+2) and F(c+1), i.e. producer iteration c+2
        const int ta = tid % TX, tb = tid / TX;
        const int ga = a0 + ta, gb = b0 + tb;
        const bool owns = ga < G.na && gb < G.nb;
        const int n_ab = gb * G.na + ga;
        const int dA_m = ga == 0 ? G.na - 1 : -1, dA_p = ga == G.na - 1 ? 1 - G.na : 1;
        const int dB_m = (gb == 0 ? G.nb - 1 : -1) * G.na, dB_p = (gb == G.nb - 1 ? 1 - G.nb : 1) * G.na;
        const int edge = XW ? wall_edges(*p, Q, ga, gb, G.na, G.nb) : 0;
        for (int c = zb; c < ze; ++c) {
            wait(full, c - zb + 4);
            if (SPLIT && c + 3 <= ze + 1) {
                const int m = c + 3;
                if (walls ? m < G.nm : true) st.m_interior(m, ta, tb);
                mbar_arrive(mint + ((c - zb) % D));
            }
            if (owns) st.template c_stage<XW>(c, ta, tb, n_ab, dA_m, dA_p, dB_m, dB_p, edge, cnt);
            mbar_arrive(empty + ((c - zb) % D));
        }
    }
}

// CTAs per SM the single-domain step is compiled for (the register cap that
// follows from it): D3Q19 keeps two 384-thread CTAs (80 registers) with FP32
// and FP16 storage and one 512-thread CTA with FP64; D2Q9 keeps four (FP32)
// or three 288-thread CTAs.
template <int Q, typename S> struct FusedOcc {
    static constexpr int kMinBlocks = Q == 19 ? (sizeof(S) == 8 ? 1 : 2) : (sizeof(S) == 4 ? 4 : 3);
};

// Single-domain fused step: CTA (x, y, z) takes tile (x TX, y TY) and the
// z-th chunk of planes.  XW: instance for domains with walls on the
// tile-plane axes (the other instance carries no trace of them).  SPLIT: the
// consumers form their own nodes' moments (fused_tile).
template <int Q, typename S, typename R, int TX, int TY, int NP, bool XW, bool SPLIT>
__global__ void __launch_bounds__(TX* TY + NP, FusedOcc<Q, S>::kMinBlocks)
    fused_step_kernel(const S* __restrict__ src, S* __restrict__ dst, KParams<R> p, MarchGeom G, Counters* cnt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_tile<Q, S, R, TX, TY, NP, false, false, XW, SPLIT>(src, dst, &p, G, p.step, blockIdx.x * TX,
                                                             blockIdx.y * TY, G.m_lo + blockIdx.z * G.chunk, cnt,
                                                             smem_raw);
}

// The same step with the fault-injection hook: the first CTA withholds the
// hand-off of plane fault_plane, so that its consumers' bounded wait runs out
// and the timeout is counted.  Launched only for handles created with
// the test hook lbm_test_drop_handoff set; the kernel above carries no trace
// of it.
template <int Q, typename S, typename R, int TX, int TY, int NP, bool SPLIT>
__global__ void __launch_bounds__(TX* TY + NP, FusedOcc<Q, S>::kMinBlocks)
    fused_step_fault_kernel(const S* __restrict__ src, S* __restrict__ dst, KParams<R> p, MarchGeom G, Counters* cnt,
                            int fault_plane) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_tile<Q, S, R, TX, TY, NP, true, false, true, SPLIT>(src, dst, &p, G, p.step, blockIdx.x * TX,
                                                              blockIdx.y * TY, G.m_lo + blockIdx.z * G.chunk, cnt,
                                                              smem_raw, fault_plane);
}

// ---------------------------------------------------------------------------
// Many domains, many steps, one persistent launch.  The work of a request is
// n steps x the table of work items (domain, tile, chunk): work index
// w = s * items + i is step s of item i.  CTAs take work indices in order from
// a global counter.  An item of step s of domain d may start once every item
// of d has finished step s - 1: its CTA waits (bounded) until the domain's
// completion counter reaches s * items(d), reading it with acquire ordering;
// a CTA that finishes an item adds 1 to the counter with release ordering.
// Every item a CTA waits for has a smaller work index, so a CTA that is
// running already holds it, and the waits always end: no deadlock, whatever
// the number of CTAs that are resident.  A domain takes part while s < left
// and reads buffer (cur + s) mod 2.  A wait that gives up counts a timeout
// on the domain and marks it aborted, so that later items of that domain skip
// their waits (and their results, which the latched LBM_ERR_TIMEOUT voids).

struct BatchItem {
    int domain, a0, b0, zb;
};

template <typename R> struct DomainDesc {
    KParams<R> kp;      // kp.step: the domain's step count at s = 0
    MarchGeom G;
    void* pop[2];
    Counters* cnt;
    int cur;            // buffer holding the state at s = 0
    int left;           // steps the domain still takes, counted from s = 0
    int n_items;        // work items of the domain in the table
};

// Scheduling state of a request in device memory: steps, the next work
// index, and per domain a completion counter and an abort flag.
struct BatchSched {
    int n_steps;
    int next;
    int pad[2];
    // followed by unsigned done[domains], int aborted[domains]
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// FAULT: the item fault_item of step 0 does not report its completion
// (tests of the bounded waits only).  XW: some domain has walls on the
// tile-plane axes.  SPLIT: the consumers form their own nodes' moments.
template <int Q, typename S, typename R, int TX, int TY, int NP, int MB, bool FAULT, bool XW, bool SPLIT>
__global__ void __launch_bounds__(TX* TY + NP, MB) fused_batch_kernel(const BatchItem* __restrict__ items,
                                                                  const DomainDesc<R>* __restrict__ doms,
                                                                  int n_items, BatchSched* sched, int n_doms,
                                                                  int fault_item) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KParams<R> kp;   // the current item's domain parameters
    __shared__ int w_sh, go_sh;
    int kp_domain = -1;         // domain whose parameters kp holds (thread 0)
    unsigned* done = reinterpret_cast<unsigned*>(sched + 1);
    int* aborted = reinterpret_cast<int*>(done + n_doms);
    const long long total = (long long)sched->n_steps * n_items;
    for (;;) {
        if (threadIdx.x == 0) w_sh = atomicAdd(&sched->next, 1);
        __syncthreads();
        const long long w = w_sh;
        if (w >= total || w < 0) break;
        const int s = (int)(w / n_items), i = (int)(w % n_items);
        const BatchItem it = items[i];
        const DomainDesc<R>* d = doms + it.domain;
        const bool active = s < d->left;
        if (active && threadIdx.x == 0) {
            if (kp_domain != it.domain) {   // consecutive items mostly share a domain
                kp = d->kp;
                kp_domain = it.domain;
            }
            int go = 1;
            if (s > 0) {
                const unsigned target = (unsigned)s * (unsigned)d->n_items;
                const long long t0 = clock64();
                while (ld_acquire_u32(done + it.domain) < target) {
                    if (*(volatile int*)(aborted + it.domain)) {
                        go = 0;
                        break;
                    }
                    if (clock64() - t0 > 1000000000ll) {   // about half a second
                        atomicExch(aborted + it.domain, 1);
                        atomicAdd(&d->cnt->timeouts, 1ull);
                        go = 0;
                        break;
                    }
                }
            }
            go_sh = go;
        }
        __syncthreads();
        if (active && go_sh) {
            const int in = (d->cur + s) & 1;
            const MarchGeom G = d->G;
            fused_tile<Q, S, R, TX, TY, NP, false, true, XW, SPLIT>((const S*)d->pop[in], (S*)d->pop[in ^ 1], &kp, G,
                                                         kp.step + (unsigned)s, it.a0, it.b0, it.zb, d->cnt,
                                                         smem_raw);
        }
        __syncthreads();
        if (active && threadIdx.x == 0) {
            bool report = true;
            if constexpr (FAULT) report = !(s == 0 && i == fault_item);
            if (report) {
                __threadfence();   // release: the item's stores before its completion
                atomicAdd(done + it.domain, 1u);
            }
        }
    }
}

// descriptor bookkeeping after a request of n steps: every domain took
// min(n, left) steps
template <typename R> __global__ void batch_advance_kernel(DomainDesc<R>* doms, int count, const BatchSched* sched) {
    const int n = sched->n_steps;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < count; d += gridDim.x * blockDim.x) {
        const int taken = doms[d].left < n ? doms[d].left : n;
        doms[d].cur ^= taken & 1;
        doms[d].kp.step += (unsigned)taken;
        doms[d].left -= taken;
    }
}

}  // namespace lbm
