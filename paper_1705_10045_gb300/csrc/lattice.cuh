// Lattice constants, storage formats and per-node arithmetic of the thermal
// multiphase LB step (Kupershtokh, Medvedev, Gribanov, arXiv:1705.10045).
// Device-side building blocks shared by every kernel of liblbm.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace lbm {

// ---------------------------------------------------------------------------
// Velocity sets (Sec. 2).  k = 0 rest, then nearest neighbours, then
// next-nearest; each direction is followed by its opposite.

template <int Q> struct Vel;

template <> struct Vel<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int k) {
        constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return v[k];
    }
    __host__ __device__ static constexpr int cy(int k) {
        constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return v[k];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    // weights w_k (Sec. 2): 4/9, 1/9, 1/36
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // force-stencil coefficients G_k and alpha (Sec. 3)
    __host__ __device__ static constexpr double G(int k) {
        return k == 0 ? 0.0 : (k <= 4 ? 1.0 : 0.25);
    }
    static constexpr double alpha = 1.5;
};

template <> struct Vel<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int cx(int k) {
        constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return v[k];
    }
    __host__ __device__ static constexpr int cy(int k) {
        constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return v[k];
    }
    __host__ __device__ static constexpr int cz(int k) {
        constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return v[k];
    }
    // weights w_k (Sec. 2): 1/3, 1/18, 1/36
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    // force-stencil coefficients G_k and alpha (Sec. 3)
    __host__ __device__ static constexpr double G(int k) {
        return k == 0 ? 0.0 : (k <= 6 ? 1.0 : 0.5);
    }
    static constexpr double alpha = 3.0;
};

__host__ __device__ constexpr int opposite(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

// ---------------------------------------------------------------------------
// Storage formats of the population sets.  FP16 stores the shifted value
// f - w_k * ref (ref = rho_ref for N, E_ref for g) with stochastic rounding:
// a node that keeps nearly the same populations step after step would
// otherwise round the same way every step, and round-to-nearest then drifts
// the mass and energy linearly in time.  The rounding is the hardware's
// stochastic-rounding conversion (cvt.rs), which rounds a value up with
// probability equal to the fraction it discards; its random bits come from a
// counter-based hash of (step, node, direction), so a run is reproducible
// bit for bit and resumes exactly from a checkpoint.

// "lowbias32" integer hash (C. Wellons' published 32-bit mixer)
__host__ __device__ __forceinline__ unsigned mix32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// per-node random word of one step, and the word of the pair of direction k.
// The conversion rounds the low half of a pair with bits 0..12 of the word
// and the high half with bits 16..28.  t = nb * (2k + 1) * golden ratio
// constant (mod 2^32) is uniform, since multiplying by an odd constant is a
// bijection; but its bits 0..12 depend on those of nb alone, the same few
// bits for every direction of a node.  The word is therefore t ^ (t >> 16):
// its low field mixes in bits 16..28, which depend on nearly all of nb, and
// both fields stay uniform and independent of each other.  (The high half of
// a 64-bit product is not uniform, and rounding with it drifted the energy.)
__device__ __forceinline__ unsigned node_bits(unsigned step, unsigned n) {
    return mix32(n * 0x9E3779B1u ^ mix32(step + 0x632BE5ABu));
}
__device__ __forceinline__ unsigned pair_word(unsigned nb, int k) {
    const unsigned t = nb * ((2u * (unsigned)k + 1u) * 0x9E3779B9u);
    return t ^ (t >> 16);
}

// Population layout in device memory.  Every kernel reads a node's N_k and
// g_k together (the moments need both sets, the collision updates both) and
// the push sends both to the same neighbour, so the two sets are interleaved:
// for each direction k an array of nn node pairs (N_k, g_k), x fastest.  The
// value of set s (0: N, 1: g), direction k, node n is element
// 2 (k nn + n) + s, and pair index k nn + n moves both in one vector access.
// Checkpoints (lbm_get_state / lbm_set_state) use the set-major layout of 2Q
// planes (N_0..N_{Q-1}, g_0..g_{Q-1}); the conversion kernels sit in
// kernels.cuh.
__host__ __device__ __forceinline__ size_t pair_index(int k, long long nn, long long n) {
    return (size_t)k * (size_t)nn + (size_t)n;
}

template <typename S, typename R> struct Store;
// load: one value at element index i (the set-major checkpoint layout).
// load2 / store2: the pair (N_k, g_k) at pair index i in one access (shifts
// sN, sG; random word t of the FP16 rounding).  load2_keep: a first read
// of lines the same SM reads again soon (L2 evict-last where it pays).
// load2_last: the read of a value's last use on this SM (the fused step's
// consumer reload); L1::no_allocate leaves L1 to the lines the moment stage
// will still reuse.  The _coh forms skip the non-coherent path, for data
// other CTAs of the same launch wrote (read after an acquire of their
// release).

template <> struct Store<double, double> {
    static constexpr bool kStochastic = false, kShifted = false;
    __device__ static double load(const double* p, size_t i, double) { return p[i]; }
    __device__ static void load2(const double* p, size_t i, double, double, double& a, double& b) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
        a = v.x;
        b = v.y;
    }
    __device__ static void load2_keep(const double* p, size_t i, double sN, double sG, double& a, double& b) {
        load2(p, i, sN, sG, a, b);
    }
    __device__ static void load2_last(const double* p, size_t i, double, double, double& a, double& b) {
        asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p + 2 * i));
    }
    __device__ static void load2_coh(const double* p, size_t i, double, double, double& a, double& b) {
        asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p + 2 * i) : "memory");
    }
    __device__ static void load2_last_coh(const double* p, size_t i, double, double, double& a, double& b) {
        asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p + 2 * i)
                     : "memory");
    }
    __device__ static void store2(double* p, size_t i, double a, double b, double, double, unsigned = 0) {
        reinterpret_cast<double2*>(p)[i] = make_double2(a, b);
    }
};

template <> struct Store<float, float> {
    static constexpr bool kStochastic = false, kShifted = false;
    __device__ static float load(const float* p, size_t i, float) { return __ldg(p + i); }
    __device__ static void load2(const float* p, size_t i, float, float, float& a, float& b) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
        a = v.x;
        b = v.y;
    }
    __device__ static void load2_keep(const float* p, size_t i, float, float, float& a, float& b) {
        unsigned long long pol;
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
        asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(a), "=f"(b) : "l"(p + 2 * i), "l"(pol));
    }
    __device__ static void load2_last(const float* p, size_t i, float, float, float& a, float& b) {
        asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p + 2 * i));
    }
    __device__ static void load2_coh(const float* p, size_t i, float, float, float& a, float& b) {
        asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p + 2 * i) : "memory");
    }
    __device__ static void load2_last_coh(const float* p, size_t i, float, float, float& a, float& b) {
        asm volatile("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p + 2 * i)
                     : "memory");
    }
    // the stored pair is read again only in the next step, after the whole
    // domain has streamed through L2: evict-first keeps L2 for the lines the
    // step itself still reads
    __device__ static void store2(float* p, size_t i, float a, float b, float, float, unsigned = 0) {
        unsigned long long pol;
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p + 2 * i), "f"(a), "f"(b), "l"(pol)
                     : "memory");
    }
};

// FP16 shifted storage: a pair is one 32-bit word, N_k in the low half, g_k in
// the high half.  rnd13: 13 random bits; adding them below the 10 FP16
// mantissa bits of the FP32 value and rounding toward zero rounds the
// magnitude up with probability equal to the discarded fraction (unbiased
// for FP16-normal values).  The conversion drops the 13 low bits itself.
// The _raw forms move the stored, shifted values as they are (kShifted: a
// kernel may do its arithmetic on shifted values and skip the shifts).
template <> struct Store<__half, float> {
    static constexpr bool kStochastic = true, kShifted = true;
    __device__ static float load(const __half* p, size_t i, float shift) {
        return __half2float(__ldg(p + i)) + shift;
    }
    __device__ static void unpack(unsigned w, float sN, float sG, float& a, float& b) {
        a = __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))) + sN;
        b = __half2float(__ushort_as_half((unsigned short)(w >> 16))) + sG;
    }
    __device__ static void unpack_raw(unsigned w, float& a, float& b) {
        a = __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu)));
        b = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
    }
    __device__ static unsigned word(const __half* p, size_t i) { return __ldg(reinterpret_cast<const unsigned*>(p) + i); }
    __device__ static unsigned word_last(const __half* p, size_t i) {
        unsigned w;
        asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(w) : "l"(p + 2 * i));
        return w;
    }
    __device__ static unsigned word_coh(const __half* p, size_t i) {
        unsigned w;
        asm volatile("ld.global.b32 %0, [%1];" : "=r"(w) : "l"(p + 2 * i) : "memory");
        return w;
    }
    __device__ static unsigned word_last_coh(const __half* p, size_t i) {
        unsigned w;
        asm volatile("ld.global.L1::no_allocate.b32 %0, [%1];" : "=r"(w) : "l"(p + 2 * i) : "memory");
        return w;
    }
    __device__ static void load2(const __half* p, size_t i, float sN, float sG, float& a, float& b) {
        unpack(word(p, i), sN, sG, a, b);
    }
    __device__ static void load2_keep(const __half* p, size_t i, float sN, float sG, float& a, float& b) {
        load2(p, i, sN, sG, a, b);
    }
    __device__ static void load2_last(const __half* p, size_t i, float sN, float sG, float& a, float& b) {
        unpack(word_last(p, i), sN, sG, a, b);
    }
    __device__ static void load2_coh(const __half* p, size_t i, float sN, float sG, float& a, float& b) {
        unpack(word_coh(p, i), sN, sG, a, b);
    }
    __device__ static void load2_last_coh(const __half* p, size_t i, float sN, float sG, float& a, float& b) {
        unpack(word_last_coh(p, i), sN, sG, a, b);
    }
    __device__ static void load2_raw(const __half* p, size_t i, float& a, float& b) { unpack_raw(word(p, i), a, b); }
    // the halves of a pair word widened, and sums with one half rounded once in
    // FP32 (mixed-precision add / sub: a half widens to FP32 exactly, so these
    // equal widening first, in one instruction fewer)
    __device__ static float lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))); }
    __device__ static float hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    __device__ static float add_lo(unsigned w, float acc) {   // acc + N half
        float r;
        asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"((unsigned short)(w & 0xFFFFu)), "f"(acc));
        return r;
    }
    __device__ static float add_hi(unsigned w, float acc) {   // acc + g half
        float r;
        asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"((unsigned short)(w >> 16)), "f"(acc));
        return r;
    }
    __device__ static float sub_lo(unsigned w, float acc) {   // N half - acc
        float r;
        asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"((unsigned short)(w & 0xFFFFu)), "f"(acc));
        return r;
    }
    __device__ static void load2_last_raw(const __half* p, size_t i, float& a, float& b) {
        unpack_raw(word_last(p, i), a, b);
    }
    __device__ static void load2_coh_raw(const __half* p, size_t i, float& a, float& b) {
        unpack_raw(word_coh(p, i), a, b);
    }
    __device__ static void load2_last_coh_raw(const __half* p, size_t i, float& a, float& b) {
        unpack_raw(word_last_coh(p, i), a, b);
    }
    // both halves rounded stochastically by one packed conversion (g_k in the
    // high half) with the random word t; a, b already shifted
    __device__ static void store2_raw(__half* p, size_t i, float a, float b, unsigned t) {
        unsigned w;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(b), "f"(a), "r"(t));
        reinterpret_cast<unsigned*>(p)[i] = w;
    }
    __device__ static void store2(__half* p, size_t i, float a, float b, float sN, float sG, unsigned t = 0) {
        store2_raw(p, i, a - sN, b - sG, t);
    }
};

// ---------------------------------------------------------------------------
// Parameters as seen by the kernels (arithmetic type R).

template <typename R> struct KParams {
    int nx, ny, nz;
    long long nn;
    R kappa, A, T0;
    int barotropic;
    R omega, omega_E;     // 1/tau, 1/tau_E
    R c_v;
    int chi_mode;
    R lambda, chi;
    R g[3];
    int wall;                       // walls of the last axis
    int T_fixed_lo, T_fixed_hi;
    R T_lo, T_hi;
    int wall_x, wall_y;             // walls of x, and of y (D3Q19)
    int T_fixed_x[2], T_fixed_y[2]; // per wall (low, high end)
    R T_x[2], T_y[2];
    int pressure_work, conduction, pseudoforce;
    R rho_ref, E_ref;     // FP16 shifts
    unsigned step;        // step counter, seeds the FP16 stochastic rounding
    R latent;             // rho_liq Q of Sec. 5 (0: no latent heat)
    const R* coex;        // rho_v then rho_l on T = 0.5 + j/1024, j = 0..512
};

// reduced van der Waals EOS scaled by kappa (Sec. 3); T0 when barotropic (Sec. 4)
template <typename R>
__device__ __forceinline__ R eos_pressure(const KParams<R>& p, R rho, R T) {
    R Te = p.barotropic ? p.T0 : T;
    return p.kappa * fma(R(-3) * rho, rho, R(8) * rho * Te / (R(3) - rho));
}

template <typename R>
__device__ __forceinline__ R conductivity(const KParams<R>& p, R rho) {
    return p.chi_mode ? rho * p.c_v * p.chi : p.lambda;
}

// Latent heat of the phase transition (Sec. 5): inside the transition layer
// rho_v(T) < rho < rho_l(T) the energy changes by
//   (rho_liq Q / (rho_l - rho_v)) drho/dt,  drho/dt = -rho div(u*),
// with the Maxwell densities interpolated linearly in T in the table
// (T below the grid takes its first point; no layer at T >= 1).  div is the
// centred-difference divergence of u* the pressure work uses.
template <typename R>
__device__ __forceinline__ R latent_heat(const KParams<R>& p, R rho, R T, R div) {
    if (!(T < R(1))) return R(0);
    R s = (T - R(0.5)) * R(1024);
    if (s < R(0)) s = R(0);
    int j = (int)floor(s);
    if (j > 511) j = 511;
    const R f = s - (R)j;
    const R* v = p.coex;
    const R* l = p.coex + 513;
    const R rv = v[j] + f * (v[j + 1] - v[j]);
    const R rl = l[j] + f * (l[j + 1] - l[j]);
    if (!(rho > rv && rho < rl)) return R(0);
    return -p.latent * rho * div / (rl - rv);
}

// ---------------------------------------------------------------------------
// Neighbour index along the lattice.  Every axis is periodic or closed by
// walls half a node beyond its ends (the last axis: `wall`; x: wall_x; y of
// D3Q19: wall_y).  g[a] is -1/+1 when the step crosses the low/high wall of
// lattice axis a and ghost is nonzero when it crosses any wall; the index
// then points at the mirror node.

struct Nb {
    long long n;
    int ghost;
    int g[3];
};

__device__ __forceinline__ int axis_step(int i, int n, int walled, int& g) {
    g = 0;
    if (!walled) return i < 0 ? i + n : (i >= n ? i - n : i);
    if (i < 0) { g = -1; return -1 - i; }
    if (i >= n) { g = 1; return 2 * n - 1 - i; }
    return i;
}

template <int D, typename R>
__device__ __forceinline__ Nb neighbour(int x, int y, int z, int dx, int dy, int dz, const KParams<R>& p) {
    Nb r;
    const int X = axis_step(x + dx, p.nx, p.wall_x, r.g[0]);
    int Y, Z;
    if (D == 2) {
        Y = axis_step(y + dy, p.ny, p.wall, r.g[1]);
        Z = 0;
        r.g[2] = 0;
    } else {
        Y = axis_step(y + dy, p.ny, p.wall_y, r.g[1]);
        Z = axis_step(z + dz, p.nz, p.wall, r.g[2]);
    }
    r.ghost = r.g[0] | r.g[1] | r.g[2];
    r.n = ((long long)Z * p.ny + Y) * p.nx + X;
    return r;
}

// Temperature mode of the wall at end `hi` (0 low, 1 high) of lattice axis a:
// true and the wall temperature Tw when that wall is held at a fixed T.
template <int D, typename R>
__device__ __forceinline__ bool wall_T(const KParams<R>& p, int a, int hi, R& Tw) {
    if (a == D - 1) {
        Tw = hi ? p.T_hi : p.T_lo;
        return hi ? p.T_fixed_hi : p.T_fixed_lo;
    }
    if (a == 0) {
        Tw = p.T_x[hi];
        return p.T_fixed_x[hi];
    }
    Tw = p.T_y[hi];
    return p.T_fixed_y[hi];
}

// ---------------------------------------------------------------------------
// Equilibrium per unit density (Eq. (feq)) with theta = 1/3:
//   e_k(u) = w_k (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2),  N_k^eq = rho e_k(u)
// and its EDM increment (Eq. (edm)) per unit density:
//   d_k = e_k(u + du) - e_k(u)
//       = w_k (3 c.du + 9/2 c.du (2 c.u + c.du) - 3/2 du.(2u + du))
// written as a difference so that FP32 keeps its precision for small du.

template <int Q, typename R>
__device__ __forceinline__ R cdot(int k, R ux, R uy, R uz) {
    using V = Vel<Q>;
    R s = R(0);
    if (V::cx(k) == 1) s += ux; else if (V::cx(k) == -1) s -= ux;
    if (V::cy(k) == 1) s += uy; else if (V::cy(k) == -1) s -= uy;
    if (V::D == 3) { if (V::cz(k) == 1) s += uz; else if (V::cz(k) == -1) s -= uz; }
    return s;
}

}  // namespace lbm
