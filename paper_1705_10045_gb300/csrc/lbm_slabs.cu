// Slabs: one domain cut along its last axis (y for D2Q9, z for D3Q19) into
// sub-domains that each step on their own and swap halo planes after every
// step (lbm_slab_plan, lbm_slabs_*, lbm_plane_bytes, lbm_get_planes,
// lbm_set_planes).
//
// Reach of one step along the last axis.  The collision of plane c needs the
// moments of planes c-1..c+1 (the finite differences of Sec. 4 and Sec. 6.2)
// and the velocity change du of planes c-1..c+1 (u* = u + du/2 inside
// div u*), and du of plane c+1 needs Phi of planes c..c+2 (the force of
// Sec. 3): the post-collision values of plane c depend on the populations of
// planes c-2..c+2.  Streaming then moves them one plane.  So a slab that
// holds LBM_SLAB_HALO = 2 copies of its neighbours' planes beyond each cut
// collides every plane it owns exactly; it collides only those
// (lbm_set_step_planes), and its edge planes push the populations that cross
// a cut into its halo planes.  After the step the exchange runs in two
// rounds: (1) each cut's crossing populations (the directions whose velocity
// points across it: 5 for D3Q19, 3 for D2Q9) go from the pushing slab's halo
// plane to the owning slab's edge plane, which completes the neighbours'
// edge planes; (2) each slab's two halo planes are overwritten with those
// complete edge planes.
//
// Per cut and direction that moves 2 Q + (crossing directions) node pairs
// per node of the plane, and no plane is collided twice.  Every slab uses the
// same per-node arithmetic as the whole domain, so FP64 and FP32 slabs
// reproduce the undivided domain bit for bit.  FP16 storage keys its
// stochastic rounding by the node index within a handle, so FP16 slabs round
// differently (same distribution, not the same bits).
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

struct lbm_slabs {
    lbm_params p;                  // the whole domain
    int count = 0;
    int D = 0;
    long long plane = 0;           // nodes per plane of the last axis
    long long nn = 0;              // nodes of the whole domain
    std::vector<lbm_slab> plan;
    std::vector<lbm_handle*> h;
    double* tmp = nullptr;         // (D + 3) field planes of the largest slab
    double* partials = nullptr;    // reduction partials, then kSums results
    long long steps = 0;
    cudaStream_t main = nullptr;   // the caller's stream, which every slab steps on
};

namespace {

using lbm::cuda_error;
using lbm::set_error;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int last_axis(const lbm_params& p) { return p.lattice == LBM_D2Q9 ? p.ny : p.nz; }
long long plane_nodes(const lbm_params& p) { return p.lattice == LBM_D2Q9 ? (long long)p.nx : (long long)p.nx * p.ny; }

// rows of `width` bytes at src + r * spitch -> dst + r * dpitch, r < gridDim.y
template <typename W>
__global__ void __launch_bounds__(256) copy_rows_kernel(const unsigned char* __restrict__ src, long long spitch,
                                                        unsigned char* __restrict__ dst, long long dpitch,
                                                        long long words) {
    const W* s = reinterpret_cast<const W*>(src + (long long)blockIdx.y * spitch);
    W* d = reinterpret_cast<W*>(dst + (long long)blockIdx.y * dpitch);
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (long long)gridDim.x * blockDim.x)
        d[w] = s[w];
}

// Copy `rows` strided rows in the widest word that divides every address,
// pitch and width (16, 8, 4 or 2 bytes; population values are at least 2).
int copy_rows(const void* src, long long spitch, void* dst, long long dpitch, long long width, int rows,
              cudaStream_t stream) {
    if (width <= 0 || rows <= 0) return LBM_OK;
    const unsigned long long all = (unsigned long long)(size_t)src | (unsigned long long)(size_t)dst |
                                   (unsigned long long)spitch | (unsigned long long)dpitch |
                                   (unsigned long long)width;
    const int wb = (all & 15) == 0 ? 16 : (all & 7) == 0 ? 8 : (all & 3) == 0 ? 4 : 2;
    const long long words = width / wb;
    long long bx = (words + 255) / 256;
    if (bx > 1024) bx = 1024;
    const dim3 grid((unsigned)bx, (unsigned)rows);
    const auto* s = static_cast<const unsigned char*>(src);
    auto* d = static_cast<unsigned char*>(dst);
    switch (wb) {
        case 16: copy_rows_kernel<uint4><<<grid, 256, 0, stream>>>(s, spitch, d, dpitch, words); break;
        case 8: copy_rows_kernel<unsigned long long><<<grid, 256, 0, stream>>>(s, spitch, d, dpitch, words); break;
        case 4: copy_rows_kernel<unsigned><<<grid, 256, 0, stream>>>(s, spitch, d, dpitch, words); break;
        default: copy_rows_kernel<unsigned short><<<grid, 256, 0, stream>>>(s, spitch, d, dpitch, words); break;
    }
    return cuda_error(cudaGetLastError(), "plane copy launch");
}

// Directions whose velocity component along the last axis is `sign`, in
// increasing k: the populations a plane pushes across a cut above it (+1) or
// below it (-1).  Returns how many (5 for D3Q19, 3 for D2Q9).
int crossing_dirs(int Q, int sign, int* ks) {
    int n = 0;
    for (int k = 0; k < Q; ++k) {
        const int c = Q == 9 ? lbm::Vel<9>::cy(k) : lbm::Vel<19>::cz(k);
        if (c == sign) ks[n++] = k;
    }
    return n;
}

// up to 8 rows of `width` bytes: src + src[r] -> dst + dst[r], r < gridDim.y
struct RowTable {
    long long src[8], dst[8];
};
template <typename W>
__global__ void __launch_bounds__(256) copy_table_kernel(const unsigned char* __restrict__ src,
                                                         unsigned char* __restrict__ dst, RowTable t,
                                                         long long words) {
    const W* s = reinterpret_cast<const W*>(src + t.src[blockIdx.y]);
    W* d = reinterpret_cast<W*>(dst + t.dst[blockIdx.y]);
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (long long)gridDim.x * blockDim.x)
        d[w] = s[w];
}

int copy_table(const void* src, void* dst, const RowTable& t, int rows, long long width, cudaStream_t stream) {
    if (width <= 0 || rows <= 0) return LBM_OK;
    unsigned long long all = (unsigned long long)(size_t)src | (unsigned long long)(size_t)dst |
                             (unsigned long long)width;
    for (int r = 0; r < rows; ++r) all |= (unsigned long long)t.src[r] | (unsigned long long)t.dst[r];
    const int wb = (all & 15) == 0 ? 16 : (all & 7) == 0 ? 8 : (all & 3) == 0 ? 4 : 2;
    const long long words = width / wb;
    long long bx = (words + 255) / 256;
    if (bx > 1024) bx = 1024;
    const dim3 grid((unsigned)bx, (unsigned)rows);
    const auto* s = static_cast<const unsigned char*>(src);
    auto* d = static_cast<unsigned char*>(dst);
    switch (wb) {
        case 16: copy_table_kernel<uint4><<<grid, 256, 0, stream>>>(s, d, t, words); break;
        case 8: copy_table_kernel<unsigned long long><<<grid, 256, 0, stream>>>(s, d, t, words); break;
        case 4: copy_table_kernel<unsigned><<<grid, 256, 0, stream>>>(s, d, t, words); break;
        default: copy_table_kernel<unsigned short><<<grid, 256, 0, stream>>>(s, d, t, words); break;
    }
    return cuda_error(cudaGetLastError(), "crossing copy launch");
}

// Crossing populations beside a wall across the plane.  A population that
// arrives at a cut's edge plane moving away from a wall on x (or on y of
// D3Q19) would come from a node beyond that wall: no slab pushes it.  The
// receiving node's own bounce-back wrote it in the receiving slab's step, and
// the pushing slab's halo slot holds no value of this step.  So the crossing
// copy skips, per direction, the column x = 0 (c_x = +1) or x = nx - 1
// (c_x = -1) across a wall on x, and the row y = 0 or ny - 1 across a wall on
// y.  -1: no skip.
struct CrossSkip {
    int x[8], y[8];
};

// the skips of the crossing directions ks[0..n) of a plane of `p`; false when
// there are none (no walls across the plane)
bool crossing_skips(const lbm_params& p, const int* ks, int n, CrossSkip& sk) {
    bool any = false;
    for (int j = 0; j < n; ++j) {
        const int cx = p.lattice == LBM_D2Q9 ? lbm::Vel<9>::cx(ks[j]) : lbm::Vel<19>::cx(ks[j]);
        const int cy = p.lattice == LBM_D2Q9 ? 0 : lbm::Vel<19>::cy(ks[j]);
        sk.x[j] = p.wall_x && cx ? (cx > 0 ? 0 : p.nx - 1) : -1;
        sk.y[j] = p.lattice == LBM_D3Q19 && p.wall_y && cy ? (cy > 0 ? 0 : p.ny - 1) : -1;
        any = any || sk.x[j] >= 0 || sk.y[j] >= 0;
    }
    return any;
}

// rows j < gridDim.y of node pairs P: pair n of a plane (x = n mod nx,
// y = n / nx) from src + t.src[j] to dst + t.dst[j], except column sk.x[j] and
// row sk.y[j]
template <typename P>
__global__ void __launch_bounds__(256) crossing_kernel(const unsigned char* __restrict__ src,
                                                       unsigned char* __restrict__ dst, RowTable t, CrossSkip sk,
                                                       long long plane, int nx) {
    const P* s = reinterpret_cast<const P*>(src + t.src[blockIdx.y]);
    P* d = reinterpret_cast<P*>(dst + t.dst[blockIdx.y]);
    const int sx = sk.x[blockIdx.y];
    const long long sy = sk.y[blockIdx.y];
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < plane;
         n += (long long)gridDim.x * blockDim.x) {
        const long long y = n / nx;
        if ((int)(n - y * nx) == sx || y == sy) continue;
        d[n] = s[n];
    }
}

// crossing rows with wall skips; every address and offset must be a multiple
// of the pair size (2 elem bytes)
int copy_crossing_rows(const void* src, void* dst, const RowTable& t, const CrossSkip& sk, int rows,
                       long long plane, int nx, int elem, cudaStream_t stream) {
    if (plane <= 0 || rows <= 0) return LBM_OK;
    long long bx = (plane + 255) / 256;
    if (bx > 1024) bx = 1024;
    const dim3 grid((unsigned)bx, (unsigned)rows);
    const auto* s = static_cast<const unsigned char*>(src);
    auto* d = static_cast<unsigned char*>(dst);
    switch (2 * elem) {
        case 16: crossing_kernel<uint4><<<grid, 256, 0, stream>>>(s, d, t, sk, plane, nx); break;
        case 8: crossing_kernel<unsigned long long><<<grid, 256, 0, stream>>>(s, d, t, sk, plane, nx); break;
        default: crossing_kernel<unsigned><<<grid, 256, 0, stream>>>(s, d, t, sk, plane, nx); break;
    }
    return cuda_error(cudaGetLastError(), "crossing copy launch");
}


// Conservation sums of nodes [i0, i0 + n) of a population buffer whose
// arrays are nn apart: per-thread compensated sums in the arithmetic type,
// combined in FP64 in a fixed order (as in the whole-domain reduction).
template <int Q, typename S, typename R>
__global__ void __launch_bounds__(lbm::kReduceThreads) range_reduce_kernel(const S* __restrict__ pop, long long nn,
                                                                          long long i0, long long n,
                                                                          lbm::KParams<R> p,
                                                                          double* __restrict__ partials) {
    lbm::Kahan acc[lbm::kSums];   // FP64, compensated, as the whole-domain sums
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        R rho, jx, jy, jz, E;
        lbm::node_moments<Q, S, R>(pop, nn, i0 + t, p, rho, jx, jy, jz, E);
        acc[0].add((double)rho);
        acc[1].add((double)jx);
        acc[2].add((double)jy);
        acc[3].add((double)jz);
        acc[4].add((double)E);
    }
    __shared__ double sh[lbm::kSums][lbm::kReduceThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < lbm::kSums; ++q) {
        double v = lbm::warp_sum(acc[q].s - acc[q].c);
        if (lane == 0) sh[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < lbm::kSums) {
        lbm::Kahan b;
        for (int w = 0; w < lbm::kReduceThreads / 32; ++w) b.add(sh[threadIdx.x][w]);
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = b.s;
    }
}

__global__ void __launch_bounds__(32) range_final_kernel(const double* __restrict__ partials, int nblocks,
                                                         double* __restrict__ out) {
    if (threadIdx.x < lbm::kSums) {
        lbm::Kahan b;
        for (int j = 0; j < nblocks; ++j) b.add(partials[(size_t)threadIdx.x * nblocks + j]);
        out[threadIdx.x] = b.s;
    }
}

template <int Q, typename S, typename R>
int launch_range_sums(const lbm_handle* h, long long i0, long long n, double* partials, double* out) {
    lbm::KParams<R> kp{};
    kp.nn = h->nn;
    kp.rho_ref = h->p.storage == LBM_STORE_FP16 ? (R)h->p.rho_ref : R(0);
    kp.E_ref = h->p.storage == LBM_STORE_FP16 ? (R)h->p.E_ref : R(0);
    range_reduce_kernel<Q, S, R><<<lbm::kReduceBlocks, lbm::kReduceThreads, 0, h->stream>>>(
        (const S*)h->pop[h->cur], h->nn, i0, n, kp, partials);
    range_final_kernel<<<1, 32, 0, h->stream>>>(partials, lbm::kReduceBlocks, out);
    return cuda_error(cudaGetLastError(), "slab sums launch");
}

int range_sums(const lbm_handle* h, long long i0, long long n, double* partials, double* out) {
    if (h->Q == 9) {
        switch (h->p.storage) {
            case LBM_STORE_FP64: return launch_range_sums<9, double, double>(h, i0, n, partials, out);
            case LBM_STORE_FP32: return launch_range_sums<9, float, float>(h, i0, n, partials, out);
            default: return launch_range_sums<9, __half, float>(h, i0, n, partials, out);
        }
    }
    switch (h->p.storage) {
        case LBM_STORE_FP64: return launch_range_sums<19, double, double>(h, i0, n, partials, out);
        case LBM_STORE_FP32: return launch_range_sums<19, float, float>(h, i0, n, partials, out);
        default: return launch_range_sums<19, __half, float>(h, i0, n, partials, out);
    }
}

// global planes of slab s's local planes, in at most two runs (a periodic
// domain wraps the first slab's lower halo to the top of the domain)
struct Run {
    int local, global, count;
};
std::vector<Run> local_runs(const lbm_slab& s, int nm) {
    std::vector<Run> runs;
    const int nl = s.lo + s.own + s.hi;
    int j = 0;
    while (j < nl) {
        int g = ((s.first - s.lo + j) % nm + nm) % nm;
        int len = nm - g < nl - j ? nm - g : nl - j;
        runs.push_back({j, g, len});
        j += len;
    }
    return runs;
}

int check_slabs(const lbm_slabs* s) {
    if (!s) {
        set_error("null slabs");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

// Rows of one exchange phase for one launch: absolute row addresses (every
// row of a phase has the same length) and, for crossing rows, the wall
// column and row the receiver keeps (-1: none).  At most kListRows rows per
// launch (3.8 KB of kernel parameters); longer lists take several launches.
constexpr int kListRows = 150;
struct RowList {
    unsigned long long src[kListRows], dst[kListRows];
    short skip_x[kListRows], skip_y[kListRows];
};

// crossing rows: node pairs P of a plane, all but the wall column and row
template <typename P>
__global__ void __launch_bounds__(256) crossing_list_kernel(RowList t, long long plane, int nx) {
    const P* s = reinterpret_cast<const P*>(t.src[blockIdx.y]);
    P* d = reinterpret_cast<P*>(t.dst[blockIdx.y]);
    const int sx = t.skip_x[blockIdx.y];
    const long long sy = t.skip_y[blockIdx.y];
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < plane;
         n += (long long)gridDim.x * blockDim.x) {
        const long long y = n / nx;
        if ((int)(n - y * nx) == sx || y == sy) continue;
        d[n] = s[n];
    }
}

// plain rows of `words` words W
template <typename W>
__global__ void __launch_bounds__(256) rows_list_kernel(RowList t, long long words) {
    const W* s = reinterpret_cast<const W*>(t.src[blockIdx.y]);
    W* d = reinterpret_cast<W*>(t.dst[blockIdx.y]);
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (long long)gridDim.x * blockDim.x)
        d[w] = s[w];
}

// one phase of the exchange: `rows` rows of `bytes` bytes each, crossing rows
// (pair granularity, wall skips; pair = 2 elem bytes) or plain rows (the
// widest word that divides every address and the length)
int launch_list(const std::vector<unsigned long long>& src, const std::vector<unsigned long long>& dst,
                const std::vector<short>& skx, const std::vector<short>& sky, long long bytes, bool crossing,
                long long plane, int nx, int elem, cudaStream_t stream) {
    const int n = (int)src.size();
    for (int r0 = 0; r0 < n; r0 += kListRows) {
        const int rows = n - r0 < kListRows ? n - r0 : kListRows;
        RowList t;
        unsigned long long all = (unsigned long long)bytes;
        for (int r = 0; r < rows; ++r) {
            t.src[r] = src[r0 + r];
            t.dst[r] = dst[r0 + r];
            t.skip_x[r] = skx[r0 + r];
            t.skip_y[r] = sky[r0 + r];
            all |= t.src[r] | t.dst[r];
        }
        if (crossing) {
            long long bx = (plane + 255) / 256;
            if (bx > 512) bx = 512;
            const dim3 grid((unsigned)bx, (unsigned)rows);
            switch (2 * elem) {
                case 16: crossing_list_kernel<uint4><<<grid, 256, 0, stream>>>(t, plane, nx); break;
                case 8: crossing_list_kernel<unsigned long long><<<grid, 256, 0, stream>>>(t, plane, nx); break;
                default: crossing_list_kernel<unsigned><<<grid, 256, 0, stream>>>(t, plane, nx); break;
            }
        } else {
            const int wb = (all & 15) == 0 ? 16 : (all & 7) == 0 ? 8 : (all & 3) == 0 ? 4 : 2;
            const long long words = bytes / wb;
            long long bx = (words + 255) / 256;
            if (bx > 512) bx = 512;
            const dim3 grid((unsigned)bx, (unsigned)rows);
            switch (wb) {
                case 16: rows_list_kernel<uint4><<<grid, 256, 0, stream>>>(t, words); break;
                case 8: rows_list_kernel<unsigned long long><<<grid, 256, 0, stream>>>(t, words); break;
                case 4: rows_list_kernel<unsigned><<<grid, 256, 0, stream>>>(t, words); break;
                default: rows_list_kernel<unsigned short><<<grid, 256, 0, stream>>>(t, words); break;
            }
        }
        if (int rc = cuda_error(cudaGetLastError(), "exchange launch")) return rc;
    }
    return LBM_OK;
}

// the two phases of the exchange (see the top of this file), on `stream`,
// one launch each: every slab's rows go into one list
int exchange(lbm_slabs* s, cudaStream_t stream) {
    const int H = LBM_SLAB_HALO;
    const long long plane = plane_nodes(s->p);
    const int elem = (int)s->h[0]->elem;
    const long long e = 2 * (long long)elem;
    auto base = [&](int i) { return (unsigned long long)(size_t)s->h[i]->pop[s->h[i]->cur]; };
    std::vector<unsigned long long> src, dst;
    std::vector<short> skx, sky;
    // (1) crossing populations: slab i's upper edge plane pushed them into its
    // halo plane lo + own, its lower edge plane into lo - 1; they go to the
    // neighbour's edge plane (wall columns and rows of the receiver skipped)
    for (int i = 0; i < s->count; ++i) {
        const lbm_slab& a = s->plan[i];
        for (int sign = 1; sign >= -1; sign -= 2) {
            if (sign > 0 ? !a.hi : !a.lo) continue;
            const int j = sign > 0 ? a.above : a.below;
            const lbm_slab& b = s->plan[j];
            const int sp = sign > 0 ? a.lo + a.own : a.lo - 1, dp = sign > 0 ? b.lo : b.lo + b.own - 1;
            int ks[8];
            const int n = crossing_dirs(s->h[i]->Q, sign, ks);
            CrossSkip sk;
            crossing_skips(s->h[j]->p, ks, n, sk);
            for (int r = 0; r < n; ++r) {
                src.push_back(base(i) + (unsigned long long)((ks[r] * s->h[i]->nn + sp * plane) * e));
                dst.push_back(base(j) + (unsigned long long)((ks[r] * s->h[j]->nn + dp * plane) * e));
                skx.push_back((short)sk.x[r]);
                sky.push_back((short)sk.y[r]);
            }
        }
    }
    if (int rc = launch_list(src, dst, skx, sky, plane * e, true, plane, s->p.nx, elem, stream)) return rc;
    // (2) halo planes from the neighbours' edge planes, now complete: per
    // side Q rows of H planes
    src.clear(); dst.clear(); skx.clear(); sky.clear();
    for (int i = 0; i < s->count; ++i) {
        const lbm_slab& a = s->plan[i];
        for (int sign = 1; sign >= -1; sign -= 2) {
            if (sign > 0 ? !a.hi : !a.lo) continue;
            const int j = sign > 0 ? a.above : a.below;
            const lbm_slab& b = s->plan[j];
            const int first_a = sign > 0 ? a.lo + a.own : 0, first_b = sign > 0 ? b.lo : b.lo + b.own - H;
            for (int k = 0; k < s->h[i]->Q; ++k) {
                dst.push_back(base(i) + (unsigned long long)((k * s->h[i]->nn + first_a * plane) * e));
                src.push_back(base(j) + (unsigned long long)((k * s->h[j]->nn + first_b * plane) * e));
                skx.push_back(-1);
                sky.push_back(-1);
            }
        }
    }
    return launch_list(src, dst, skx, sky, H * plane * e, false, plane, s->p.nx, elem, stream);
}

}  // namespace

extern "C" {

int lbm_slab_plan(const lbm_params* p, int count, int i, lbm_slab* out) {
    if (!p || !out) {
        set_error("lbm_slab_plan: null argument");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) {
        set_error("lbm_slab_plan: lattice must be LBM_D2Q9 or LBM_D3Q19");
        return LBM_ERR_INVALID_ARG;
    }
    const int nm = last_axis(*p);
    if (count < 1 || i < 0 || i >= count) {
        set_error("lbm_slab_plan: need count >= 1 and 0 <= i < count");
        return LBM_ERR_INVALID_ARG;
    }
    if (count > 1 && nm / count < LBM_SLAB_HALO) {
        set_error("lbm_slab_plan: every slab must own at least " + std::to_string(LBM_SLAB_HALO) +
                  " planes of the last axis (" + std::to_string(nm) + " planes into " + std::to_string(count) +
                  " slabs)");
        return LBM_ERR_INVALID_ARG;
    }
    std::memset(out, 0, sizeof(*out));
    const int base = nm / count, extra = nm % count;
    out->first = i * base + (i < extra ? i : extra);
    out->own = base + (i < extra ? 1 : 0);
    const bool periodic = p->wall == 0;
    out->lo = count > 1 && (periodic || i > 0) ? LBM_SLAB_HALO : 0;
    out->hi = count > 1 && (periodic || i < count - 1) ? LBM_SLAB_HALO : 0;
    out->below = out->lo ? (i + count - 1) % count : -1;
    out->above = out->hi ? (i + 1) % count : -1;
    out->p = *p;
    const int nl = out->lo + out->own + out->hi;
    if (p->lattice == LBM_D2Q9)
        out->p.ny = nl;
    else
        out->p.nz = nl;
    // a cut is no wall: the fixed temperatures stay with the slabs at the ends
    if (out->lo) out->p.T_fixed_lo = 0;
    if (out->hi) out->p.T_fixed_hi = 0;
    return LBM_OK;
}

int lbm_slabs_create(const lbm_params* p, int count, lbm_slabs** out) {
    if (!p || !out) {
        set_error("lbm_slabs_create: null argument");
        return LBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    lbm_slab first;
    if (count < 1) {
        set_error("lbm_slabs_create: need count >= 1");
        return LBM_ERR_INVALID_ARG;
    }
    if (int rc = lbm_slab_plan(p, count, 0, &first)) return rc;   // rejects thin slabs before any allocation
    lbm_slabs* s = new (std::nothrow) lbm_slabs();
    if (!s) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
    s->p = *p;
    s->count = count;
    s->main = (cudaStream_t)p->stream;
    s->D = p->lattice == LBM_D2Q9 ? 2 : 3;
    s->plane = plane_nodes(*p);
    s->nn = (long long)p->nx * p->ny * p->nz;
    int rc = LBM_OK;
    long long max_nl = 0;
    for (int i = 0; i < count && !rc; ++i) {
        lbm_slab sl;
        rc = lbm_slab_plan(p, count, i, &sl);
        if (rc) break;
        s->plan.push_back(sl);
        lbm_handle* h = nullptr;
        rc = lbm_create(&sl.p, &h);
        if (rc) break;
        s->h.push_back(h);
        rc = lbm_set_step_planes(h, sl.lo, sl.own);   // halo planes are refreshed, not collided
        if (rc) break;

        const long long nl = sl.lo + sl.own + sl.hi;
        if (nl > max_nl) max_nl = nl;
    }
    if (!rc) {
        DeviceGuard dg(p->device);
        rc = cuda_error(cudaMalloc((void**)&s->tmp, sizeof(double) * (size_t)(s->D + 3) * max_nl * s->plane),
                        "slab field allocation");
        if (!rc)
            rc = cuda_error(cudaMalloc((void**)&s->partials,
                                       sizeof(double) * (size_t)(lbm::kSums * lbm::kReduceBlocks + lbm::kSums)),
                            "slab reduction scratch allocation");
    }
    if (rc) {
        lbm_slabs_destroy(s);
        return rc;
    }
    *out = s;
    return LBM_OK;
}

int lbm_slabs_count(const lbm_slabs* s) { return s ? s->count : LBM_ERR_INVALID_ARG; }

lbm_handle* lbm_slabs_domain(lbm_slabs* s, int i) {
    if (!s || i < 0 || i >= s->count) {
        set_error("lbm_slabs_domain: no such slab");
        return nullptr;
    }
    return s->h[i];
}

int lbm_slabs_init(lbm_slabs* s, const double* rho, const double* u, const double* eps, int mem) {
    lbm::TraceRange trace_("lbm_slabs_init");
    if (int rc = check_slabs(s)) return rc;
    if (!rho || !u || !eps || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE)) {
        set_error("lbm_slabs_init: null field or bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(s->p.device);
    const int nm = last_axis(s->p);
    const cudaMemcpyKind kind = mem == LBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t pb = sizeof(double) * (size_t)s->plane;
    for (int i = 0; i < s->count; ++i) {
        const lbm_slab& sl = s->plan[i];
        lbm_handle* h = s->h[i];
        const long long nl = h->nn;   // nodes of the slab's local domain
        // fields of the slab's local planes (halos included) in its own layout
        double* lr = s->tmp;
        double* lu = s->tmp + nl;
        double* le = s->tmp + (1 + s->D) * nl;
        for (const Run& r : local_runs(sl, nm)) {
            const size_t off_l = (size_t)r.local * s->plane, off_g = (size_t)r.global * s->plane;
            int rc = cuda_error(cudaMemcpyAsync(lr + off_l, rho + off_g, pb * r.count, kind, h->stream), "slab init copy");
            for (int c = 0; c < s->D && !rc; ++c)
                rc = cuda_error(cudaMemcpyAsync(lu + c * nl + off_l, u + c * s->nn + off_g, pb * r.count, kind, h->stream),
                                "slab init copy");
            if (!rc)
                rc = cuda_error(cudaMemcpyAsync(le + off_l, eps + off_g, pb * r.count, kind, h->stream), "slab init copy");
            if (rc) return rc;
        }
        // synchronising: the next slab may reuse the field buffer afterwards
        if (int rc = lbm_init(h, lr, lu, le, LBM_MEM_DEVICE)) return rc;
    }
    s->steps = 0;
    return LBM_OK;
}

int lbm_slabs_step(lbm_slabs* s, int n) {
    lbm::TraceRange trace_("lbm_slabs_step");
    if (int rc = check_slabs(s)) return rc;
    if (n < 0) {
        set_error("lbm_slabs_step: n < 0");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(s->p.device);
    for (int t = 0; t < n; ++t) {
        for (int i = 0; i < s->count; ++i)
            if (int rc = lbm_step(s->h[i], 1)) return rc;
        if (s->count > 1) {
            lbm::TraceRange swap_("halo swap");
            if (int rc = exchange(s, s->main)) return rc;
        }
        ++s->steps;
    }
    return LBM_OK;
}

int lbm_slabs_moments(lbm_slabs* s, double* rho, double* u, double* T, double* P, int mem) {
    lbm::TraceRange trace_("lbm_slabs_moments");
    if (int rc = check_slabs(s)) return rc;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) {
        set_error("lbm_slabs_moments: bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(s->p.device);
    const cudaMemcpyKind kind = mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t pb = sizeof(double) * (size_t)s->plane;
    int latched = LBM_OK;
    for (int i = 0; i < s->count; ++i) {
        const lbm_slab& sl = s->plan[i];
        lbm_handle* h = s->h[i];
        const long long nl = h->nn;
        double* lr = s->tmp;
        double* lu = s->tmp + nl;
        double* lT = s->tmp + (1 + s->D) * nl;
        double* lP = s->tmp + (2 + s->D) * nl;
        int rc = lbm_moments(h, rho ? lr : nullptr, u ? lu : nullptr, T ? lT : nullptr, P ? lP : nullptr,
                             LBM_MEM_DEVICE);
        if (rc == LBM_ERR_NONPHYSICAL && !latched)
            latched = rc;
        else if (rc)
            return rc;
        // the slab's own planes into the whole-domain fields
        const size_t off_l = (size_t)sl.lo * s->plane, off_g = (size_t)sl.first * s->plane, bytes = pb * sl.own;
        if (rho) rc = cuda_error(cudaMemcpyAsync(rho + off_g, lr + off_l, bytes, kind, h->stream), "slab moments copy");
        for (int c = 0; c < s->D && u && !rc; ++c)
            rc = cuda_error(cudaMemcpyAsync(u + c * s->nn + off_g, lu + c * nl + off_l, bytes, kind, h->stream),
                            "slab moments copy");
        if (T && !rc) rc = cuda_error(cudaMemcpyAsync(T + off_g, lT + off_l, bytes, kind, h->stream), "slab moments copy");
        if (P && !rc) rc = cuda_error(cudaMemcpyAsync(P + off_g, lP + off_l, bytes, kind, h->stream), "slab moments copy");
        if (!rc) rc = cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize");
        if (rc) return rc;
    }
    return latched;
}

int lbm_slabs_diagnostics(lbm_slabs* s, double out[8]) {
    lbm::TraceRange trace_("lbm_slabs_diagnostics");
    if (int rc = check_slabs(s)) return rc;
    if (!out) {
        set_error("lbm_slabs_diagnostics: null output");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(s->p.device);
    double tot[lbm::kSums] = {0}, comp[lbm::kSums] = {0};   // Kahan sums over the slabs
    double clamps = 0, bad = 0;
    int latched = LBM_OK;
    double* res = s->partials + lbm::kSums * lbm::kReduceBlocks;
    for (int i = 0; i < s->count; ++i) {
        const lbm_slab& sl = s->plan[i];
        lbm_handle* h = s->h[i];
        int rc = range_sums(h, (long long)sl.lo * s->plane, (long long)sl.own * s->plane, s->partials, res);
        double sums[lbm::kSums];
        lbm::Counters c;
        if (!rc) rc = cuda_error(cudaMemcpyAsync(sums, res, sizeof(sums), cudaMemcpyDeviceToHost, h->stream), "slab sums copy");
        if (!rc) rc = cuda_error(cudaMemcpyAsync(&c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "slab counters copy");
        if (rc) return rc;
        rc = lbm_sync(h);   // waits for the copies; reports a latched device error
        if (rc == LBM_ERR_NONPHYSICAL && !latched)
            latched = rc;
        else if (rc)
            return rc;
        for (int q = 0; q < lbm::kSums; ++q) {
            const double y = sums[q] - comp[q], t = tot[q] + y;
            comp[q] = (t - tot[q]) - y;
            tot[q] = t;
        }
        clamps += (double)c.clamps;
        bad += (double)c.bad;
    }
    for (int q = 0; q < lbm::kSums; ++q) out[q] = tot[q];
    out[5] = clamps;
    out[6] = bad;
    out[7] = (double)s->steps;
    return latched;
}

int lbm_slabs_sync(lbm_slabs* s) {
    if (int rc = check_slabs(s)) return rc;
    int latched = LBM_OK;
    for (int i = 0; i < s->count; ++i) {
        const int rc = lbm_sync(s->h[i]);
        if (rc == LBM_ERR_NONPHYSICAL && !latched)
            latched = rc;
        else if (rc)
            return rc;
    }
    return latched;
}

void lbm_slabs_destroy(lbm_slabs* s) {
    if (!s) return;
    {
        DeviceGuard dg(s->p.device);
        if (s->tmp) cudaFree(s->tmp);
        if (s->partials) cudaFree(s->partials);
    }
    for (lbm_handle* h : s->h) lbm_destroy(h);
    delete s;
}

size_t lbm_plane_bytes(const lbm_handle* h) {
    if (!h) return 0;
    return (size_t)2 * h->Q * (size_t)plane_nodes(h->p) * h->elem;
}

int lbm_get_planes(lbm_handle* h, int first, int count, void* buf, int mem) {
    if (!h || !buf || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE)) {
        set_error("lbm_get_planes: null handle or buffer, or bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    const int nm = last_axis(h->p);
    if (!h->initialised || first < 0 || count < 0 || first + count > nm) {
        set_error("lbm_get_planes: no state, or planes outside [0, " + std::to_string(nm) + ")");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    const long long e = 2 * (long long)h->elem, width = count * plane_nodes(h->p) * e;
    const auto* src = static_cast<const unsigned char*>(h->pop[h->cur]) + first * plane_nodes(h->p) * e;
    if (mem == LBM_MEM_DEVICE) return copy_rows(src, h->nn * e, buf, width, width, h->Q, h->stream);
    for (int r = 0; r < h->Q; ++r)
        if (int rc = cuda_error(cudaMemcpyAsync(static_cast<unsigned char*>(buf) + r * width, src + r * h->nn * e,
                                                (size_t)width, cudaMemcpyDeviceToHost, h->stream),
                                "plane copy"))
            return rc;
    return cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize");
}

int lbm_set_planes(lbm_handle* h, int first, int count, const void* buf, int mem) {
    if (!h || !buf || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE)) {
        set_error("lbm_set_planes: null handle or buffer, or bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    const int nm = last_axis(h->p);
    if (!h->initialised || first < 0 || count < 0 || first + count > nm) {
        set_error("lbm_set_planes: no state, or planes outside [0, " + std::to_string(nm) + ")");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    const long long e = 2 * (long long)h->elem, width = count * plane_nodes(h->p) * e;
    auto* dst = static_cast<unsigned char*>(h->pop[h->cur]) + first * plane_nodes(h->p) * e;
    if (mem == LBM_MEM_DEVICE) return copy_rows(buf, width, dst, h->nn * e, width, h->Q, h->stream);
    for (int r = 0; r < h->Q; ++r)
        if (int rc = cuda_error(cudaMemcpyAsync(dst + r * h->nn * e, static_cast<const unsigned char*>(buf) + r * width,
                                                (size_t)width, cudaMemcpyHostToDevice, h->stream),
                                "plane copy"))
            return rc;
    return cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize");
}

int lbm_set_step_planes(lbm_handle* h, int first, int count) {
    if (!h) {
        set_error("lbm_set_step_planes: null handle");
        return LBM_ERR_INVALID_ARG;
    }
    const int nm = last_axis(h->p);
    if (first < 0 || count < 0 || first + count > nm) {
        set_error("lbm_set_step_planes: planes outside [0, " + std::to_string(nm) + ")");
        return LBM_ERR_INVALID_ARG;
    }
    h->step_first = count ? first : 0;
    h->step_count = count;
    return LBM_OK;
}

size_t lbm_crossing_bytes(const lbm_handle* h) {
    if (!h) return 0;
    int ks[8];
    return (size_t)crossing_dirs(h->Q, 1, ks) * (size_t)plane_nodes(h->p) * 2 * h->elem;
}

namespace {
// checks of lbm_get_crossing / lbm_set_crossing; the row offsets of the
// plane's crossing pairs in the state and in a packed buffer
int crossing_rows(lbm_handle* h, int plane, int sign, const void* buf, int mem, const char* who, RowTable& state,
                  RowTable& packed, int& rows, long long& width) {
    if (!h || !buf || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) || (sign != 1 && sign != -1)) {
        set_error(std::string(who) + ": null handle or buffer, bad mem flag, or sign not +1 / -1");
        return LBM_ERR_INVALID_ARG;
    }
    const int nm = last_axis(h->p);
    if (!h->initialised || plane < 0 || plane >= nm) {
        set_error(std::string(who) + ": no state, or plane outside [0, " + std::to_string(nm) + ")");
        return LBM_ERR_INVALID_ARG;
    }
    int ks[8];
    rows = crossing_dirs(h->Q, sign, ks);
    const long long pn = plane_nodes(h->p), e = 2 * (long long)h->elem;
    width = pn * e;
    for (int j = 0; j < rows; ++j) {
        state.src[j] = state.dst[j] = (ks[j] * h->nn + plane * pn) * e;
        packed.src[j] = packed.dst[j] = j * width;
    }
    return LBM_OK;
}
}  // namespace

int lbm_get_crossing(lbm_handle* h, int plane, int sign, void* buf, int mem) {
    RowTable st, pk;
    int rows = 0;
    long long width = 0;
    if (int rc = crossing_rows(h, plane, sign, buf, mem, "lbm_get_crossing", st, pk, rows, width)) return rc;
    DeviceGuard dg(h->p.device);
    const auto* src = static_cast<const unsigned char*>(h->pop[h->cur]);
    if (mem == LBM_MEM_DEVICE) {
        RowTable t;
        for (int j = 0; j < rows; ++j) {
            t.src[j] = st.src[j];
            t.dst[j] = pk.dst[j];
        }
        return copy_table(src, buf, t, rows, width, h->stream);
    }
    for (int j = 0; j < rows; ++j)
        if (int rc = cuda_error(cudaMemcpyAsync(static_cast<unsigned char*>(buf) + pk.dst[j], src + st.src[j],
                                                (size_t)width, cudaMemcpyDeviceToHost, h->stream),
                                "crossing copy"))
            return rc;
    return cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize");
}

int lbm_set_crossing(lbm_handle* h, int plane, int sign, const void* buf, int mem) {
    RowTable st, pk;
    int rows = 0;
    long long width = 0;
    if (int rc = crossing_rows(h, plane, sign, buf, mem, "lbm_set_crossing", st, pk, rows, width)) return rc;
    DeviceGuard dg(h->p.device);
    auto* dst = static_cast<unsigned char*>(h->pop[h->cur]);
    int ks[8];
    CrossSkip sk;
    crossing_dirs(h->Q, sign, ks);
    if (crossing_skips(h->p, ks, rows, sk)) {
        // walls across the plane: the rows go through the wall-skipping copy,
        // from the caller's device buffer if it is aligned to a pair, else
        // staged in the handle's host-transfer buffer ((D + 3) planes of
        // doubles: room for the crossing rows of a plane of any slab of at
        // least two planes; no step reads it)
        const long long e = 2 * (long long)h->elem;
        const void* from = buf;
        if (mem == LBM_MEM_HOST || ((unsigned long long)(size_t)buf % (unsigned long long)e) != 0) {
            if ((size_t)(rows * width) > sizeof(double) * (size_t)(h->D + 3) * (size_t)h->nn) {
                set_error("lbm_set_crossing: a domain of one plane cannot stage the crossing rows; pass an aligned "
                          "device buffer");
                return LBM_ERR_INVALID_ARG;
            }
            if (int rc = lbm::ensure_staging(h)) return rc;
            auto* stage = reinterpret_cast<unsigned char*>(h->staging);
            const cudaMemcpyKind kind = mem == LBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
            if (int rc = cuda_error(cudaMemcpyAsync(stage, buf, (size_t)(rows * width), kind, h->stream),
                                    "crossing copy"))
                return rc;
            from = stage;
        }
        RowTable t;
        for (int j = 0; j < rows; ++j) {
            t.src[j] = pk.src[j];
            t.dst[j] = st.dst[j];
        }
        if (int rc = copy_crossing_rows(from, dst, t, sk, rows, plane_nodes(h->p), h->p.nx, h->elem, h->stream))
            return rc;
        return mem == LBM_MEM_HOST ? cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize") : LBM_OK;
    }
    if (mem == LBM_MEM_DEVICE) {
        RowTable t;
        for (int j = 0; j < rows; ++j) {
            t.src[j] = pk.src[j];
            t.dst[j] = st.dst[j];
        }
        return copy_table(buf, dst, t, rows, width, h->stream);
    }
    for (int j = 0; j < rows; ++j)
        if (int rc = cuda_error(cudaMemcpyAsync(dst + st.dst[j], static_cast<const unsigned char*>(buf) + pk.src[j],
                                                (size_t)width, cudaMemcpyHostToDevice, h->stream),
                                "crossing copy"))
            return rc;
    return cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize");
}

}  // extern "C"
