// Launch sequences of the liblbm back end for one lattice, for every storage
// format.  Included once per lattice by lbm_d2q9.cu and lbm_d3q19.cu.
//
// A time step is either the fused single launch (fused_step_kernel, the
// default) or the three-launch form fields -> force -> collide, kept as a
// second, independently structured statement of the same step.
#pragma once

#include "fused.cuh"
#include "internal.h"
#include "kernels.cuh"

namespace lbm {

template <typename R> KParams<R> make_kparams(const lbm_handle* h) {
    const lbm_params& q = h->p;
    KParams<R> k;
    k.nx = q.nx; k.ny = q.ny; k.nz = q.nz; k.nn = h->nn;
    k.kappa = (R)q.kappa; k.A = (R)q.A; k.T0 = (R)q.T0; k.barotropic = q.barotropic != 0;
    k.omega = (R)(1.0 / q.tau); k.omega_E = (R)(1.0 / q.tau_E);
    k.c_v = (R)q.c_v;
    k.chi_mode = q.chi_mode != 0; k.lambda = (R)q.lambda; k.chi = (R)q.chi;
    for (int a = 0; a < 3; ++a) k.g[a] = (R)q.gravity[a];
    k.wall = q.wall != 0;
    k.T_fixed_lo = q.T_fixed_lo != 0; k.T_fixed_hi = q.T_fixed_hi != 0;
    k.T_lo = (R)q.T_lo; k.T_hi = (R)q.T_hi;
    k.wall_x = q.wall_x != 0; k.wall_y = q.lattice == LBM_D3Q19 && q.wall_y != 0;
    for (int e = 0; e < 2; ++e) {
        k.T_fixed_x[e] = q.T_fixed_x[e] != 0; k.T_fixed_y[e] = q.T_fixed_y[e] != 0;
        k.T_x[e] = (R)q.T_x[e]; k.T_y[e] = (R)q.T_y[e];
    }
    k.pressure_work = q.pressure_work != 0; k.conduction = q.conduction != 0; k.pseudoforce = q.pseudoforce != 0;
    const bool shifted = q.storage == LBM_STORE_FP16;
    k.rho_ref = shifted ? (R)q.rho_ref : R(0);
    k.E_ref = shifted ? (R)q.E_ref : R(0);
    k.step = (unsigned)h->steps;
    k.latent = (R)q.latent;
    k.coex = (const R*)h->coex;
    return k;
}

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// CTA shape of the fused kernel: a TX x TY tile of consumer threads plus NP
// producer threads.  D3Q19 uses 32 x 8 nodes with 128 producers (two CTAs per
// SM) in FP32/FP16 and 256 producers in FP64.  D2Q9 uses rows of 128 nodes
// with 160 producers: one producer per node of the 132-node ring row, so the
// moments of a row take a single round of loads.
// SPLIT: the consumers form the moments of their own nodes and the producers
// only those of the ring's border (fused_tile)
template <int Q, typename R> struct FusedTile;
template <typename R> struct FusedTile<9, R> { static constexpr int TX = 128, TY = 1, NP = 160; static constexpr bool SPLIT = false; };
template <> struct FusedTile<19, float> { static constexpr int TX = 32, TY = 8, NP = 128; static constexpr bool SPLIT = true; };
template <> struct FusedTile<19, double> { static constexpr int TX = 32, TY = 8, NP = 256; static constexpr bool SPLIT = true; };

// CTA shapes a batch may run with (TX x TY consumers + NP producers); the
// autotuner times each on the batch and keeps the fastest.
// MB: CTAs per SM the batch kernel is compiled for (its register cap).
// SPLIT: as for the single-domain step (D3Q19: consumers form their own
// nodes' moments).
template <int Q, typename R, int V> struct BatchShape;
template <typename R> struct BatchShape<9, R, 0> { static constexpr int TX = 128, TY = 1, NP = 160, MB = 3; static constexpr bool SPLIT = false; };
template <typename R> struct BatchShape<9, R, 1> { static constexpr int TX = 32, TY = 1, NP = 32, MB = 16; static constexpr bool SPLIT = false; };
template <typename R> struct BatchShape<9, R, 2> { static constexpr int TX = 64, TY = 1, NP = 64, MB = 8; static constexpr bool SPLIT = false; };
template <typename R> struct BatchShape<19, R, 0> { static constexpr int TX = 32, TY = 8, NP = 128, MB = 2; static constexpr bool SPLIT = true; };
template <typename R> struct BatchShape<19, R, 1> { static constexpr int TX = 32, TY = 8, NP = 160, MB = 2; static constexpr bool SPLIT = true; };
template <typename R> struct BatchShape<19, R, 2> { static constexpr int TX = 32, TY = 4, NP = 96, MB = 3; static constexpr bool SPLIT = true; };

template <int Q, typename S, typename R> struct Impl {
    static constexpr int TX = FusedTile<Q, R>::TX, TY = FusedTile<Q, R>::TY, NP = FusedTile<Q, R>::NP;
    static constexpr bool SPLIT = FusedTile<Q, R>::SPLIT;
    static int launches(const lbm_handle* h) { return h->p.step_kernel == LBM_STEP_THREE_LAUNCH ? 3 : 1; }

    // planes [m_lo, m_hi) collided; m_hi < 0: the handle's own range
    // (lbm_set_step_planes; all by default)
    static MarchGeom geometry(const lbm_handle* h, int m_lo = 0, int m_hi = -1) {
        MarchGeom G;
        G.na = h->p.nx;
        G.nb = Q == 9 ? 1 : h->p.ny;
        G.nm = Q == 9 ? h->p.ny : h->p.nz;
        if (m_hi < 0) {
            G.m_lo = h->step_count > 0 ? h->step_first : 0;
            G.m_hi = h->step_count > 0 ? h->step_first + h->step_count : G.nm;
        } else {
            G.m_lo = m_lo;
            G.m_hi = m_hi;
        }
        const int len = G.m_hi - G.m_lo;
        // planes per CTA: enough CTAs for about two per SM on 152 SMs, and
        // at least 8 planes so that the extra ring planes stay a minority
        const long long tiles = (long long)((G.na + TX - 1) / TX) * ((G.nb + TY - 1) / TY);
        long long c = (len * tiles + 303) / 304;
        c = c < 8 ? 8 : (c > 64 ? 64 : c);
        G.chunk = (int)(c > len ? len : c);
        return G;
    }

    static void launch_fused(lbm_handle* h, const KParams<R>& kp) {
        launch_fused_range(h, kp, geometry(h), (const S*)h->pop[h->cur], (S*)h->pop[h->cur ^ 1]);
        h->cur ^= 1;
    }

    // the fused step over the planes of G, src -> dst (no buffer swap)
    static void launch_fused_range(lbm_handle* h, const KParams<R>& kp, const MarchGeom& G, const S* src, S* dst) {
        const size_t smem = FusedShape<TX, TY, SPLIT>::template smem_bytes<R>();
        const bool xw = h->p.wall_x || (Q == 19 && h->p.wall_y);
        auto kern = xw ? fused_step_kernel<Q, S, R, TX, TY, NP, true, SPLIT>
                       : fused_step_kernel<Q, S, R, TX, TY, NP, false, SPLIT>;
        if (!h->fused_ready) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            h->fused_ready = true;
        }
        const dim3 grid((G.na + TX - 1) / TX, (G.nb + TY - 1) / TY, (G.m_hi - G.m_lo + G.chunk - 1) / G.chunk);
        if (h->fault_drop > 0) {   // fault-injection test hook (lbm_test_drop_handoff)
            auto fk = fused_step_fault_kernel<Q, S, R, TX, TY, NP, SPLIT>;
            cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            fk<<<grid, TX * TY + NP, smem, h->stream>>>(src, dst, kp, G, (Counters*)h->cnt, h->fault_drop - 1);
        } else {
            kern<<<grid, TX * TY + NP, smem, h->stream>>>(src, dst, kp, G, (Counters*)h->cnt);
        }
    }

    // planes [first, first + count) of the step lbm_step_begin opened: it has
    // already made the destination buffer current, so the source is the other
    static int step_range(lbm_handle* h, int first, int count) {
        KParams<R> kp = make_kparams<R>(h);
        kp.step = (unsigned)h->pending_step;
        launch_fused_range(h, kp, geometry(h, first, first + count), (const S*)h->pop[h->cur ^ 1],
                           (S*)h->pop[h->cur]);
        return cuda_error(cudaGetLastError(), "lbm_step_begin launch");
    }

    // launch j of one time step; the last launch of a step swaps the buffers
    static void launch(lbm_handle* h, const KParams<R>& kp, int j) {
        if (h->p.step_kernel != LBM_STEP_THREE_LAUNCH) {
            launch_fused(h, kp);
            return;
        }
        const unsigned g = grid_for(h->nn, 256);
        R* fld = (R*)h->fld;
        const S* src = (const S*)h->pop[h->cur];
        S* dst = (S*)h->pop[h->cur ^ 1];
        if (j == 0) fields_kernel<Q, S, R><<<g, 256, 0, h->stream>>>(src, fld, kp, (Counters*)h->cnt, 1);
        if (j == 1) force_kernel<Q, R><<<g, 256, 0, h->stream>>>(fld, kp);
        if (j == 2) {
            collide_kernel<Q, S, R><<<g, 256, 0, h->stream>>>(src, dst, fld, kp);
            h->cur ^= 1;
        }
    }

    static int step(lbm_handle* h, int n) {
        KParams<R> kp = make_kparams<R>(h);
        const int L = launches(h);
        for (int s = 0; s < n; ++s) {
            kp.step = (unsigned)(h->steps + s);
            for (int j = 0; j < L; ++j) launch(h, kp, j);
        }
        return cuda_error(cudaGetLastError(), "lbm_step launch");
    }

    // n steps with an event pair around every launch; ms[j] = mean duration of launch j
    static int profile(lbm_handle* h, int n, double* ms, int cap) {
        KParams<R> kp = make_kparams<R>(h);
        const int L = launches(h);
        cudaEvent_t ev[6];
        for (int e = 0; e < 2 * L; ++e)
            if (int rc = cuda_error(cudaEventCreate(&ev[e]), "event create")) return rc;
        double acc[3] = {0.0, 0.0, 0.0};
        int rc = LBM_OK;
        for (int s = 0; s < n && !rc; ++s) {
            kp.step = (unsigned)(h->steps + s);
            for (int j = 0; j < L; ++j) {
                cudaEventRecord(ev[2 * j], h->stream);
                launch(h, kp, j);
                cudaEventRecord(ev[2 * j + 1], h->stream);
            }
            rc = cuda_error(cudaEventSynchronize(ev[2 * L - 1]), "profile synchronize");
            for (int j = 0; j < L && !rc; ++j) {
                float t = 0.f;
                rc = cuda_error(cudaEventElapsedTime(&t, ev[2 * j], ev[2 * j + 1]), "event time");
                acc[j] += t;
            }
        }
        for (int e = 0; e < 2 * L; ++e) cudaEventDestroy(ev[e]);
        if (rc) return rc;
        for (int j = 0; j < L && j < cap; ++j) ms[j] = n > 0 ? acc[j] / n : 0.0;
        return L;
    }

    static int init(lbm_handle* h, const double* rho, const double* u, const double* eps) {
        KParams<R> kp = make_kparams<R>(h);
        kp.step = 0xFFFFFFFFu;   // rounding seed of the initial state, distinct from every step
        init_kernel<Q, S, R><<<grid_for(h->nn, 256), 256, 0, h->stream>>>((S*)h->pop[h->cur], rho, u, eps, kp,
                                                                           (Counters*)h->cnt);
        return cuda_error(cudaGetLastError(), "lbm_init launch");
    }
    static int moments(lbm_handle* h, double* rho, double* u, double* T, double* P) {
        const KParams<R> kp = make_kparams<R>(h);
        const unsigned g = grid_for(h->nn, 256);
        R* fld = (R*)h->fld;
        fields_kernel<Q, S, R><<<g, 256, 0, h->stream>>>((const S*)h->pop[h->cur], fld, kp, (Counters*)h->cnt, 0);
        force_kernel<Q, R><<<g, 256, 0, h->stream>>>(fld, kp);
        output_kernel<Q, R><<<g, 256, 0, h->stream>>>(fld, kp, rho, u, T, P);
        return cuda_error(cudaGetLastError(), "lbm_moments launch");
    }
    // ---- batches ---------------------------------------------------------
    // CTA shapes a batch can run with; the autotuner picks one per batch
    template <int V> struct Shape;
    static constexpr int kVariants = 3;

    template <int BTX, int BTY, int BNP, int BMB>
    static MarchGeom batch_geometry(const lbm_handle* h) {
        MarchGeom G;
        G.na = h->p.nx;
        G.nb = Q == 9 ? 1 : h->p.ny;
        G.nm = Q == 9 ? h->p.ny : h->p.nz;
        // planes per work item: 64 (or the whole axis).  Every item recomputes
        // the ring planes at its ends and, with the split moment stage, forms
        // the moments of its first three planes in the producers alone, so long
        // items pay; the items of the other domains of a batch fill the waves
        // (measured: shorter items for four waves per domain gave 31 instead of
        // 40 jobs/s on the D2Q9 batch and 2.1 instead of 2.4 served jobs/s)
        G.chunk = G.nm < 64 ? G.nm : 64;
        G.m_lo = 0;
        G.m_hi = G.nm;
        return G;
    }

    template <int BTX, int BTY, int BNP, int BMB, bool BSP>
    static int build_shape(lbm_batch* b) {
        std::vector<BatchItem> items;
        DomainDesc<R>* descs = (DomainDesc<R>*)b->h_descs;
        for (size_t d = 0; d < b->doms.size(); ++d) {
            lbm_handle* h = b->doms[d];
            DomainDesc<R> dd{};
            if (h) {
                dd.kp = make_kparams<R>(h);
                dd.G = batch_geometry<BTX, BTY, BNP, BMB>(h);
                dd.pop[0] = h->pop[0];
                dd.pop[1] = h->pop[1];
                dd.cnt = (Counters*)h->cnt;
                dd.cur = h->cur;
                dd.left = 0;
                const int tx = (dd.G.na + BTX - 1) / BTX, ty = (dd.G.nb + BTY - 1) / BTY;
                const int tz = (dd.G.nm + dd.G.chunk - 1) / dd.G.chunk;
                dd.n_items = tx * ty * tz;
                // only the domains that step in this request get work items: a
                // paused domain would cost every persistent CTA a pass over them
                if (d < b->in_table.size() && b->in_table[d])
                    for (int z = 0; z < tz; ++z)
                        for (int y = 0; y < ty; ++y)
                            for (int x = 0; x < tx; ++x) items.push_back({(int)d, x * BTX, y * BTY, z * dd.G.chunk});
            }
            descs[d] = dd;
        }
        if (items.size() > b->items_cap) {
            cudaFree(b->d_items);
            b->d_items = nullptr;
            b->items_cap = 0;
            if (int rc = cuda_error(cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()), "batch table")) return rc;
            b->items_cap = items.size();
        }
        b->n_items = (int)items.size();
        if (!items.empty())
            if (int rc = cuda_error(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                                                    cudaMemcpyHostToDevice, b->stream), "batch table copy"))
                return rc;
        // one persistent CTA per resident slot: occupancy times the SM count
        const size_t smem = FusedShape<BTX, BTY, BSP>::template smem_bytes<R>();
        b->xw = false;
        for (auto* h : b->doms) b->xw = b->xw || (h && (h->p.wall_x || (Q == 19 && h->p.wall_y)));
        const void* kerns[3] = {(const void*)fused_batch_kernel<Q, S, R, BTX, BTY, BNP, BMB, true, true, BSP>,
                                (const void*)fused_batch_kernel<Q, S, R, BTX, BTY, BNP, BMB, false, true, BSP>,
                                (const void*)fused_batch_kernel<Q, S, R, BTX, BTY, BNP, BMB, false, false, BSP>};
        for (const void* kern : kerns)
            if (int rc = cuda_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                    "batch kernel attribute"))
                return rc;
        int per_sm = 0, sms = 0;
        if (int rc = cuda_error(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kerns[b->xw ? 1 : 2],
                                                                              BTX * BTY + BNP, smem),
                                "batch occupancy"))
            return rc;
        if (int rc = cuda_error(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->common.device),
                                "SM count"))
            return rc;
        b->grid = std::max(1, per_sm) * std::max(1, sms);
        return LBM_OK;
    }

    // the persistent launch of a request (steps and scheduling state already in device memory)
    template <int BTX, int BTY, int BNP, int BMB, bool BSP>
    static void launch_shape(lbm_batch* b) {
        const size_t smem = FusedShape<BTX, BTY, BSP>::template smem_bytes<R>();
        const int n_doms = (int)b->doms.size();
        const int grid = std::max(1, b->grid);   // CTAs beyond the work of a request leave at once
        const auto* items = (const BatchItem*)b->d_items;
        const auto* descs = (const DomainDesc<R>*)b->d_descs;
        auto* sched = (BatchSched*)b->d_sched;
        if (b->fault_item >= 0)
            fused_batch_kernel<Q, S, R, BTX, BTY, BNP, BMB, true, true, BSP><<<grid, BTX * BTY + BNP, smem, b->stream>>>(
                items, descs, b->n_items, sched, n_doms, b->fault_item);
        else if (b->xw)
            fused_batch_kernel<Q, S, R, BTX, BTY, BNP, BMB, false, true, BSP><<<grid, BTX * BTY + BNP, smem, b->stream>>>(
                items, descs, b->n_items, sched, n_doms, -1);
        else
            fused_batch_kernel<Q, S, R, BTX, BTY, BNP, BMB, false, false, BSP><<<grid, BTX * BTY + BNP, smem, b->stream>>>(
                items, descs, b->n_items, sched, n_doms, -1);
    }

    static int batch_build(lbm_batch* b);
    static int batch_launch(lbm_batch* b, int advance);

    static int reduce(lbm_handle* h, double* out_dev) {
        const KParams<R> kp = make_kparams<R>(h);
        reduce_kernel<Q, S, R><<<kReduceBlocks, kReduceThreads, 0, h->stream>>>((const S*)h->pop[h->cur], kp,
                                                                                h->partials);
        reduce_final_kernel<<<1, 32, 0, h->stream>>>(h->partials, kReduceBlocks, out_dev);
        return cuda_error(cudaGetLastError(), "lbm_diagnostics launch");
    }
};

template <int Q, typename S, typename R> int Impl<Q, S, R>::batch_build(lbm_batch* b) {
    switch (b->variant) {
        case 0: return build_shape<BatchShape<Q, R, 0>::TX, BatchShape<Q, R, 0>::TY, BatchShape<Q, R, 0>::NP, BatchShape<Q, R, 0>::MB, BatchShape<Q, R, 0>::SPLIT>(b);
        case 1: return build_shape<BatchShape<Q, R, 1>::TX, BatchShape<Q, R, 1>::TY, BatchShape<Q, R, 1>::NP, BatchShape<Q, R, 1>::MB, BatchShape<Q, R, 1>::SPLIT>(b);
        default: return build_shape<BatchShape<Q, R, 2>::TX, BatchShape<Q, R, 2>::TY, BatchShape<Q, R, 2>::NP, BatchShape<Q, R, 2>::MB, BatchShape<Q, R, 2>::SPLIT>(b);
    }
}

// One request: clear the scheduling state, the persistent launch, and (when
// `advance`) the descriptor bookkeeping of the steps taken.
template <int Q, typename S, typename R> int Impl<Q, S, R>::batch_launch(lbm_batch* b, int advance) {
    if (b->n_items > 0) {
        const size_t clear = sizeof(BatchSched) - sizeof(int) + 2 * sizeof(int) * b->doms.size();
        if (int rc = cuda_error(cudaMemsetAsync((char*)b->d_sched + sizeof(int), 0, clear, b->stream), "batch clear"))
            return rc;
        switch (b->variant) {
            case 0: launch_shape<BatchShape<Q, R, 0>::TX, BatchShape<Q, R, 0>::TY, BatchShape<Q, R, 0>::NP, BatchShape<Q, R, 0>::MB, BatchShape<Q, R, 0>::SPLIT>(b); break;
            case 1: launch_shape<BatchShape<Q, R, 1>::TX, BatchShape<Q, R, 1>::TY, BatchShape<Q, R, 1>::NP, BatchShape<Q, R, 1>::MB, BatchShape<Q, R, 1>::SPLIT>(b); break;
            default: launch_shape<BatchShape<Q, R, 2>::TX, BatchShape<Q, R, 2>::TY, BatchShape<Q, R, 2>::NP, BatchShape<Q, R, 2>::MB, BatchShape<Q, R, 2>::SPLIT>(b); break;
        }
    }
    if (advance && !b->doms.empty()) {
        const int count = (int)b->doms.size();
        batch_advance_kernel<R><<<(count + 127) / 128, 128, 0, b->stream>>>((DomainDesc<R>*)b->d_descs, count,
                                                                            (const BatchSched*)b->d_sched);
    }
    return cuda_error(cudaGetLastError(), "batch launch");
}

#define LBM_DISPATCH(h, CALL)                                                   \
    switch ((h)->p.storage) {                                                   \
        case LBM_STORE_FP64: return Impl<Q, double, double>::CALL;              \
        case LBM_STORE_FP32: return Impl<Q, float, float>::CALL;                \
        case LBM_STORE_FP16: return Impl<Q, __half, float>::CALL;               \
        default: set_error("unknown storage format"); return LBM_ERR_INVALID_ARG; \
    }

template <int Q> int Backend<Q>::step(lbm_handle* h, int n) { LBM_DISPATCH(h, step(h, n)); }
template <int Q> int Backend<Q>::step_range(lbm_handle* h, int first, int count) {
    LBM_DISPATCH(h, step_range(h, first, count));
}
template <int Q> int Backend<Q>::profile(lbm_handle* h, int n, double* ms, int cap) {
    LBM_DISPATCH(h, profile(h, n, ms, cap));
}
template <int Q> const char* Backend<Q>::launch_name(const lbm_handle* h, int j) {
    static const char* three[] = {"fields_kernel", "force_kernel", "collide_kernel"};
    if (h->p.step_kernel == LBM_STEP_THREE_LAUNCH) return j >= 0 && j < 3 ? three[j] : "";
    return j == 0 ? "fused_step_kernel" : "";
}
template <int Q> int Backend<Q>::launches(const lbm_handle* h) {
    return h->p.step_kernel == LBM_STEP_THREE_LAUNCH ? 3 : 1;
}
template <int Q> int Backend<Q>::init(lbm_handle* h, const double* rho, const double* u, const double* eps) {
    LBM_DISPATCH(h, init(h, rho, u, eps));
}
template <int Q> int Backend<Q>::moments(lbm_handle* h, double* rho, double* u, double* T, double* P) {
    LBM_DISPATCH(h, moments(h, rho, u, T, P));
}
template <int Q> int Backend<Q>::reduce(lbm_handle* h, double* out_dev) { LBM_DISPATCH(h, reduce(h, out_dev)); }
#define LBM_BATCH_DISPATCH(b, CALL)                                              \
    switch ((b)->common.storage) {                                               \
        case LBM_STORE_FP64: return Impl<Q, double, double>::CALL;               \
        case LBM_STORE_FP32: return Impl<Q, float, float>::CALL;                 \
        case LBM_STORE_FP16: return Impl<Q, __half, float>::CALL;                \
        default: set_error("unknown storage format"); return LBM_ERR_INVALID_ARG; \
    }
template <int Q> int Backend<Q>::batch_variants() { return 3; }
template <int Q> const char* Backend<Q>::batch_variant_name(int v) {
    static const char* n9[] = {"128x1+160", "32x1+32", "64x1+64"};
    static const char* n19[] = {"32x8+128", "32x8+160", "32x4+96"};
    if (v < 0 || v > 2) return "";
    return Q == 9 ? n9[v] : n19[v];
}
template <int Q> int Backend<Q>::batch_build(lbm_batch* b) { LBM_BATCH_DISPATCH(b, batch_build(b)); }
template <int Q> int Backend<Q>::batch_launch(lbm_batch* b, int advance) { LBM_BATCH_DISPATCH(b, batch_launch(b, advance)); }
template <int Q> size_t Backend<Q>::desc_bytes(int storage) {
    return storage == LBM_STORE_FP64 ? sizeof(DomainDesc<double>) : sizeof(DomainDesc<float>);
}
#undef LBM_BATCH_DISPATCH

template <int Q> size_t Backend<Q>::field_bytes(int storage) {
    return (size_t)F_COUNT * (storage == LBM_STORE_FP64 ? sizeof(double) : sizeof(float));
}

#undef LBM_DISPATCH

}  // namespace lbm
