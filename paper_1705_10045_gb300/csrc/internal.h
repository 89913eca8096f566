// Host-side state of one liblbm handle and the per-lattice back ends.
#pragma once

#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include <nvtx3/nvToolsExt.h>

struct lbm_handle {
    lbm_params p;
    int Q = 0, D = 0;
    long long nn = 0;
    size_t elem = 0;            // bytes per stored population value
    void* pop[2] = {nullptr, nullptr};   // ping-pong population buffers, 2Q planes each
    int cur = 0;                // buffer holding the current state
    void* fld = nullptr;        // field planes (arithmetic type)
    void* cnt = nullptr;        // lbm::Counters on the device
    double* partials = nullptr; // reduction scratch: block partials + 8 results
    double* staging = nullptr;  // (D + 3) planes of doubles for host transfers, allocated on demand
    void* coex = nullptr;       // coexistence table (arithmetic type) when p.latent != 0
    unsigned long long reported_bad = 0;
    long long steps = 0;
    bool initialised = false;
    bool fused_ready = false;   // shared-memory limit of the fused kernel raised
    int fault_drop = 0;         // lbm_test_drop_handoff hook: 1 + plane, 0 = off
    int step_first = 0;         // lbm_set_step_planes: the fused step collides planes
    int step_count = 0;         // [step_first, step_first + step_count) of the last axis (0: all)
    bool pending = false;       // lbm_step_begin opened a step that lbm_step_end has not closed
    long long pending_step = 0; // its step count (the FP16 rounding seed)
    cudaStream_t stream = nullptr;
};

// Many domains advanced together (lbm_batch_*): every domain is an
// lbm_handle; one persistent launch per request covers all of them and all
// steps through a work table.
struct lbm_batch {
    lbm_params common;
    int Q = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;            // created by lbm_batch_create
    std::vector<lbm_handle*> doms;      // slot -> domain handle (nullptr: free slot)
    std::vector<long long> budget;      // steps each domain may still take
    void* d_items = nullptr;            // BatchItem[items_cap]
    size_t items_cap = 0;
    int n_items = 0;
    void* d_descs = nullptr;            // DomainDesc<R>[descs_cap]
    void* h_descs = nullptr;            // pinned staging of the descriptors
    size_t descs_cap = 0;
    bool dirty = true;                  // work table out of date
    std::vector<char> in_table;         // slot -> its tiles are in the work table (a step budget
                                        // this request; every domain while tuning)
    int variant = 0;                    // CTA shape (see lbm_batch_variants)
    void* d_sched = nullptr;            // lbm::BatchSched + done[descs_cap] + aborted[descs_cap]
    int* h_steps = nullptr;             // pinned staging of the request's step count
    int sched_steps = 0;                // step count of the current request (host copy)
    int grid = 0;                       // persistent CTAs of the current shape
    bool xw = false;                    // some domain has walls on the tile-plane axes
    int fault_item = -1;                // lbm_batch_test_drop_item hook: item of step 0, -1 = off
    cudaGraphExec_t graph = nullptr;    // clear + persistent launch + descriptor advance
    int graph_items = -1, graph_variant = -1, graph_doms = -1, graph_fault = -2;
};

namespace lbm {


// NVTX range around a library call: named spans on a profiler's timeline
// (Nsight Systems), a cheap no-op when no tool is attached.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// error reporting shared by the translation units
void set_error(const std::string& msg);
int cuda_error(cudaError_t e, const char* where);
int ensure_staging(lbm_handle* h);   // the handle's host-transfer buffer, allocated on first use


// per-lattice entry points, dispatched on the storage format inside
template <int Q> struct Backend {
    static int step(lbm_handle* h, int n);
    static int step_range(lbm_handle* h, int first, int count);   // planes of the step lbm_step_begin opened
    static int profile(lbm_handle* h, int n, double* ms, int cap);   // returns launches per step
    static const char* launch_name(const lbm_handle* h, int j);
    static int launches(const lbm_handle* h);
    static int init(lbm_handle* h, const double* rho, const double* u, const double* eps);   // device pointers
    static int moments(lbm_handle* h, double* rho, double* u, double* T, double* P);       // device pointers
    static int reduce(lbm_handle* h, double* out_dev);   // 5 sums into device memory
    static size_t field_bytes(int storage);
    // batches: shapes, work table, descriptors, and one request (clear, the
    // persistent launch, and the descriptor advance when `advance`)
    static int batch_variants();
    static const char* batch_variant_name(int v);
    static int batch_build(lbm_batch* b);
    static int batch_launch(lbm_batch* b, int advance);
    static size_t desc_bytes(int storage);
};

}  // namespace lbm
