// Batches of domains advanced together (lbm_batch_* in include/lbm.h).
//
// Every domain is an ordinary lbm_handle (own population buffers, counters
// and moments scratch), created on the batch's stream.  One persistent launch
// per request covers every step of every domain through a table of work
// items (domain, tile, chunk); each domain's descriptor in device memory
// holds its pointers, parameters, the buffer holding its state and the steps
// it still takes in the request.  Inside the launch, per-domain completion
// counters order the steps (fused.cuh, fused_batch_kernel).  The request --
// clearing the scheduling state, the launch and the descriptor advance -- is
// captured once into a CUDA graph and replayed; the step count it reads is
// uploaded with the descriptors.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "fused.cuh"
#include "coexistence.h"
#include "internal.h"

using lbm::cuda_error;
using lbm::set_error;

namespace {

int be_build(lbm_batch* b) { return b->Q == 9 ? lbm::Backend<9>::batch_build(b) : lbm::Backend<19>::batch_build(b); }
int be_launch(lbm_batch* b, int advance) {
    return b->Q == 9 ? lbm::Backend<9>::batch_launch(b, advance) : lbm::Backend<19>::batch_launch(b, advance);
}
size_t be_desc_bytes(const lbm_batch* b) {
    return b->Q == 9 ? lbm::Backend<9>::desc_bytes(b->common.storage) : lbm::Backend<19>::desc_bytes(b->common.storage);
}

int check_batch(const lbm_batch* b) {
    if (!b) {
        set_error("null batch");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

int check_slot(const lbm_batch* b, int id) {
    if (id < 0 || (size_t)id >= b->doms.size() || !b->doms[id]) {
        set_error("no domain with id " + std::to_string(id) + " in this batch");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

void drop_graph(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_items = b->graph_variant = b->graph_doms = -1;
    b->graph_fault = -2;
}

// Descriptor storage for every slot (device array + pinned staging).
int ensure_descs(lbm_batch* b) {
    const size_t need = std::max<size_t>(b->doms.size(), 1);
    if (need <= b->descs_cap) return LBM_OK;
    const size_t cap = std::max<size_t>(need, 2 * b->descs_cap);
    const size_t bytes = cap * be_desc_bytes(b);
    const size_t sched = sizeof(lbm::BatchSched) + 2 * sizeof(int) * cap;
    void *d = nullptr, *h = nullptr, *ds = nullptr;
    if (int rc = cuda_error(cudaMalloc(&d, bytes), "batch descriptors")) return rc;
    if (int rc = cuda_error(cudaMalloc(&ds, sched), "batch scheduling state")) {
        cudaFree(d);
        return rc;
    }
    if (int rc = cuda_error(cudaMallocHost(&h, bytes), "batch descriptor staging")) {
        cudaFree(d);
        cudaFree(ds);
        return rc;
    }
    std::memset(h, 0, bytes);
    if (!b->h_steps)
        if (int rc = cuda_error(cudaMallocHost((void**)&b->h_steps, sizeof(int)), "batch step staging")) {
            cudaFree(d);
            cudaFree(ds);
            cudaFreeHost(h);
            return rc;
        }
    if (b->d_descs) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->d_descs);
        cudaFree(b->d_sched);
        cudaFreeHost(b->h_descs);
    }
    b->d_descs = d;
    b->d_sched = ds;
    b->h_descs = h;
    b->descs_cap = cap;
    drop_graph(b);   // the graph baked the old descriptor address
    return LBM_OK;
}

// Domains whose tiles belong in the work table: those with a step budget
// (all: every domain, for the tuner's one step of each).
std::vector<char> table_set(const lbm_batch* b, bool all) {
    std::vector<char> in(b->doms.size(), 0);
    for (size_t d = 0; d < b->doms.size(); ++d) in[d] = b->doms[d] && (all || b->budget[d] > 0);
    return in;
}

// Work table for the current slots, budgets and shape; descriptors restaged.
int rebuild(lbm_batch* b, bool all = false) {
    if (int rc = cudaStreamSynchronize(b->stream)) return cuda_error((cudaError_t)rc, "batch synchronize");
    if (int rc = ensure_descs(b)) return rc;
    b->in_table = table_set(b, all);
    if (int rc = be_build(b)) return rc;
    b->dirty = all;   // a table of every domain serves the tuner only
    return LBM_OK;
}

// Host copy of the per-domain descriptor fields that change between requests:
// the buffer holding the state, the step counter and the steps to take.
template <typename R> void stage_descs(lbm_batch* b, long long n) {
    auto* dd = (lbm::DomainDesc<R>*)b->h_descs;
    for (size_t d = 0; d < b->doms.size(); ++d) {
        lbm_handle* h = b->doms[d];
        if (!h) {
            dd[d].left = 0;
            continue;
        }
        dd[d].cur = h->cur;
        dd[d].kp.step = (unsigned)h->steps;
        dd[d].left = (int)std::min<long long>(b->budget[d], n);
    }
}

// descriptors and the request's step count (n <= 2^31 / items, see lbm_batch_step)
int upload_descs(lbm_batch* b, long long n) {
    if (b->common.storage == LBM_STORE_FP64) stage_descs<double>(b, n);
    else stage_descs<float>(b, n);
    *b->h_steps = (int)n;
    b->sched_steps = (int)n;
    if (int rc = cuda_error(cudaMemcpyAsync(b->d_sched, b->h_steps, sizeof(int), cudaMemcpyHostToDevice, b->stream),
                            "batch step count copy"))
        return rc;
    return cuda_error(cudaMemcpyAsync(b->d_descs, b->h_descs, b->doms.size() * be_desc_bytes(b), cudaMemcpyHostToDevice,
                                      b->stream),
                      "batch descriptor copy");
}

int capture_graph(lbm_batch* b) {
    cudaGraph_t g = nullptr;
    if (int rc = cuda_error(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture"))
        return rc;
    const int rc = be_launch(b, 1);
    const int rc_end = cuda_error(cudaStreamEndCapture(b->stream, &g), "graph capture end");
    if (rc || rc_end) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : rc_end;
    }
    const int rc_i = cuda_error(cudaGraphInstantiate(&b->graph, g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    if (rc_i) return rc_i;
    b->graph_items = b->n_items;
    b->graph_variant = b->variant;
    b->graph_doms = (int)b->doms.size();
    b->graph_fault = b->fault_item;
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_domain_bytes(const lbm_params* p) {
    if (!p || (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19)) return 0;
    const size_t nn = (size_t)p->nx * p->ny * p->nz;
    const size_t elem = p->storage == LBM_STORE_FP64 ? 8 : (p->storage == LBM_STORE_FP32 ? 4 : 2);
    const size_t fields = p->lattice == LBM_D2Q9 ? lbm::Backend<9>::field_bytes(p->storage)
                                                 : lbm::Backend<19>::field_bytes(p->storage);
    // two population buffers of 2Q planes, the moments fields, reduction and counter scratch,
    // the staging planes a domain keeps once it has been initialised from host fields
    // (rho, eps and d velocity planes, plus one), and the coexistence table
    const size_t d = p->lattice == LBM_D2Q9 ? 2 : 3;
    const size_t staging = sizeof(double) * (d + 3) * nn;
    const size_t coex = p->latent != 0.0 ? 2 * (size_t)(lbm::kCoexIntervals + 1) * (elem == 8 ? 8 : 4) : 0;
    return 2 * 2 * (size_t)p->lattice * nn * elem + fields * nn +
           sizeof(double) * (lbm::kSums * lbm::kReduceBlocks + 8) + sizeof(lbm::Counters) + staging + coex;
}

int lbm_batch_create(const lbm_params* common, lbm_batch** out) {
    if (!common || !out) {
        set_error("lbm_batch_create: null argument");
        return LBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (common->lattice != LBM_D2Q9 && common->lattice != LBM_D3Q19) {
        set_error("lattice must be LBM_D2Q9 or LBM_D3Q19");
        return LBM_ERR_INVALID_ARG;
    }
    if (common->storage < LBM_STORE_FP64 || common->storage > LBM_STORE_FP16) {
        set_error("unknown storage format");
        return LBM_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || common->device < 0 || common->device >= ndev) {
        set_error("no CUDA device with ordinal " + std::to_string(common->device));
        return LBM_ERR_CUDA;
    }
    cudaSetDevice(common->device);
    lbm_batch* b = new lbm_batch();
    b->common = *common;
    b->Q = common->lattice;
    // graphs cannot be captured on the legacy default stream: own one when none is given
    if (common->stream) {
        b->stream = (cudaStream_t)common->stream;
    } else if (int rc = cuda_error(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "batch stream")) {
        delete b;
        return rc;
    } else {
        b->own_stream = true;
    }
    b->common.stream = b->stream;
    *out = b;
    return LBM_OK;
}

int lbm_batch_add(lbm_batch* b, const lbm_params* p, const double* rho, const double* u, const double* eps, int mem,
                  long long steps, int* id) {
    lbm::TraceRange trace_("lbm_batch_add");
    if (int rc = check_batch(b)) return rc;
    if (!p || !id || steps < 0) {
        set_error("lbm_batch_add: null parameters or id, or steps < 0");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->lattice != b->common.lattice || p->storage != b->common.storage) {
        set_error("lbm_batch_add: a domain must have the batch's lattice and storage");
        return LBM_ERR_INVALID_ARG;
    }
    lbm_params q = *p;
    q.stream = b->stream;
    q.device = b->common.device;
    q.step_kernel = LBM_STEP_FUSED;
    lbm_handle* h = nullptr;
    if (int rc = lbm_create(&q, &h)) return rc;
    if (int rc = lbm_init(h, rho, u, eps, mem)) {
        lbm_destroy(h);
        return rc;
    }
    size_t slot = 0;
    while (slot < b->doms.size() && b->doms[slot]) ++slot;
    if (slot == b->doms.size()) {
        b->doms.push_back(nullptr);
        b->budget.push_back(0);
    }
    b->doms[slot] = h;
    b->budget[slot] = steps;
    b->dirty = true;
    *id = (int)slot;
    return LBM_OK;
}

int lbm_batch_remove(lbm_batch* b, int id) {
    if (int rc = check_batch(b)) return rc;
    if (int rc = check_slot(b, id)) return rc;
    cudaStreamSynchronize(b->stream);
    lbm_destroy(b->doms[id]);
    b->doms[id] = nullptr;
    b->budget[id] = 0;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
    lbm::TraceRange trace_("lbm_batch_step");
    if (int rc = check_batch(b)) return rc;
    if (n < 0) {
        set_error("lbm_batch_step: n < 0");
        return LBM_ERR_INVALID_ARG;
    }
    if (n == 0) return LBM_OK;
    cudaSetDevice(b->common.device);
    if (b->dirty || table_set(b, false) != b->in_table)
        if (int rc = rebuild(b)) return rc;
    // the pinned staging may still feed the previous request's copy
    if (int rc = cuda_error(cudaStreamSynchronize(b->stream), "batch synchronize")) return rc;
    // one request per chunk of steps small enough for 32-bit work indices
    const long long per = std::max<long long>(1, (long long)(0x7FFFFFFF / std::max(1, b->n_items)) - 1);
    for (long long done = 0; done < n;) {
        const long long m = std::min<long long>(per, n - done);
        if (int rc = upload_descs(b, m)) return rc;
        if (!b->graph || b->graph_items != b->n_items || b->graph_variant != b->variant ||
            b->graph_doms != (int)b->doms.size() || b->graph_fault != b->fault_item) {
            drop_graph(b);
            if (int rc = capture_graph(b)) return rc;
        }
        if (int rc = cuda_error(cudaGraphLaunch(b->graph, b->stream), "graph launch")) return rc;
        done += m;
        if (done < n)   // the staging feeds the next chunk's copies
            if (int rc = cuda_error(cudaStreamSynchronize(b->stream), "batch synchronize")) return rc;
        for (size_t d = 0; d < b->doms.size() && done < n; ++d) {
            lbm_handle* h = b->doms[d];
            if (!h) continue;
            const long long taken = std::min<long long>(b->budget[d], m);
            h->cur ^= (int)(taken & 1);
            h->steps += taken;
            b->budget[d] -= taken;
        }
        if (done >= n) {
            n = m;   // the mirrors below account for the last chunk
            break;
        }
    }
    // host mirrors follow the same arithmetic as the device descriptors
    for (size_t d = 0; d < b->doms.size(); ++d) {
        lbm_handle* h = b->doms[d];
        if (!h) continue;
        const long long taken = std::min<long long>(b->budget[d], n);
        h->cur ^= (int)(taken & 1);
        h->steps += taken;
        b->budget[d] -= taken;
    }
    return LBM_OK;
}

int lbm_batch_status(const lbm_batch* b, int id, long long* steps_done, long long* steps_left) {
    if (int rc = check_batch(b)) return rc;
    if (int rc = check_slot(b, id)) return rc;
    if (steps_done) *steps_done = b->doms[id]->steps;
    if (steps_left) *steps_left = b->budget[id];
    return LBM_OK;
}

int lbm_batch_set_budget(lbm_batch* b, int id, long long steps) {
    if (int rc = check_batch(b)) return rc;
    if (int rc = check_slot(b, id)) return rc;
    if (steps < 0) {
        set_error("lbm_batch_set_budget: steps < 0");
        return LBM_ERR_INVALID_ARG;
    }
    b->budget[id] = steps;
    return LBM_OK;
}

lbm_handle* lbm_batch_domain(lbm_batch* b, int id) {
    if (!b || check_slot(b, id)) return nullptr;
    return b->doms[id];
}

int lbm_batch_size(const lbm_batch* b) {
    if (!b) return 0;
    int n = 0;
    for (auto* h : b->doms) n += h != nullptr;
    return n;
}

int lbm_batch_variants(const lbm_batch* b) {
    if (!b) return 0;
    return b->Q == 9 ? lbm::Backend<9>::batch_variants() : lbm::Backend<19>::batch_variants();
}

const char* lbm_batch_variant_name(const lbm_batch* b, int v) {
    if (!b) return "";
    return b->Q == 9 ? lbm::Backend<9>::batch_variant_name(v) : lbm::Backend<19>::batch_variant_name(v);
}

int lbm_batch_set_variant(lbm_batch* b, int v) {
    if (int rc = check_batch(b)) return rc;
    if (v < 0 || v >= lbm_batch_variants(b)) {
        set_error("lbm_batch_set_variant: no such CTA shape");
        return LBM_ERR_INVALID_ARG;
    }
    b->variant = v;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int reps, int* best, double* ms) {
    lbm::TraceRange trace_("lbm_batch_tune");
    if (int rc = check_batch(b)) return rc;
    if (reps < 1) {
        set_error("lbm_batch_tune: reps < 1");
        return LBM_ERR_INVALID_ARG;
    }
    cudaSetDevice(b->common.device);
    // one step of every domain from its current buffer into the other one
    // leaves the state untouched; the counters are restored afterwards
    std::vector<lbm::Counters> saved(b->doms.size());
    if (int rc = cuda_error(cudaStreamSynchronize(b->stream), "batch synchronize")) return rc;
    for (size_t d = 0; d < b->doms.size(); ++d)
        if (b->doms[d]) cudaMemcpy(&saved[d], b->doms[d]->cnt, sizeof(lbm::Counters), cudaMemcpyDeviceToHost);
    const int nv = lbm_batch_variants(b);
    int best_v = b->variant;
    double best_ms = 1e30;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = LBM_OK;
    for (int v = 0; v < nv && !rc; ++v) {
        b->variant = v;
        if ((rc = rebuild(b, true))) break;
        std::vector<long long> keep = b->budget;
        for (auto& x : b->budget) x = 1;
        if ((rc = upload_descs(b, 1))) break;
        b->budget = keep;
        rc = be_launch(b, 0);   // warm-up: one step into the spare buffers, no descriptor advance
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && !rc; ++r) rc = be_launch(b, 0);
        cudaEventRecord(e1, b->stream);
        if (!rc) rc = cuda_error(cudaEventSynchronize(e1), "tune synchronize");
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        const double per = t / reps;
        if (ms) ms[v] = per;
        if (per < best_ms) {
            best_ms = per;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t d = 0; d < b->doms.size(); ++d)
        if (b->doms[d]) cudaMemcpy(b->doms[d]->cnt, &saved[d], sizeof(lbm::Counters), cudaMemcpyHostToDevice);
    b->variant = best_v;
    b->dirty = true;
    drop_graph(b);
    if (best) *best = best_v;
    return rc;
}

int lbm_batch_test_drop_item(lbm_batch* b, int item) {
    if (int rc = check_batch(b)) return rc;
    b->fault_item = item < 0 ? -1 : item;
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
    lbm::TraceRange trace_("lbm_batch_sync");
    if (int rc = check_batch(b)) return rc;
    int rc = LBM_OK;
    for (auto* h : b->doms)
        if (h && !rc) rc = lbm_sync(h);
    if (!rc) rc = cuda_error(cudaStreamSynchronize(b->stream), "batch synchronize");
    return rc;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->common.device);
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto* h : b->doms) lbm_destroy(h);
    cudaFree(b->d_items);
    cudaFree(b->d_descs);
    cudaFree(b->d_sched);
    cudaFreeHost(b->h_descs);
    cudaFreeHost(b->h_steps);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
