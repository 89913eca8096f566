// C-ABI of liblbm (declared in include/lbm.h): parameter validation, device
// memory, host/device transfers, error latching and dispatch to the
// per-lattice back ends.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "coexistence.h"
#include "internal.h"
#include "kernels.cuh"

namespace lbm {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

int cuda_error(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LBM_OK;
    // the runtime also keeps the error as its last error; clear it so that a
    // later launch check does not report it again (a failed allocation is not
    // sticky and leaves the context usable)
    (void)cudaGetLastError();
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

// the handle's (D + 3)-plane device buffer for host transfers, allocated on
// first use
int ensure_staging(lbm_handle* h) {
    if (h->staging) return LBM_OK;
    return cuda_error(cudaMalloc((void**)&h->staging, sizeof(double) * (size_t)(h->D + 3) * h->nn),
                      "staging allocation");
}

}  // namespace lbm

using lbm::cuda_error;
using lbm::ensure_staging;
using lbm::set_error;

namespace {

constexpr uint32_t kStateMagic = 0x314d424cu;   // "LBM1"

// Convert the Q nn population pairs of `from` (to_pairs: 2Q set-major planes
// of `from`) into the other layout in `to`; elem is the storage element size.
int convert_layout(const void* from, void* to, long long qnn, size_t elem, bool to_pairs, cudaStream_t stream) {
    long long blocks = (qnn + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    const unsigned g = (unsigned)(blocks > 0 ? blocks : 1);
    switch (elem) {
        case 8:
            if (to_pairs)
                lbm::sets_to_pairs_kernel<<<g, 256, 0, stream>>>((const unsigned long long*)from,
                                                                (unsigned long long*)to, qnn);
            else
                lbm::pairs_to_sets_kernel<<<g, 256, 0, stream>>>((const unsigned long long*)from,
                                                                (unsigned long long*)to, qnn);
            break;
        case 4:
            if (to_pairs)
                lbm::sets_to_pairs_kernel<<<g, 256, 0, stream>>>((const unsigned*)from, (unsigned*)to, qnn);
            else
                lbm::pairs_to_sets_kernel<<<g, 256, 0, stream>>>((const unsigned*)from, (unsigned*)to, qnn);
            break;
        default:
            if (to_pairs)
                lbm::sets_to_pairs_kernel<<<g, 256, 0, stream>>>((const unsigned short*)from, (unsigned short*)to,
                                                                qnn);
            else
                lbm::pairs_to_sets_kernel<<<g, 256, 0, stream>>>((const unsigned short*)from, (unsigned short*)to,
                                                                qnn);
            break;
    }
    return cuda_error(cudaGetLastError(), "layout conversion launch");
}
constexpr size_t kStateHeader = 16;

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

int check_handle(const lbm_handle* h) {
    if (!h) {
        set_error("null handle");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

int need_init(const lbm_handle* h) {
    if (!h->initialised) {
        set_error("handle has no state: call lbm_init or lbm_set_state first");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

// calls that start a step or replace the state wait for an open split step
// (lbm_step_begin) to be closed
int no_pending(const lbm_handle* h, const char* who) {
    if (h->pending) {
        set_error(std::string(who) + ": a step opened by lbm_step_begin is still open (call lbm_step_end)");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

// Coexistence table of the latent-heat source in the kernels' arithmetic
// type: rho_v at the kCoexIntervals + 1 grid temperatures, then rho_l.
int upload_coexistence(lbm_handle* h) {
    constexpr int n = lbm::kCoexIntervals + 1;
    std::vector<double> tab(2 * n);
    lbm::coexistence_table(tab.data(), tab.data() + n);
    const bool dbl = h->p.storage == LBM_STORE_FP64;
    const size_t bytes = (dbl ? sizeof(double) : sizeof(float)) * tab.size();
    if (int rc = cuda_error(cudaMalloc(&h->coex, bytes), "coexistence table allocation")) return rc;
    if (dbl) return cuda_error(cudaMemcpy(h->coex, tab.data(), bytes, cudaMemcpyHostToDevice), "coexistence table");
    std::vector<float> f(tab.begin(), tab.end());
    return cuda_error(cudaMemcpy(h->coex, f.data(), bytes, cudaMemcpyHostToDevice), "coexistence table");
}

int be_step(lbm_handle* h, int n) {
    return h->Q == 9 ? lbm::Backend<9>::step(h, n) : lbm::Backend<19>::step(h, n);
}
int be_init(lbm_handle* h, const double* r, const double* u, const double* e) {
    return h->Q == 9 ? lbm::Backend<9>::init(h, r, u, e) : lbm::Backend<19>::init(h, r, u, e);
}
int be_moments(lbm_handle* h, double* r, double* u, double* T, double* P) {
    return h->Q == 9 ? lbm::Backend<9>::moments(h, r, u, T, P) : lbm::Backend<19>::moments(h, r, u, T, P);
}
int be_reduce(lbm_handle* h, double* out) {
    return h->Q == 9 ? lbm::Backend<9>::reduce(h, out) : lbm::Backend<19>::reduce(h, out);
}

// FP64 -> FP32, round to nearest (the FP32 twin of the moments)
__global__ void narrow_kernel(const double* __restrict__ src, float* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// Wait for the stream and report non-physical nodes counted since the last report.
int sync_and_latch(lbm_handle* h) {
    lbm::Counters c;
    int rc = cuda_error(cudaMemcpyAsync(&c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "counter read");
    if (rc) return rc;
    rc = cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (rc) return rc;
    if (c.timeouts) {
        set_error("fused step: a bounded wait gave up (a producer/consumer hand-off inside a CTA, or in a batch the "
                  "wait for the domain's previous step; " + std::to_string(c.timeouts) +
                  " times); the state is not valid until lbm_init or lbm_set_state");
        return LBM_ERR_TIMEOUT;
    }
    if (c.bad > h->reported_bad) {
        h->reported_bad = c.bad;
        set_error("non-physical state: non-finite or non-positive density or energy at " + std::to_string(c.bad) +
                  " node-steps");
        return LBM_ERR_NONPHYSICAL;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lattice = LBM_D2Q9;
    p->nx = 64;
    p->ny = 64;
    p->nz = 1;
    p->kappa = 0.01;
    p->A = -0.152;
    p->T0 = 0.8;
    p->tau = 1.0;
    p->tau_E = 1.0;
    p->c_v = 1.5;
    p->lambda = 0.05;
    p->pressure_work = 1;
    p->conduction = 1;
    p->pseudoforce = 1;
    p->storage = LBM_STORE_FP32;
    p->rho_ref = 1.0;
    p->E_ref = 1.2;
}

int lbm_create(const lbm_params* p, lbm_handle** out) {
    lbm::TraceRange trace_("lbm_create");
    if (!p || !out) {
        set_error("lbm_create: null argument");
        return LBM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) {
        set_error("lattice must be LBM_D2Q9 or LBM_D3Q19");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == LBM_D2Q9 && p->nz != 1)) {
        set_error("sizes must be >= 1 and nz must be 1 for D2Q9");
        return LBM_ERR_INVALID_ARG;
    }
    if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) {
        set_error("domains are limited to 2^31 - 1 nodes");
        return LBM_ERR_INVALID_ARG;
    }
    const int last = p->lattice == LBM_D2Q9 ? p->ny : p->nz;
    if ((p->wall && last < 2) || (p->wall_x && p->nx < 2) || (p->wall_y && p->ny < 2)) {
        set_error("a walled axis needs at least 2 nodes");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->lattice == LBM_D2Q9 && p->wall_y) {
        set_error("D2Q9: y is the last axis, its walls are `wall` (wall_y must be 0)");
        return LBM_ERR_INVALID_ARG;
    }
    if (!(p->tau > 0.5) || !(p->tau_E > 0.5) || !(p->c_v > 0.0) || !(p->kappa > 0.0)) {
        set_error("need tau > 1/2, tau_E > 1/2, c_v > 0 and kappa > 0");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->storage < LBM_STORE_FP64 || p->storage > LBM_STORE_FP16) {
        set_error("unknown storage format");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->step_kernel != LBM_STEP_FUSED && p->step_kernel != LBM_STEP_THREE_LAUNCH) {
        set_error("step_kernel must be LBM_STEP_FUSED or LBM_STEP_THREE_LAUNCH");
        return LBM_ERR_INVALID_ARG;
    }
    if (!std::isfinite(p->latent)) {
        set_error("latent must be finite");
        return LBM_ERR_INVALID_ARG;
    }
    if (p->chi_mode && p->conduction && !(p->chi < 0.5 / (p->lattice == LBM_D2Q9 ? 2 : 3))) {
        set_error("explicit conduction needs chi < 0.5/d (Sec. 6.1)");
        return LBM_ERR_UNSTABLE_PARAMS;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
        set_error("no CUDA device with ordinal " + std::to_string(p->device));
        return LBM_ERR_CUDA;
    }
    DeviceGuard dg(p->device);
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
    h->p = *p;
    h->Q = p->lattice;
    h->D = p->lattice == LBM_D2Q9 ? 2 : 3;
    h->nn = (long long)p->nx * p->ny * p->nz;
    h->elem = p->storage == LBM_STORE_FP64 ? 8 : (p->storage == LBM_STORE_FP32 ? 4 : 2);
    h->stream = (cudaStream_t)p->stream;
    const size_t popb = (size_t)2 * h->Q * h->nn * h->elem;
    const size_t fldb = (h->Q == 9 ? lbm::Backend<9>::field_bytes(p->storage)
                                   : lbm::Backend<19>::field_bytes(p->storage)) * (size_t)h->nn;
    int rc = LBM_OK;
    if (!rc) rc = cuda_error(cudaMalloc(&h->pop[0], popb), "population allocation");
    if (!rc) rc = cuda_error(cudaMalloc(&h->pop[1], popb), "population allocation");
    if (!rc) rc = cuda_error(cudaMalloc(&h->fld, fldb), "field allocation");
    if (!rc) rc = cuda_error(cudaMalloc(&h->cnt, sizeof(lbm::Counters)), "counter allocation");
    if (!rc) rc = cuda_error(cudaMalloc((void**)&h->partials, sizeof(double) * (lbm::kSums * lbm::kReduceBlocks + 8)),
                             "reduction scratch allocation");
    if (!rc) rc = cuda_error(cudaMemsetAsync(h->cnt, 0, sizeof(lbm::Counters), h->stream), "counter reset");
    if (!rc && p->latent != 0.0) rc = upload_coexistence(h);
    if (rc) {
        lbm_destroy(h);
        return rc;
    }
    *out = h;
    return LBM_OK;
}

int lbm_coexistence(double T, double* rho_v, double* rho_l) {
    if (!rho_v || !rho_l || !lbm::coexistence(T, rho_v, rho_l)) {
        set_error("lbm_coexistence: need 0 < T < 1 and two output pointers");
        return LBM_ERR_INVALID_ARG;
    }
    return LBM_OK;
}

int lbm_init(lbm_handle* h, const double* rho, const double* u, const double* eps, int mem) {
    lbm::TraceRange trace_("lbm_init");
    if (int rc = check_handle(h)) return rc;
    if (int rc = no_pending(h, "lbm_init")) return rc;
    if (!rho || !u || !eps || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE)) {
        set_error("lbm_init: null field or bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    const size_t plane = sizeof(double) * (size_t)h->nn;
    int rc;
    if (mem == LBM_MEM_HOST) {
        if ((rc = ensure_staging(h))) return rc;
        double* s = h->staging;
        if ((rc = cuda_error(cudaMemcpyAsync(s, rho, plane, cudaMemcpyHostToDevice, h->stream), "init copy"))) return rc;
        if ((rc = cuda_error(cudaMemcpyAsync(s + h->nn, u, plane * h->D, cudaMemcpyHostToDevice, h->stream),
                             "init copy")))
            return rc;
        if ((rc = cuda_error(cudaMemcpyAsync(s + (1 + h->D) * h->nn, eps, plane, cudaMemcpyHostToDevice, h->stream),
                             "init copy")))
            return rc;
        rho = s;
        u = s + h->nn;
        eps = s + (1 + h->D) * h->nn;
    }
    if ((rc = cuda_error(cudaMemsetAsync(h->cnt, 0, sizeof(lbm::Counters), h->stream), "counter reset"))) return rc;
    h->reported_bad = 0;
    h->initialised = false;
    if ((rc = be_init(h, rho, u, eps))) return rc;
    lbm::Counters c;
    if ((rc = cuda_error(cudaMemcpyAsync(&c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "counter read")))
        return rc;
    if ((rc = cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize"))) return rc;
    if ((rc = cuda_error(cudaMemsetAsync(h->cnt, 0, sizeof(lbm::Counters), h->stream), "counter reset"))) return rc;
    if (c.bad) {
        set_error("lbm_init: " + std::to_string(c.bad) +
                  " nodes with rho <= 0, eps <= 0, non-finite values or U = p - rho/3 >= 0");
        return LBM_ERR_NONPHYSICAL;
    }
    if (c.unstable) {
        set_error("lbm_init: " + std::to_string(c.unstable) +
                  " nodes break (dp/drho)_T <= 4/3 (Sec. 3) or chi < 0.5/d (Sec. 6.1)");
        return LBM_ERR_UNSTABLE_PARAMS;
    }
    h->steps = 0;
    h->initialised = true;
    return LBM_OK;
}

int lbm_step(lbm_handle* h, int n) {
    lbm::TraceRange trace_("lbm_step");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    if (int rc = no_pending(h, "lbm_step")) return rc;
    if (n < 0) {
        set_error("lbm_step: n < 0");
        return LBM_ERR_INVALID_ARG;
    }
    if (n == 0) return LBM_OK;
    DeviceGuard dg(h->p.device);
    int rc = be_step(h, n);
    if (!rc) h->steps += n;
    return rc;
}

int lbm_step_begin(lbm_handle* h, int first, int count) {
    lbm::TraceRange trace_("lbm_step_begin");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    const int nm = h->Q == 9 ? h->p.ny : h->p.nz;
    if (first < 0 || count < 1 || first + count > nm) {
        set_error("lbm_step_begin: planes [first, first + count) outside [0, " + std::to_string(nm) + ")");
        return LBM_ERR_INVALID_ARG;
    }
    if (h->p.step_kernel == LBM_STEP_THREE_LAUNCH) {
        set_error("lbm_step_begin: split steps need the fused step kernel");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    if (!h->pending) {   // open the step: its destination becomes the current state
        h->pending = true;
        h->pending_step = h->steps;
        h->cur ^= 1;
        h->steps += 1;
    }
    return h->Q == 9 ? lbm::Backend<9>::step_range(h, first, count) : lbm::Backend<19>::step_range(h, first, count);
}

int lbm_step_end(lbm_handle* h) {
    lbm::TraceRange trace_("lbm_step_end");
    if (int rc = check_handle(h)) return rc;
    if (!h->pending) {
        set_error("lbm_step_end: no step is open");
        return LBM_ERR_INVALID_ARG;
    }
    h->pending = false;
    return LBM_OK;
}

int lbm_moments(lbm_handle* h, double* rho, double* u, double* T, double* P, int mem) {
    lbm::TraceRange trace_("lbm_moments");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) {
        set_error("lbm_moments: bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    int rc;
    if (mem == LBM_MEM_DEVICE) {
        if ((rc = be_moments(h, rho, u, T, P))) return rc;
        return sync_and_latch(h);
    }
    if ((rc = ensure_staging(h))) return rc;
    const long long nn = h->nn;
    double* s = h->staging;
    double *dr = rho ? s : nullptr, *du = u ? s + nn : nullptr, *dT = T ? s + (1 + h->D) * nn : nullptr,
           *dP = P ? s + (2 + h->D) * nn : nullptr;
    if ((rc = be_moments(h, dr, du, dT, dP))) return rc;
    const size_t plane = sizeof(double) * (size_t)nn;
    if (rho && (rc = cuda_error(cudaMemcpyAsync(rho, dr, plane, cudaMemcpyDeviceToHost, h->stream), "moments copy")))
        return rc;
    if (u && (rc = cuda_error(cudaMemcpyAsync(u, du, plane * h->D, cudaMemcpyDeviceToHost, h->stream), "moments copy")))
        return rc;
    if (T && (rc = cuda_error(cudaMemcpyAsync(T, dT, plane, cudaMemcpyDeviceToHost, h->stream), "moments copy")))
        return rc;
    if (P && (rc = cuda_error(cudaMemcpyAsync(P, dP, plane, cudaMemcpyDeviceToHost, h->stream), "moments copy")))
        return rc;
    return sync_and_latch(h);
}

int lbm_moments_f(lbm_handle* h, float* rho, float* u, float* T, float* P, int mem) {
    lbm::TraceRange trace_("lbm_moments_f");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    if (int rc = no_pending(h, "lbm_moments_f")) return rc;   // host output stages in the idle buffer
    if (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE) {
        set_error("lbm_moments_f: bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    int rc;
    if ((rc = ensure_staging(h))) return rc;
    const long long nn = h->nn;
    double* s = h->staging;
    double *dr = rho ? s : nullptr, *du = u ? s + nn : nullptr, *dT = T ? s + (1 + h->D) * nn : nullptr,
           *dP = P ? s + (2 + h->D) * nn : nullptr;
    if ((rc = be_moments(h, dr, du, dT, dP))) return rc;
    // the floats: straight into device outputs, or into the idle population
    // buffer (at least (d + 3) floats per node in every storage format)
    float* idle = static_cast<float*>(h->pop[h->cur ^ 1]);
    struct Field {
        const double* src;
        float* dst;
        long long n;
    } fields[4] = {{dr, rho, nn}, {du, u, h->D * nn}, {dT, T, nn}, {dP, P, nn}};
    long long off = 0;
    for (const Field& f : fields) {
        if (!f.dst) continue;
        float* d = mem == LBM_MEM_DEVICE ? f.dst : idle + off;
        const unsigned blocks = (unsigned)std::min<long long>((f.n + 255) / 256, 4096);
        narrow_kernel<<<blocks, 256, 0, h->stream>>>(f.src, d, f.n);
        if ((rc = cuda_error(cudaGetLastError(), "moments narrowing launch"))) return rc;
        if (mem == LBM_MEM_HOST &&
            (rc = cuda_error(cudaMemcpyAsync(f.dst, d, sizeof(float) * (size_t)f.n, cudaMemcpyDeviceToHost, h->stream),
                             "moments copy")))
            return rc;
        off += f.n;
    }
    return sync_and_latch(h);
}

int lbm_diagnostics(lbm_handle* h, double out[8]) {
    lbm::TraceRange trace_("lbm_diagnostics");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    if (!out) {
        set_error("lbm_diagnostics: null output");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    double* res = h->partials + lbm::kSums * lbm::kReduceBlocks;
    int rc;
    if ((rc = be_reduce(h, res))) return rc;
    double sums[lbm::kSums];
    lbm::Counters c;
    if ((rc = cuda_error(cudaMemcpyAsync(sums, res, sizeof(sums), cudaMemcpyDeviceToHost, h->stream), "diag copy")))
        return rc;
    if ((rc = cuda_error(cudaMemcpyAsync(&c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "diag copy")))
        return rc;
    if ((rc = sync_and_latch(h)) == LBM_ERR_CUDA || rc == LBM_ERR_TIMEOUT) return rc;
    for (int q = 0; q < lbm::kSums; ++q) out[q] = sums[q];
    out[5] = (double)c.clamps;
    out[6] = (double)c.bad;
    out[7] = (double)h->steps;
    return rc;
}

size_t lbm_state_bytes(const lbm_handle* h) {
    if (!h) return 0;
    return kStateHeader + (size_t)2 * h->Q * h->nn * h->elem;
}

int lbm_get_state(lbm_handle* h, void* buf, int mem) {
    lbm::TraceRange trace_("lbm_get_state");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    if (int rc = no_pending(h, "lbm_get_state")) return rc;   // converts in the idle buffer
    if (!buf || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE)) {
        set_error("lbm_get_state: null buffer or bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    unsigned char hdr[kStateHeader];
    const uint32_t magic = kStateMagic;
    const uint16_t q = (uint16_t)h->Q, st = (uint16_t)h->p.storage;
    const int64_t steps = h->steps;
    std::memcpy(hdr, &magic, 4);
    std::memcpy(hdr + 4, &q, 2);
    std::memcpy(hdr + 6, &st, 2);
    std::memcpy(hdr + 8, &steps, 8);
    const cudaMemcpyKind k_h = mem == LBM_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k_d = mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    int rc;
    if ((rc = cuda_error(cudaMemcpyAsync(buf, hdr, kStateHeader, k_h, h->stream), "state copy"))) return rc;
    // set-major planes, formed in the idle population buffer (the next step
    // overwrites all of it)
    void* idle = h->pop[h->cur ^ 1];
    if ((rc = convert_layout(h->pop[h->cur], idle, (long long)h->Q * h->nn, h->elem, false, h->stream))) return rc;
    if ((rc = cuda_error(cudaMemcpyAsync((unsigned char*)buf + kStateHeader, idle, lbm_state_bytes(h) - kStateHeader,
                                         k_d, h->stream),
                         "state copy")))
        return rc;
    return sync_and_latch(h);
}

int lbm_set_state(lbm_handle* h, const void* buf, int mem) {
    lbm::TraceRange trace_("lbm_set_state");
    if (int rc = check_handle(h)) return rc;
    if (int rc = no_pending(h, "lbm_set_state")) return rc;
    if (!buf || (mem != LBM_MEM_HOST && mem != LBM_MEM_DEVICE)) {
        set_error("lbm_set_state: null buffer or bad mem flag");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    unsigned char hdr[kStateHeader];
    int rc;
    if ((rc = cuda_error(cudaMemcpy(hdr, buf, kStateHeader,
                                    mem == LBM_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost),
                         "state header read")))
        return rc;
    uint32_t magic;
    uint16_t q, st;
    int64_t steps;
    std::memcpy(&magic, hdr, 4);
    std::memcpy(&q, hdr + 4, 2);
    std::memcpy(&st, hdr + 6, 2);
    std::memcpy(&steps, hdr + 8, 8);
    if (magic != kStateMagic || q != h->Q || st != h->p.storage) {
        set_error("lbm_set_state: buffer does not hold a state of this lattice and storage format");
        return LBM_ERR_INVALID_ARG;
    }
    void* idle = h->pop[h->cur ^ 1];
    if ((rc = cuda_error(cudaMemcpyAsync(idle, (const unsigned char*)buf + kStateHeader,
                                         lbm_state_bytes(h) - kStateHeader,
                                         mem == LBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                         h->stream),
                         "state copy")))
        return rc;
    if ((rc = convert_layout(idle, h->pop[h->cur], (long long)h->Q * h->nn, h->elem, true, h->stream))) return rc;
    if ((rc = cuda_error(cudaMemsetAsync(h->cnt, 0, sizeof(lbm::Counters), h->stream), "counter reset"))) return rc;
    if ((rc = cuda_error(cudaStreamSynchronize(h->stream), "stream synchronize"))) return rc;
    h->reported_bad = 0;
    h->steps = steps;
    h->initialised = true;
    return LBM_OK;
}

int lbm_sync(lbm_handle* h) {
    lbm::TraceRange trace_("lbm_sync");
    if (int rc = check_handle(h)) return rc;
    DeviceGuard dg(h->p.device);
    return sync_and_latch(h);
}

int lbm_launches_per_step(const lbm_handle* h) {
    if (!h) return 0;
    return h->Q == 9 ? lbm::Backend<9>::launches(h) : lbm::Backend<19>::launches(h);
}

int lbm_profile_step(lbm_handle* h, int n, double* ms, int cap) {
    lbm::TraceRange trace_("lbm_profile_step");
    if (int rc = check_handle(h)) return rc;
    if (int rc = need_init(h)) return rc;
    if (int rc = no_pending(h, "lbm_profile_step")) return rc;
    if (n < 1 || !ms || cap < 1) {
        set_error("lbm_profile_step: need n >= 1 and an output array");
        return LBM_ERR_INVALID_ARG;
    }
    DeviceGuard dg(h->p.device);
    int r = h->Q == 9 ? lbm::Backend<9>::profile(h, n, ms, cap) : lbm::Backend<19>::profile(h, n, ms, cap);
    if (r > 0) h->steps += n;
    return r;
}

const char* lbm_launch_name(const lbm_handle* h, int j) {
    if (!h) return "";
    return h->Q == 9 ? lbm::Backend<9>::launch_name(h, j) : lbm::Backend<19>::launch_name(h, j);
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    DeviceGuard dg(h->p.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->pop[0]);
    cudaFree(h->pop[1]);
    cudaFree(h->fld);
    cudaFree(h->cnt);
    cudaFree(h->partials);
    cudaFree(h->staging);
    cudaFree(h->coex);
    delete h;
}

int lbm_test_drop_handoff(lbm_handle* h, int plane) {
    if (int rc = check_handle(h)) return rc;
    h->fault_drop = plane < 0 ? 0 : plane + 1;
    return LBM_OK;
}

const char* lbm_last_error(void) { return lbm::g_error.c_str(); }

}  // extern "C"
