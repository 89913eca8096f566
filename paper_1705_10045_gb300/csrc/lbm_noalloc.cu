// Conservation sums without any device allocation (lbm_conservation_sums_noalloc).
//
// Some callers cannot allocate device memory: programs whose device memory is
// owned by another framework's pool (every byte must come from that pool), and
// loops that must not let an allocation synchronise the device and stall
// their other streams.  For them this entry point computes the same
// compensated sums as lbm_diagnostics (per-thread partials, combined in FP64)
// on a population buffer they own, using only a fixed scratch array that is
// part of the loaded library image.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds it (40,960 bytes) until the process exits.  Its name in host
// code is only a host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, by the
// first call made on it; that first call should come before any stream
// capture.  The address is kept for the life of the process, so the call must
// not be used on a device after cudaDeviceReset (which unloads the library's
// device image).  All calls share the array: the reduction overwrites every
// block partial it reads, so nothing has to start at zero, but two calls
// whose kernels overlap on the GPU (different streams without ordering) race
// on it.
#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.cuh"

namespace {

constexpr int kScratchDoubles = lbm::kSums * lbm::kReduceBlocks;   // one partial per block and sum
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once)
int scratch_for_current_device(double** out) {
    int dev = -1;
    if (int rc = lbm::cuda_error(cudaGetDevice(&dev), "lbm_conservation_sums_noalloc: cudaGetDevice")) return rc;
    if (dev < 0 || dev >= kMaxDevices) {
        lbm::set_error("lbm_conservation_sums_noalloc: device ordinal beyond the supported 64");
        return LBM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (int rc = lbm::cuda_error(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                                     "lbm_conservation_sums_noalloc: cudaGetSymbolAddress"))
            return rc;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

template <int Q, typename S, typename R>
int launch_sums(int nx, int ny, int nz, double rho_ref, double E_ref, const void* pop, double* scratch,
                double* sums, cudaStream_t stream) {
    lbm::KParams<R> kp{};
    kp.nx = nx;
    kp.ny = ny;
    kp.nz = nz;
    kp.nn = (long long)nx * ny * nz;
    kp.rho_ref = (R)rho_ref;
    kp.E_ref = (R)E_ref;
    // the caller's buffer holds set-major planes (the checkpoint layout)
    lbm::reduce_kernel<Q, S, R, false>
        <<<lbm::kReduceBlocks, lbm::kReduceThreads, 0, stream>>>((const S*)pop, kp, scratch);
    lbm::reduce_final_kernel<<<1, 32, 0, stream>>>(scratch, lbm::kReduceBlocks, sums);
    return lbm::cuda_error(cudaGetLastError(), "lbm_conservation_sums_noalloc launch");
}

}  // namespace

extern "C" int lbm_conservation_sums_noalloc(int lattice, int storage, int nx, int ny, int nz, double rho_ref,
                                             double E_ref, const void* populations, double* sums, void* stream) {
    if (!populations || !sums) {
        lbm::set_error("lbm_conservation_sums_noalloc: null populations or sums");
        return LBM_ERR_INVALID_ARG;
    }
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) {
        lbm::set_error("lbm_conservation_sums_noalloc: lattice must be LBM_D2Q9 or LBM_D3Q19");
        return LBM_ERR_INVALID_ARG;
    }
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == LBM_D2Q9 && nz != 1)) {
        lbm::set_error("lbm_conservation_sums_noalloc: sizes must be >= 1 and nz must be 1 for D2Q9");
        return LBM_ERR_INVALID_ARG;
    }
    if ((long long)nx * ny * nz >= (1ll << 31)) {
        lbm::set_error("lbm_conservation_sums_noalloc: at most 2^31 - 1 nodes, the largest domain lbm_create "
                       "accepts");
        return LBM_ERR_INVALID_ARG;
    }
    if (storage < LBM_STORE_FP64 || storage > LBM_STORE_FP16) {
        lbm::set_error("lbm_conservation_sums_noalloc: unknown storage format");
        return LBM_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    if (int rc = scratch_for_current_device(&scratch)) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    // the FP16 shifts only apply to shifted storage, as in the library's own kernels
    const double rr = storage == LBM_STORE_FP16 ? rho_ref : 0.0, er = storage == LBM_STORE_FP16 ? E_ref : 0.0;
    if (lattice == LBM_D2Q9) {
        switch (storage) {
            case LBM_STORE_FP64: return launch_sums<9, double, double>(nx, ny, nz, rr, er, populations, scratch, sums, s);
            case LBM_STORE_FP32: return launch_sums<9, float, float>(nx, ny, nz, rr, er, populations, scratch, sums, s);
            default: return launch_sums<9, __half, float>(nx, ny, nz, rr, er, populations, scratch, sums, s);
        }
    }
    switch (storage) {
        case LBM_STORE_FP64: return launch_sums<19, double, double>(nx, ny, nz, rr, er, populations, scratch, sums, s);
        case LBM_STORE_FP32: return launch_sums<19, float, float>(nx, ny, nz, rr, er, populations, scratch, sums, s);
        default: return launch_sums<19, __half, float>(nx, ny, nz, rr, er, populations, scratch, sums, s);
    }
}
