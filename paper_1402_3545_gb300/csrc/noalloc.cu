// noalloc.cu -- r = f - A u and ||r||_2 without any device allocation.
//
// For callers that must not allocate device memory once they are running: applications whose
// framework already owns nearly all device memory through its own pool (a raw cudaMalloc there
// can fail or fragment the pool), and latency-critical loops where cudaMalloc's implicit device
// synchronisation is not acceptable. The regular entry points allocate their workspace inside an
// operator object; this one takes the level's coefficients directly and keeps its only scratch --
// one partial sum per thread block -- in a file-scope __device__ array of fixed size.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.cuh"
#include "tpmg.h"

using namespace tpmg;

// Per-block partial sums of ||r||^2. Every GPU that loads the library holds this array (512 KB)
// until the process exits; every call on a device shares it.
static __device__ __align__(256) double g_noalloc_partials[TPMG_NOALLOC_MAX_BLOCKS];

static constexpr int MAX_DEVICES = 64;
static double* g_partials_addr[MAX_DEVICES] = {};
static std::mutex g_setup_mutex;
static thread_local std::string g_noalloc_err;

// Device address of g_noalloc_partials for the current device. In host code the symbol's name is
// only a host-side stand-in, so the address is looked up once per device with that device current.
static cudaError_t partials_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

extern "C" const char* tpmg_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" tpmg_status tpmg_residual_norm_noalloc(int nx, int ny, int nz, double cx, double cy, const double* v,
                                                  const double* u, const double* f, double* r,
                                                  double* norm_out, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !v || !u || !f || !r || !norm_out) {
        g_noalloc_err = "tpmg_residual_norm_noalloc: sizes must be >= 1 and pointers non-NULL";
        return TPMG_ERR_ARG;
    }
    Lv<PolF64> L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.cx = cx;
    L.cy = cy;
    L.v = v;
    L.finv = nullptr;
    L.fw = nullptr;
    L.fac_percol = 0;
    L.variant = -1;
    // the block count is planned by the same decisions the launch takes, and checked against the
    // fixed array before anything is launched: no kernel ever writes past its end
    const int nblocks = residual_launch_blocks<PolF64, PolF64>(L, u, f, r);
    if (nblocks < 1 || nblocks > TPMG_NOALLOC_MAX_BLOCKS) {
        g_noalloc_err = "tpmg_residual_norm_noalloc: " + std::to_string(nblocks) +
                        " thread blocks needed, the fixed scratch holds " +
                        std::to_string(TPMG_NOALLOC_MAX_BLOCKS) + " (grid too large for its kernel)";
        return TPMG_ERR_ARG;
    }
    double* partials = nullptr;
    cudaError_t e = partials_for_current_device(&partials);
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return TPMG_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // every entry that the sum reads is written by this call's residual kernel before the
    // finalize kernel runs (same stream), so nothing has to be cleared beforehand
    const int launched = launch_residual<PolF64, PolF64>(L, u, f, r, partials, nullptr, s);
    if (launched != nblocks) {
        g_noalloc_err = "tpmg_residual_norm_noalloc: internal block-count mismatch";
        return TPMG_ERR_CUDA;
    }
    launch_finalize_norm(partials, nblocks, FIN_STORE, nullptr, nullptr, norm_out, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("launch: ") + cudaGetErrorString(e);
        return TPMG_ERR_CUDA;
    }
    return TPMG_OK;
}
