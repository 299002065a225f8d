// k_probe.cu -- measured arithmetic rates of this GPU, the denominators of the ALU rooflines.
//
// The stencil and line-solve kernels move about 24 bytes per 12 arithmetic operations in FP64; on a
// part whose FP64 pipe is narrow that pipe, not HBM, bounds them. The probe measures the rate the
// pipe sustains on independent chains of one operation: every thread of a full-occupancy grid runs
// NCH independent accumulators through `iters` dependent steps, so the pipe always has work and the
// latency of one step is hidden by the other chains and warps.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "tpmg.h"

namespace tpmg {

static constexpr int PROBE_NCH = 8;
static constexpr int PROBE_NT = 256;

template <class T, int OP>
__global__ void __launch_bounds__(PROBE_NT) k_alu_probe(int iters, T b, T c, T* sink) {
    T a[PROBE_NCH];
#pragma unroll
    for (int q = 0; q < PROBE_NCH; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < PROBE_NCH; ++q) {
            if (OP == 0) a[q] = fma(a[q], b, c);  // multiply-add
            if (OP == 1) a[q] = a[q] + c;         // add
            if (OP == 2) a[q] = a[q] * b;         // multiply
        }
    }
    T s = 0;
#pragma unroll
    for (int q = 0; q < PROBE_NCH; ++q) s += a[q];
    // never true for the arguments the host passes; keeps the chains from being removed
    if (s == (T)-1.25e30) sink[blockIdx.x * PROBE_NT + threadIdx.x] = s;
}

template <class T, int OP>
static cudaError_t run_probe(int iters, int blocks, T* sink, cudaStream_t s) {
    // b close to 1 and c small keep every value finite and normal over any number of steps
    k_alu_probe<T, OP><<<blocks, PROBE_NT, 0, s>>>(iters, (T)0.999999, (T)1e-6, sink);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpmg

using namespace tpmg;

extern "C" tpmg_status tpmg_measure_alu_rate(int which, int reps, double* ops_per_s, double* ms_per_launch) {
    if (which < 0 || which > 3 || reps < 1 || !ops_per_s) return TPMG_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int blocks = sms * (per_sm / PROBE_NT);
    const int iters = (which == 3) ? 1 << 16 : 1 << 11;  // FP32 is many times faster: more steps
    void* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * PROBE_NT * sizeof(double)) != cudaSuccess) return TPMG_ERR_OOM;
    cudaStream_t s = nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() -> cudaError_t {
        switch (which) {
            case 0: return run_probe<double, 0>(iters, blocks, (double*)sink, s);
            case 1: return run_probe<double, 1>(iters, blocks, (double*)sink, s);
            case 2: return run_probe<double, 2>(iters, blocks, (double*)sink, s);
            default: return run_probe<float, 0>(iters, blocks, (float*)sink, s);
        }
    };
    cudaError_t err = launch();  // warm-up
    float best = 0.0f;
    for (int r = 0; r < reps && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        err = launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r == 0 || t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return TPMG_ERR_CUDA;
    const double ops = (double)blocks * PROBE_NT * PROBE_NCH * (double)iters;
    *ops_per_s = ops / (best * 1e-3);
    if (ms_per_launch) *ms_per_launch = best;
    return TPMG_OK;
}
