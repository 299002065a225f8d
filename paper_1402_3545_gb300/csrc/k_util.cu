// k_util.cu -- single-block finalize kernels that turn per-block partial sums into the solver's
// scalars on the device (norms, CG's alpha and beta, the convergence decision of Eq. (10)), and
// the precision conversion kernels.
//
// The partial sums are added in a fixed order (thread t adds entries t, t+256, ...; then a fixed
// tree), so every reduction is deterministic: two identical solves give identical iterates.
#include <math.h>

#include "kernels.cuh"

namespace tpmg {

static constexpr int FT = 256;

unsigned long long& launch_counter() {
    static unsigned long long count = 0;
    return count;
}

__device__ double ordered_sum(const double* a, int n) {
    __shared__ double buf[FT];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += FT) s += a[t];
    buf[threadIdx.x] = s;
    __syncthreads();
    for (int h = FT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) buf[threadIdx.x] += buf[threadIdx.x + h];
        __syncthreads();
    }
    double r = buf[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

__global__ void k_finalize_norm(const double* __restrict__ partials, int nparts, int mode,
                                Scalars* sc, double* history, double* out) {
    if (mode == FIN_MG_CYCLE && *(volatile int*)&sc->done) return;
    double ss = ordered_sum(partials, nparts);
    if (threadIdx.x != 0) return;
    if (mode == FIN_SUM) {
        if (out) *out = ss;
        return;
    }
    double nrm = sqrt(ss);
    if (out) *out = nrm;
    if (mode == FIN_STORE) return;
    sc->last_norm = nrm;
    if (!finite_d(nrm)) {
        sc->nonfinite = 1;
        sc->done = 1;
        return;
    }
    if (mode == FIN_MG_INIT) {
        sc->r0 = nrm;
        sc->rel = 1.0;
        sc->iters = 0;
        if (history) history[0] = 1.0;
        if (nrm == 0.0) {
            sc->converged = 1;
            sc->done = 1;
        } else if (sc->max_iter <= 0) {
            sc->done = 1;
        }
        return;
    }
    // FIN_MG_CYCLE: the norm belongs to the iterate after cycle number ++iters
    int it = ++sc->iters;
    double rel = nrm / sc->r0;
    sc->rel = rel;
    if (history) history[it] = rel;
    if (rel < sc->tol) {
        sc->converged = 1;
        sc->done = 1;
    } else if (it >= sc->max_iter) {
        sc->done = 1;
    }
}

// alpha = <r,z> / <p, A p>
__global__ void k_cg_alpha(const double* __restrict__ partials, int nparts, Scalars* sc) {
    if (*(volatile int*)&sc->done) return;
    double sigma = ordered_sum(partials, nparts);
    if (threadIdx.x != 0) return;
    if (!finite_d(sigma)) {
        sc->nonfinite = 1;
        sc->alpha = 0.0;
        sc->done = 1;
    } else if (sigma <= 0.0) {  // p = 0 (exact solution reached) or loss of positivity
        sc->alpha = 0.0;
        sc->done = 1;
    } else {
        sc->alpha = sc->kappa / sigma;
    }
}

// after the fused Tridiag: rel = ||r||/||r0||, beta = <r,z>_new / <r,z>_old
__global__ void k_cg_beta(const double* __restrict__ partials, int nparts, int init, Scalars* sc,
                          double* history) {
    if (*(volatile int*)&sc->done) return;
    double rr = ordered_sum(partials, nparts);
    double rz = ordered_sum(partials + nparts, nparts);
    if (threadIdx.x != 0) return;
    double nrm = sqrt(rr);
    sc->last_norm = nrm;
    if (!finite_d(nrm) || !finite_d(rz)) {
        sc->nonfinite = 1;
        sc->done = 1;
        return;
    }
    if (init) {
        sc->r0 = nrm;
        sc->rel = 1.0;
        sc->iters = 0;
        sc->kappa = rz;
        sc->alpha = 0.0;
        sc->beta = 0.0;
        if (history) history[0] = 1.0;
        if (nrm == 0.0) {
            sc->converged = 1;
            sc->done = 1;
        } else if (sc->max_iter <= 0) {
            sc->done = 1;
        }
        return;
    }
    int it = ++sc->iters;
    double rel = nrm / sc->r0;
    sc->rel = rel;
    if (history) history[it] = rel;
    sc->beta = rz / sc->kappa;
    sc->kappa = rz;
    if (rel < sc->tol) {
        sc->converged = 1;
        sc->done = 1;
    } else if (it >= sc->max_iter) {
        sc->done = 1;
    }
}

__global__ void k_scalars_init(Scalars* sc, double tol, int max_iter) {
    Scalars s;
    s.r0 = 0.0;
    s.rel = 0.0;
    s.tol = tol;
    s.alpha = 0.0;
    s.beta = 0.0;
    s.kappa = 0.0;
    s.last_norm = 0.0;
    s.iters = 0;
    s.max_iter = max_iter;
    s.done = 0;
    s.converged = 0;
    s.nonfinite = 0;
    s.pad = 0;
    *sc = s;
}

__global__ void k_set_ab(Scalars* sc, double alpha, double beta) {
    sc->alpha = alpha;
    sc->beta = beta;
    sc->done = 0;
}

template <class S>
__global__ void k_copy(size_t n, const S* __restrict__ src, S* __restrict__ dst, const int* done) {
    if (done && *(volatile const int*)done) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        dst[t] = src[t];
}

__global__ void k_f64_to_dw(size_t n, const double* __restrict__ x, float2* __restrict__ y) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        double v = x[t];
        float h = __double2float_rn(v);
        y[t] = make_float2(h, __double2float_rn(v - (double)h));
    }
}
__global__ void k_dw_to_f64(size_t n, const float2* __restrict__ x, double* __restrict__ y) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        float2 v = x[t];
        y[t] = (double)v.x + (double)v.y;
    }
}
__global__ void k_f64_to_f32(size_t n, const double* __restrict__ x, float* __restrict__ y) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        y[t] = __double2float_rn(x[t]);
}
__global__ void k_f32_to_f64(size_t n, const float* __restrict__ x, double* __restrict__ y) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        y[t] = (double)x[t];
}
// coarse vertical coefficient: the average of the 2x2 children
__global__ void k_coarsen_v(int nxf, int nyf, const double* __restrict__ vf, double* __restrict__ vc) {
    const int nxc = nxf / 2, nyc = nyf / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= nxc || J >= nyc) return;
    const size_t a = (size_t)(2 * J) * nxf + 2 * I, b = a + nxf;
    vc[(size_t)J * nxc + I] = 0.25 * (vf[a] + vf[a + 1] + vf[b] + vf[b + 1]);
}

static unsigned grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b == 0) b = 1;
    return (unsigned)b;
}

void launch_finalize_norm(const double* partials, int nparts, int mode, Scalars* sc,
                          double* history, double* out, cudaStream_t s) {
    k_finalize_norm<<<1, FT, 0, s>>>(partials, nparts, mode, sc, history, out);
    note_launch();
}
void launch_cg_alpha(const double* partials, int nparts, Scalars* sc, cudaStream_t s) {
    k_cg_alpha<<<1, FT, 0, s>>>(partials, nparts, sc);
    note_launch();
}
void launch_cg_beta(const double* partials, int nparts, int init, Scalars* sc, double* history,
                    cudaStream_t s) {
    k_cg_beta<<<1, FT, 0, s>>>(partials, nparts, init, sc, history);
    note_launch();
}
void launch_scalars_init(Scalars* sc, double tol, int max_iter, cudaStream_t s) {
    k_scalars_init<<<1, 1, 0, s>>>(sc, tol, max_iter);
    note_launch();
}
void launch_set_ab(Scalars* sc, double alpha, double beta, cudaStream_t s) {
    k_set_ab<<<1, 1, 0, s>>>(sc, alpha, beta);
    note_launch();
}
template <class P>
void launch_copy(size_t n, const typename P::S* src, typename P::S* dst, const int* done, cudaStream_t s) {
    k_copy<typename P::S><<<grid_for(n), 256, 0, s>>>(n, src, dst, done);
    note_launch();
}
template void launch_copy<PolF64>(size_t, const double*, double*, const int*, cudaStream_t);
template void launch_copy<PolF32>(size_t, const float*, float*, const int*, cudaStream_t);
template void launch_copy<PolDW>(size_t, const float2*, float2*, const int*, cudaStream_t);

void launch_f64_to_dw(size_t n, const double* x, float2* y, cudaStream_t s) {
    k_f64_to_dw<<<grid_for(n), 256, 0, s>>>(n, x, y);
    note_launch();
}
void launch_dw_to_f64(size_t n, const float2* x, double* y, cudaStream_t s) {
    k_dw_to_f64<<<grid_for(n), 256, 0, s>>>(n, x, y);
    note_launch();
}
void launch_f64_to_f32(size_t n, const double* x, float* y, cudaStream_t s) {
    k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(n, x, y);
    note_launch();
}
void launch_f32_to_f64(size_t n, const float* x, double* y, cudaStream_t s) {
    k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(n, x, y);
    note_launch();
}
void launch_coarsen_v_f64(int nxf, int nyf, const double* vf, double* vc, cudaStream_t s) {
    dim3 blk(32, 8), grd((nxf / 2 + 31) / 32, (nyf / 2 + 7) / 8);
    k_coarsen_v<<<grd, blk, 0, s>>>(nxf, nyf, vf, vc);
    note_launch();
}

// ---------------------------------------------------------------- layout transposition
// out[c * rows + r] = in[r * cols + c]: a rows x cols row-major matrix transposed through 32 x 32
// tiles in shared memory, padded by one element per row so that neither the row-wise fill nor the
// column-wise drain of a tile meets a bank conflict; both global sides are read and written in
// 32-element rows (coalesced). Converts between the vertically contiguous field layout of CPU codes
// (column c = j*nx + i holds its nz values contiguously: rows = nx*ny, cols = nz) and the
// horizontally contiguous layout of the kernels (rows = nz, cols = nx*ny), Sec. 5.1.
template <class T>
__global__ void __launch_bounds__(256) k_transpose(const T* __restrict__ in, T* __restrict__ out, size_t rows,
                                                   size_t cols, size_t tiles_c) {
    __shared__ T tile[32][33];
    const size_t t = blockIdx.x;
    const size_t r0 = (t / tiles_c) * 32, c0 = (t % tiles_c) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads, four rows each
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const size_t r = r0 + ty + 8 * q, c = c0 + tx;
        if (r < rows && c < cols) tile[ty + 8 * q][tx] = in[r * cols + c];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const size_t c = c0 + ty + 8 * q, r = r0 + tx;
        if (r < rows && c < cols) out[c * rows + r] = tile[tx][ty + 8 * q];
    }
}

template <class T>
void launch_transpose(const T* in, T* out, size_t rows, size_t cols, cudaStream_t s) {
    const size_t tiles_r = (rows + 31) / 32, tiles_c = (cols + 31) / 32;
    k_transpose<T><<<(unsigned)(tiles_r * tiles_c), dim3(32, 8), 0, s>>>(in, out, rows, cols, tiles_c);
    note_launch();
}
template void launch_transpose<double>(const double*, double*, size_t, size_t, cudaStream_t);
template void launch_transpose<float>(const float*, float*, size_t, size_t, cudaStream_t);

}  // namespace tpmg
