// k_fcg.cu -- flexible CG(1) with a variable preconditioner (Notay 2000), on double-word vectors:
// the search direction is the preconditioned residual A-orthogonalised against the previous
// direction only, which tolerates a preconditioner that changes between applications (here: an
// FP32 V-cycle followed by the learned correction, accepted only when it lowers the residual).
//
// The scalars live on the device (FcgScalars); every decision -- alpha, beta, convergence, whether
// the learned correction is kept -- is taken by single-thread kernels, the host only reads the flag.
#include <math.h>

#include "fcg.cuh"
#include "kernels.cuh"

namespace tpmg {

__device__ __forceinline__ int fwrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// q = A p; partial sums of <p, q> and <p, r> (two per block)
__global__ void __launch_bounds__(128) k_fcg_apply(Lv<PolDW> L, const float2* __restrict__ p, const float2* __restrict__ r,
                                                   float2* __restrict__ q, double* partials) {
    typedef PolDW P;
    typedef P::R R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool act = i < L.nx && j < L.ny;
    P::Acc s1 = 0, c1 = 0, s2 = 0, c2 = 0;
    if (act) {
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const size_t pl = (size_t)nx * ny, c = (size_t)j * nx + i;
        const size_t cw = (size_t)j * nx + fwrap(i - 1, nx), ce = (size_t)j * nx + fwrap(i + 1, nx);
        const size_t cs = (size_t)fwrap(j - 1, ny) * nx + i, cn = (size_t)fwrap(j + 1, ny) * nx + i;
        const R cx = P::cst(L.cx), cy = P::cst(L.cy), vv = P::ld(L.v, c);
        const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy), dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        R pm = P::zero(), pc = P::ld(p, c);
        for (int k = 0; k < nz; ++k) {
            const size_t b = (size_t)k * pl;
            const R pp = (k + 1 < nz) ? P::ld(p, b + pl + c) : P::zero();
            const R hx = P::add(P::ld(p, b + cw), P::ld(p, b + ce));
            const R hy = P::add(P::ld(p, b + cs), P::ld(p, b + cn));
            const R diag = (nz == 1) ? dh : ((k == 0 || k == nz - 1) ? dh1 : dh2);
            R ap = P::mul(diag, pc);
            ap = P::sub(ap, P::mul(cx, hx));
            ap = P::sub(ap, P::mul(cy, hy));
            ap = P::sub(ap, P::mul(vv, P::add(pm, pp)));
            P::st(q, b + c, ap);
            P::acc_dot(s1, c1, pc, ap);
            P::acc_dot(s2, c2, pc, P::ld(r, b + c));
            pm = pc;
            pc = pp;
        }
    }
    const double a = block_sum(P::acc_get(s1, c1));
    const double b2 = block_sum(P::acc_get(s2, c2));
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
        partials[blk] = a;
        partials[nb + blk] = b2;
    }
}

// u += alpha p ; r -= alpha q ; partial sums of ||r||^2
__global__ void __launch_bounds__(256) k_fcg_update(size_t n, const FcgScalars* sc, float2* __restrict__ u,
                                                    const float2* __restrict__ p, float2* __restrict__ r,
                                                    const float2* __restrict__ q, double* partials) {
    typedef PolDW P;
    if (*(volatile const int*)&sc->done) return;
    const P::R al = P::cst(sc->alpha);
    P::Acc s = 0, c = 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        P::st(u, t, P::add(P::ld_plain(u, t), P::mul(al, P::ld(p, t))));
        const P::R rn = P::sub(P::ld_plain(r, t), P::mul(al, P::ld(q, t)));
        P::st(r, t, rn);
        P::acc_dot(s, c, rn, rn);
    }
    const double tot = block_sum(P::acc_get(s, c));
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// partial sums of <a, b>
__global__ void __launch_bounds__(256) k_fcg_dot(size_t n, const float2* __restrict__ a, const float2* __restrict__ b,
                                                 double* partials) {
    typedef PolDW P;
    P::Acc s = 0, c = 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        P::acc_dot(s, c, P::ld(a, t), P::ld(b, t));
    const double tot = block_sum(P::acc_get(s, c));
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// p = z - beta p
__global__ void __launch_bounds__(256) k_fcg_direction(size_t n, const FcgScalars* sc, const float2* __restrict__ z,
                                                       float2* __restrict__ p) {
    typedef PolDW P;
    if (*(volatile const int*)&sc->done) return;
    const P::R be = P::cst(sc->beta);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        P::st(p, t, P::sub(P::ld(z, t), P::mul(be, P::ld_plain(p, t))));
}

// c = z1 + s D^{-1} y with s = ||r1|| / sqrt(n) (the input normalisation), D = diag(A) and y the
// network output (fp32)
__global__ void __launch_bounds__(256) k_fcg_learned(size_t n, size_t ncol, int nz, float cx2cy2,
                                                     const float* __restrict__ v32, const FcgScalars* sc,
                                                     const float2* __restrict__ z1, const float* __restrict__ y,
                                                     float2* __restrict__ c) {
    typedef PolDW P;
    const double rms = sqrt(sc->r1sq / (double)n);
    const P::R s = P::cst(rms);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t col = t % ncol;
        const int k = (int)(t / ncol);
        const float yd = __ldg(y + t) * diag_inv_f32(cx2cy2, __ldg(v32 + col), k, nz);
        P::st(c, t, P::add(P::ld(z1, t), dw_mul_f(s, yd)));
    }
}

// z = keep ? c : z1 (decided on the device by k_fcg_scalar mode FCG_DECIDE)
__global__ void __launch_bounds__(256) k_fcg_select(size_t n, const FcgScalars* sc, const float2* __restrict__ c,
                                                    const float2* __restrict__ z1, float2* __restrict__ z) {
    const bool keep = sc->keep != 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        z[t] = keep ? c[t] : z1[t];
}

// double-word from fp32 (the V-cycle correction) and fp32 from double-word (the residual handed to it)
__global__ void k_dw_from_f32(size_t n, const float* __restrict__ a, float2* __restrict__ b) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        b[t] = make_float2(a[t], 0.f);
}
__global__ void k_f32_from_dw(size_t n, const float2* __restrict__ a, float* __restrict__ b) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        b[t] = __fadd_rn(a[t].x, a[t].y);
}

// scalar steps of the iteration: the block adds the partial sums in a fixed order (thread t takes
// entries t, t+256, ...; then a fixed tree), thread 0 takes the decision
static constexpr int FS = 256;
__device__ double fsum(const double* a, int n) {
    __shared__ double buf[FS];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += FS) s += a[t];
    buf[threadIdx.x] = s;
    __syncthreads();
    for (int h = FS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) buf[threadIdx.x] += buf[threadIdx.x + h];
        __syncthreads();
    }
    const double r = buf[0];
    __syncthreads();
    return r;
}
__global__ void __launch_bounds__(FS) k_fcg_scalar(int mode, const double* partials, int nparts, FcgScalars* sc,
                                                   double* history) {
    const double s0 = fsum(partials, nparts);
    const double s1 = mode == FCG_ALPHA ? fsum(partials + nparts, nparts) : 0.0;
    if (threadIdx.x != 0) return;
    switch (mode) {
        case FCG_INIT_NORM: {  // r0 from partials of ||r||^2
            const double nr = sqrt(s0);
            sc->r0 = nr;
            sc->rel = 1.0;
            sc->iters = 0;
            if (history) history[0] = 1.0;
            if (!isfinite(nr)) {
                sc->nonfinite = 1;
                sc->done = 1;
            } else if (nr == 0.0) {
                sc->converged = 1;
                sc->done = 1;
            } else if (sc->max_iter <= 0) {
                sc->done = 1;
            }
            break;
        }
        case FCG_ALPHA: {  // partials: <p,q> then <p,r>
            if (sc->done) break;
            const double pq = s0, pr = s1;
            sc->pq = pq;
            if (!isfinite(pq) || !isfinite(pr) || pq <= 0.0) {
                sc->nonfinite = !isfinite(pq) || !isfinite(pr);
                sc->alpha = 0.0;
                sc->done = 1;
            } else {
                sc->alpha = pr / pq;
            }
            break;
        }
        case FCG_CHECK: {  // after the update: partials of ||r||^2
            if (sc->done) break;
            const double nr = sqrt(s0);
            const int it = ++sc->iters;
            sc->rel = nr / sc->r0;
            if (history) history[it] = sc->rel;
            if (!isfinite(nr)) {
                sc->nonfinite = 1;
                sc->done = 1;
            } else if (sc->rel < sc->tol) {
                sc->converged = 1;
                sc->done = 1;
            } else if (it >= sc->max_iter) {
                sc->done = 1;
            }
            break;
        }
        case FCG_BETA: {  // partials of <z, q>
            if (sc->done) break;
            sc->beta = s0 / sc->pq;
            break;
        }
        case FCG_R1: {  // partials of ||r - A z1||^2
            sc->r1sq = s0;
            break;
        }
        case FCG_DECIDE: {  // partials of ||r - A c||^2: keep the learned correction only if it helps
            const double r2 = s0;
            const bool keep = isfinite(r2) && isfinite(sc->r1sq) && r2 < sc->r1sq;
            sc->keep = keep;
            if (keep) sc->accepted++;
            else sc->rejected++;
            break;
        }
        default:
            break;
    }
}

__global__ void k_fcg_init(FcgScalars* sc, double tol, int max_iter) {
    FcgScalars s;
    s.r0 = s.rel = s.alpha = s.beta = s.pq = s.r1sq = 0.0;
    s.tol = tol;
    s.iters = 0;
    s.max_iter = max_iter;
    s.done = s.converged = s.nonfinite = s.keep = s.accepted = s.rejected = 0;
    *sc = s;
}

// ---------------------------------------------------------------- launchers
static unsigned grid_n(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > FCG_MAX_BLOCKS) b = FCG_MAX_BLOCKS;
    return (unsigned)(b ? b : 1);
}
int fcg_apply(const Lv<PolDW>& L, const float2* p, const float2* r, float2* q, double* partials, cudaStream_t s) {
    dim3 blk(32, 4), grd((L.nx + 31) / 32, (L.ny + 3) / 4);
    k_fcg_apply<<<grd, blk, 0, s>>>(L, p, r, q, partials);
    note_launch();
    return (int)(grd.x * grd.y);
}
int fcg_update(size_t n, const FcgScalars* sc, float2* u, const float2* p, float2* r, const float2* q, double* partials,
               cudaStream_t s) {
    k_fcg_update<<<grid_n(n), 256, 0, s>>>(n, sc, u, p, r, q, partials);
    note_launch();
    return (int)grid_n(n);
}
int fcg_dot(size_t n, const float2* a, const float2* b, double* partials, cudaStream_t s) {
    k_fcg_dot<<<grid_n(n), 256, 0, s>>>(n, a, b, partials);
    note_launch();
    return (int)grid_n(n);
}
void fcg_direction(size_t n, const FcgScalars* sc, const float2* z, float2* p, cudaStream_t s) {
    k_fcg_direction<<<grid_n(n), 256, 0, s>>>(n, sc, z, p);
    note_launch();
}
void fcg_learned(size_t n, size_t ncol, int nz, double cx, double cy, const float* v32, const FcgScalars* sc,
                 const float2* z1, const float* y, float2* c, cudaStream_t s) {
    k_fcg_learned<<<grid_n(n), 256, 0, s>>>(n, ncol, nz, (float)(2.0 * cx + 2.0 * cy), v32, sc, z1, y, c);
    note_launch();
}
void fcg_select(size_t n, const FcgScalars* sc, const float2* c, const float2* z1, float2* z, cudaStream_t s) {
    k_fcg_select<<<grid_n(n), 256, 0, s>>>(n, sc, c, z1, z);
    note_launch();
}
void fcg_dw_from_f32(size_t n, const float* a, float2* b, cudaStream_t s) {
    k_dw_from_f32<<<grid_n(n), 256, 0, s>>>(n, a, b);
    note_launch();
}
void fcg_f32_from_dw(size_t n, const float2* a, float* b, cudaStream_t s) {
    k_f32_from_dw<<<grid_n(n), 256, 0, s>>>(n, a, b);
    note_launch();
}
void fcg_scalar(int mode, const double* partials, int nparts, FcgScalars* sc, double* history, cudaStream_t s) {
    k_fcg_scalar<<<1, FS, 0, s>>>(mode, partials, nparts, sc, history);
    note_launch();
}
void fcg_init(FcgScalars* sc, double tol, int max_iter, cudaStream_t s) {
    k_fcg_init<<<1, 1, 0, s>>>(sc, tol, max_iter);
    note_launch();
}

}  // namespace tpmg
