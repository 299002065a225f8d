// k_coarse.cu -- cell-parallel kernels for the small levels of the hierarchy (at most
// PCR_MAX_COLS columns: 64 x 64 and below).
//
// The column kernels give each vertical column one thread, which leaves the GPU nearly idle on the
// coarse levels (a 16 x 16 level has 256 columns) and, on the levels the double-word solver runs in
// native FP64, serialises about 60 FP64 instructions per cell at 1/72 of the FP32 rate. Here every
// cell has its own thread: the stencil and the transfers are pointwise, and the column block
// M_c = tridiag(-v, D_k, -v) is solved by parallel cyclic reduction (PCR): with stride s = 1, 2, 4,
// ... each row eliminates its neighbours at distance s,
//     d_k <- d_k - alpha_k d_{k-s} - gamma_k d_{k+s},
// until after ceil(log2 nz) steps the rows decouple and x_k = d_k / b_k. The multipliers alpha,
// gamma and 1/b depend only on the operator, so they are computed once per level (k_pcr_factors)
// and a solve costs 2 ceil(log2 nz) + 1 multiply-adds per cell with a block barrier per step.
//
// PCR is backward stable on the diagonally dominant column blocks, so its forward error obeys the
// same kappa(M) u bound as the Thomas algorithm the column kernels use.
#include "kernels.cuh"

namespace tpmg {

__device__ __forceinline__ int cwrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ---------------------------------------------------------------- factors
// The PCR recurrences on the coefficients (a_k, b_k, c_k) = (-v [k>0], D_k, -v [k<nz-1]) of each
// column block: at step t (stride s = 2^t) row k takes alpha = a_k / b_{k-s}, gamma = c_k / b_{k+s}
// (0 beyond the ends) and becomes (-alpha a_{k-s}, b_k - alpha c_{k-s} - gamma a_{k+s},
// -gamma c_{k+s}). Stored: alpha and gamma per step and row, then 1/b of the decoupled rows.
// Layout: index ((2t + side) * nz + k) * ncolp + col, then (2S * nz + k) * ncolp + col, where
// ncolp = ncol when percol (lambda^2 varies over the level) else 1 (one shared table).
// Block: cpb columns x nz rows, the same shape as the solve; smem holds a, b, c of every row.
template <class P>
__global__ void __launch_bounds__(256) k_pcr_factors(Lv<P> L, typename P::S* __restrict__ pcr, int percol) {
    typedef typename P::R R;
    typedef typename P::S S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = L.nz, k = threadIdx.y, cpb = blockDim.x, tx = threadIdx.x;
    const int ncol = percol ? L.nx * L.ny : 1;
    const int col = blockIdx.x * cpb + tx;
    const bool act = col < ncol;
    const size_t ncolp = (size_t)ncol;
    S* sa = reinterpret_cast<S*>(smem_raw);
    S* sb = sa + (size_t)cpb * nz;
    S* sc = sb + (size_t)cpb * nz;
    const size_t me = (size_t)k * cpb + tx;
    const R vv = P::ld(L.v, act ? col : 0);
    const R mv = P::sub(P::zero(), vv);
    R b = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    if (k > 0) b = P::add(b, vv);
    if (k < nz - 1) b = P::add(b, vv);
    R a = k > 0 ? mv : P::zero(), c = k < nz - 1 ? mv : P::zero();
    for (int t = 0; t < L.pcr_steps; ++t) {
        const int s = 1 << t;
        P::st(sa, me, a);
        P::st(sb, me, b);
        P::st(sc, me, c);
        __syncthreads();
        R al = P::zero(), ga = P::zero(), an = P::zero(), cn = P::zero(), bn = b;
        if (k - s >= 0) {
            const size_t o = (size_t)(k - s) * cpb + tx;
            al = P::mul(a, P::rcp(P::ld_plain(sb, o)));
            an = P::sub(P::zero(), P::mul(al, P::ld_plain(sa, o)));
            bn = P::sub(bn, P::mul(al, P::ld_plain(sc, o)));
        }
        if (k + s < nz) {
            const size_t o = (size_t)(k + s) * cpb + tx;
            ga = P::mul(c, P::rcp(P::ld_plain(sb, o)));
            cn = P::sub(P::zero(), P::mul(ga, P::ld_plain(sc, o)));
            bn = P::sub(bn, P::mul(ga, P::ld_plain(sa, o)));
        }
        if (act) {
            P::st(pcr, ((size_t)(2 * t) * nz + k) * ncolp + col, al);
            P::st(pcr, ((size_t)(2 * t + 1) * nz + k) * ncolp + col, ga);
        }
        a = an;
        b = bn;
        c = cn;
        __syncthreads();
    }
    if (act) P::st(pcr, ((size_t)(2 * L.pcr_steps) * nz + k) * ncolp + col, P::rcp(b));
}

template <class P>
size_t pcr_factor_count(const Lv<P>& L, int percol) {
    return (size_t)(2 * L.pcr_steps + 1) * L.nz * (percol ? (size_t)L.nx * L.ny : 1);
}

static int pcr_cpb(int nz, int ncol);

template <class P>
void launch_pcr_factors(const Lv<P>& L, typename P::S* pcr, int percol, cudaStream_t s) {
    const int ncol = percol ? L.nx * L.ny : 1;
    const int cpb = pcr_cpb(L.nz, ncol);
    const int nb = (ncol + cpb - 1) / cpb;
    const size_t smem = 3 * (size_t)cpb * L.nz * sizeof(typename P::S);
    k_pcr_factors<P><<<nb, dim3(cpb, L.nz), smem, s>>>(L, pcr, percol);
    note_launch();
}

// ---------------------------------------------------------------- the block-wide PCR solve
// The block holds cpb = blockDim.x columns x nz rows (threadIdx.y = k); buf has cpb * nz values.
// Every thread of the block calls this (inactive columns with d = 0) because of the barriers.
template <class P>
__device__ __forceinline__ typename P::R pcr_solve(const Lv<P>& L, typename P::R d, typename P::S* buf, int col,
                                                   bool act) {
    typedef typename P::R R;
    const int nz = L.nz, k = threadIdx.y, cpb = blockDim.x, tx = threadIdx.x;
    const size_t ncolp = L.fac_percol ? (size_t)L.nx * L.ny : 1;
    const int colp = (L.fac_percol && act) ? col : 0;
    for (int t = 0; t < L.pcr_steps; ++t) {
        const int s = 1 << t;
        P::sts(buf, (size_t)k * cpb + tx, d);
        __syncthreads();
        const R dm = (k - s >= 0) ? P::ld_plain(buf, (size_t)(k - s) * cpb + tx) : P::zero();
        const R dp = (k + s < nz) ? P::ld_plain(buf, (size_t)(k + s) * cpb + tx) : P::zero();
        const R al = P::ld(L.pcr, ((size_t)(2 * t) * nz + k) * ncolp + colp);
        const R ga = P::ld(L.pcr, ((size_t)(2 * t + 1) * nz + k) * ncolp + colp);
        d = P::sub(P::sub(d, P::mul(al, dm)), P::mul(ga, dp));
        __syncthreads();
    }
    return P::mul(d, P::ld(L.pcr, ((size_t)(2 * L.pcr_steps) * nz + k) * ncolp + colp));
}

// (A u) at cell (i, j, k) of column col, read from global memory
template <class P>
__device__ __forceinline__ typename P::R apply_cell(const Lv<P>& L, const typename P::S* __restrict__ u, int i,
                                                    int j, int k, typename P::R vv, typename P::R& uc) {
    typedef typename P::R R;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const size_t pl = (size_t)nx * ny, b = (size_t)k * pl;
    const size_t c = (size_t)j * nx + i;
    uc = P::ld(u, b + c);
    const R hx = P::add(P::ld(u, b + (size_t)j * nx + cwrap(i - 1, nx)), P::ld(u, b + (size_t)j * nx + cwrap(i + 1, nx)));
    const R hy = P::add(P::ld(u, b + (size_t)cwrap(j - 1, ny) * nx + i), P::ld(u, b + (size_t)cwrap(j + 1, ny) * nx + i));
    const R um = k > 0 ? P::ld(u, b - pl + c) : P::zero();
    const R up = k + 1 < nz ? P::ld(u, b + pl + c) : P::zero();
    R diag = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    if (k > 0) diag = P::add(diag, vv);
    if (k + 1 < nz) diag = P::add(diag, vv);
    R au = P::mul(diag, uc);
    au = P::sub(au, P::mul(P::cst(L.cx), hx));
    au = P::sub(au, P::mul(P::cst(L.cy), hy));
    au = P::sub(au, P::mul(vv, P::add(um, up)));
    return au;
}

// fixed-order block sum of a double (blocks of whole warps, <= 1024 threads)
__device__ __forceinline__ double block_sum_any(double x) {
    __shared__ double ws[32];
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((tid & 31) == 0) ws[tid >> 5] = x;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nt + 31) / 32; ++w) s += ws[w];
    return s;
}

// ---------------------------------------------------------------- Smooth and line solve
// MODE 0: uo = u + rho M^{-1}(f - A u) (+ partial sums of ||f - A u||^2); MODE 1: uo = rho M^{-1} u
template <class P, int MODE>
__global__ void __launch_bounds__(256) k_sweep_pcr(Lv<P> L, double rho_d, const typename P::S* __restrict__ u,
                                                   const typename P::S* __restrict__ f, typename P::S* __restrict__ uo,
                                                   double* partials, const int* done) {
    typedef typename P::R R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    typename P::S* buf = reinterpret_cast<typename P::S*>(smem_raw);
    const int ncol = L.nx * L.ny, k = threadIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = col < ncol;
    const int i = act ? col % L.nx : 0, j = act ? col / L.nx : 0;
    const size_t id = (size_t)k * ncol + col;
    R d = P::zero(), uc = P::zero();
    typename P::Acc acc = 0, cmp = 0;
    if (act) {
        if (MODE == 0) {
            const R vv = P::ld(L.v, col);
            d = P::sub(P::ld(f, id), apply_cell<P>(L, u, i, j, k, vv, uc));
            P::acc_dot(acc, cmp, d, d);
        } else {
            d = P::ld(u, id);
        }
    }
    const R x = pcr_solve<P>(L, d, buf, col, act);
    if (act) {
        const R rho = P::cst(rho_d);
        P::st(uo, id, MODE == 0 ? P::add(uc, P::mul(rho, x)) : (rho_d == 1.0 ? x : P::mul(rho, x)));
    }
    if (MODE == 0 && partials) {
        // fixed-order tree in shared memory (the block need not be a whole number of warps)
        __shared__ double red[256];
        const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
        red[tid] = P::acc_get(acc, cmp);
        for (int h = 128; h > 0; h >>= 1) {
            __syncthreads();
            if (tid < h && tid + h < nt) red[tid] += red[tid + h];
        }
        if (tid == 0) partials[blockIdx.x] = red[0];
    }
}

// ---------------------------------------------------------------- RestrictSmooth
// coarse cell: f_c = 1/4 (sum of the 2x2 fine children of r_f), u_c = rho M_c^{-1} f_c
template <class PF, class P>
__global__ void __launch_bounds__(256) k_restrict_smooth_pcr(Lv<P> Lc, double rho_d,
                                                             const typename PF::S* __restrict__ rf,
                                                             typename P::S* __restrict__ fc,
                                                             typename P::S* __restrict__ uc, const int* done) {
    typedef typename P::R R;
    typedef Conv<PF, P> CV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    typename P::S* buf = reinterpret_cast<typename P::S*>(smem_raw);
    const int ncol = Lc.nx * Lc.ny, k = threadIdx.y, nxf = 2 * Lc.nx;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = col < ncol;
    const size_t id = (size_t)k * ncol + col;
    R fk = P::zero();
    if (act) {
        const int I = col % Lc.nx, J = col / Lc.nx;
        const size_t bf = (size_t)k * 4 * ncol;
        const size_t f00 = bf + (size_t)(2 * J) * nxf + 2 * I, f01 = f00 + nxf;
        const R s = P::add(P::add(CV::f(PF::ld(rf, f00)), CV::f(PF::ld(rf, f00 + 1))),
                           P::add(CV::f(PF::ld(rf, f01)), CV::f(PF::ld(rf, f01 + 1))));
        fk = P::mul(P::cst(0.25), s);
        P::st(fc, id, fk);
    }
    const R x = pcr_solve<P>(Lc, fk, buf, col, act);
    if (act) P::st(uc, id, P::mul(P::cst(rho_d), x));
}

// ---------------------------------------------------------------- Residual (pointwise)
template <class P, class PO>
__global__ void __launch_bounds__(256) k_residual_cell(Lv<P> L, const typename P::S* __restrict__ u,
                                                       const typename P::S* __restrict__ f,
                                                       typename PO::S* __restrict__ r, double* partials,
                                                       const int* done) {
    typedef typename P::R R;
    if (done && *(volatile const int*)done) return;
    const int ncol = L.nx * L.ny;
    const size_t n = (size_t)ncol * L.nz;
    typename P::Acc acc = 0, cmp = 0;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int col = (int)(id % ncol), k = (int)(id / ncol);
        R uc;
        const R rk = P::sub(P::ld(f, id), apply_cell<P>(L, u, col % L.nx, col / L.nx, k, P::ld(L.v, col), uc));
        P::acc_dot(acc, cmp, rk, rk);
        if (PO::id == P::id)
            P::st(reinterpret_cast<typename P::S*>(r), id, rk);
        else
            PO::st(r, id, PO::from_f(P::to_f(rk)));
    }
    if (partials) {
        const double sm = block_sum_any(P::acc_get(acc, cmp));
        if (threadIdx.x == 0) partials[blockIdx.x] = sm;
    }
}

// ---------------------------------------------------------------- Prolongate (pointwise)
// u_f += P u_c at fine cell (i, j, k): cell-centred bilinear weights 9/16, 3/16, 3/16, 1/16
template <class P, class PF>
__global__ void __launch_bounds__(256) k_prolongate_cell(int nxc, int nyc, int nz, const typename P::S* __restrict__ uc,
                                                         typename PF::S* __restrict__ uf, const int* done) {
    typedef typename P::R R;
    if (done && *(volatile const int*)done) return;
    const int nxf = 2 * nxc, nyf = 2 * nyc;
    const size_t plf = (size_t)nxf * nyf, plc = (size_t)nxc * nyc, n = plf * nz;
    const R w9 = P::cst(0.5625), w3 = P::cst(0.1875), w1 = P::cst(0.0625);
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(id % nxf), j = (int)((id / nxf) % nyf), k = (int)(id / plf);
        const int I = i >> 1, J = j >> 1;
        const int I2 = cwrap((i & 1) ? I + 1 : I - 1, nxc), J2 = cwrap((j & 1) ? J + 1 : J - 1, nyc);
        const size_t bc = (size_t)k * plc;
        R val = P::mul(w9, P::ld(uc, bc + (size_t)J * nxc + I));
        val = P::add(val, P::mul(w3, P::ld(uc, bc + (size_t)J * nxc + I2)));
        val = P::add(val, P::mul(w3, P::ld(uc, bc + (size_t)J2 * nxc + I)));
        val = P::add(val, P::mul(w1, P::ld(uc, bc + (size_t)J2 * nxc + I2)));
        PF::st(uf, id, PF::add(PF::ld_plain(uf, id), Conv<P, PF>::f(val)));
    }
}

// ---------------------------------------------------------------- Prolongate, 2 x 2 fine cells per thread
// One thread per (coarse column, plane): the four fine cells (2I+a, 2J+b) of coarse cell (I, J)
// take 9/16 of it, 3/16 of its x and y neighbours on their side and 1/16 of the diagonal one;
// the 3 x 3 coarse neighbourhood is read once for all four (read-only cache), the fine values move
// as 16-byte (8-byte for FP32) pairs. No loop over the planes: every (column, plane) is a thread.
template <class P, class PF>
__global__ void __launch_bounds__(128) k_prolongate_x4(int nxc, int nyc, int nz, const typename P::S* __restrict__ uc,
                                                       typename PF::S* __restrict__ uf, const int* done) {
    typedef typename P::R R;
    typedef typename PF::S SF;
    if (done && *(volatile const int*)done) return;
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    if (I >= nxc || J >= nyc) return;
    const size_t plc = (size_t)nxc * nyc;
    const typename P::S* cp = uc + (size_t)k * plc;
    const int Im = cwrap(I - 1, nxc), Ip = cwrap(I + 1, nxc);
    const size_t rm = (size_t)cwrap(J - 1, nyc) * nxc, r0 = (size_t)J * nxc, rp = (size_t)cwrap(J + 1, nyc) * nxc;
    const R c = P::ld(cp, r0 + I);
    const R xm = P::ld(cp, r0 + Im), xp = P::ld(cp, r0 + Ip);
    const R ym = P::ld(cp, rm + I), yp = P::ld(cp, rp + I);
    const R dmm = P::ld(cp, rm + Im), dpm = P::ld(cp, rm + Ip), dmp = P::ld(cp, rp + Im), dpp = P::ld(cp, rp + Ip);
    const R w9 = P::cst(0.5625), w3 = P::cst(0.1875), w1 = P::cst(0.0625);
    const R c9 = P::mul(w9, c);
    // fine (a, b): a = 0 takes the x neighbour I-1, a = 1 takes I+1; likewise b in y
    const R v00 = P::add(P::add(c9, P::mul(w3, xm)), P::add(P::mul(w3, ym), P::mul(w1, dmm)));
    const R v10 = P::add(P::add(c9, P::mul(w3, xp)), P::add(P::mul(w3, ym), P::mul(w1, dpm)));
    const R v01 = P::add(P::add(c9, P::mul(w3, xm)), P::add(P::mul(w3, yp), P::mul(w1, dmp)));
    const R v11 = P::add(P::add(c9, P::mul(w3, xp)), P::add(P::mul(w3, yp), P::mul(w1, dpp)));
    const int nxf = 2 * nxc;
    const size_t f0 = (size_t)k * 4 * plc + (size_t)(2 * J) * nxf + 2 * I, f1 = f0 + nxf;
    PF::st(uf, f0, PF::add(PF::ld_plain(uf, f0), Conv<P, PF>::f(v00)));
    PF::st(uf, f0 + 1, PF::add(PF::ld_plain(uf, f0 + 1), Conv<P, PF>::f(v10)));
    PF::st(uf, f1, PF::add(PF::ld_plain(uf, f1), Conv<P, PF>::f(v01)));
    PF::st(uf, f1 + 1, PF::add(PF::ld_plain(uf, f1 + 1), Conv<P, PF>::f(v11)));
}

// ---------------------------------------------------------------- launchers
// columns per block: the block is cpb x nz threads (nz <= 256), at most 256 threads
static int pcr_cpb(int nz, int ncol) {
    int c = 256 / nz;
    if (c < 1) c = 1;
    if (c > ncol) c = ncol;
    return c;
}

template <class P>
static bool pcr_ok(const Lv<P>& L) {
    return L.pcr && (size_t)L.nx * L.ny <= (size_t)PCR_MAX_COLS && L.nz <= 256;
}

template <class P>
int pcr_blocks(const Lv<P>& L) {
    const int ncol = L.nx * L.ny;
    const int cpb = pcr_cpb(L.nz, ncol);
    return (ncol + cpb - 1) / cpb;
}

template <class P, int MODE>
static int run_sweep_pcr(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                         typename P::S* uo, double* partials, const int* done, cudaStream_t s) {
    const int ncol = L.nx * L.ny;
    const int cpb = pcr_cpb(L.nz, ncol);
    const int nb = (ncol + cpb - 1) / cpb;
    const size_t smem = (size_t)cpb * L.nz * sizeof(typename P::S);
    k_sweep_pcr<P, MODE><<<nb, dim3(cpb, L.nz), smem, s>>>(L, rho, u, f, uo, partials, done);
    note_launch();
    return nb;
}

template <class P>
int launch_smooth_pcr(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f, typename P::S* uo,
                      double* partials, const int* done, cudaStream_t s) {
    if (!pcr_ok(L)) return -1;
    return run_sweep_pcr<P, 0>(L, rho, u, f, uo, partials, done, s);
}

template <class P>
int launch_line_solve_pcr(const Lv<P>& L, const typename P::S* b, typename P::S* x, double scale, const int* done,
                          cudaStream_t s) {
    if (!pcr_ok(L)) return -1;
    return run_sweep_pcr<P, 1>(L, scale, b, nullptr, x, nullptr, done, s);
}

template <class PF, class P>
int launch_restrict_smooth_pcr(const Lv<P>& Lc, double rho, const typename PF::S* rf, typename P::S* fc,
                               typename P::S* uc, const int* done, cudaStream_t s) {
    if (!pcr_ok(Lc)) return -1;
    const int ncol = Lc.nx * Lc.ny;
    const int cpb = pcr_cpb(Lc.nz, ncol);
    const int nb = (ncol + cpb - 1) / cpb;
    const size_t smem = (size_t)cpb * Lc.nz * sizeof(typename P::S);
    k_restrict_smooth_pcr<PF, P><<<nb, dim3(cpb, Lc.nz), smem, s>>>(Lc, rho, rf, fc, uc, done);
    note_launch();
    return nb;
}

// pointwise kernels: used on levels with at most PCR_MAX_COLS columns; fixed block count
int cell_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 1024) b = 1024;
    return (int)(b ? b : 1);
}

template <class P, class PO>
int launch_residual_cell(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r,
                         double* partials, const int* done, cudaStream_t s) {
    if ((size_t)L.nx * L.ny > (size_t)PCR_MAX_COLS) return -1;
    const int nb = cell_blocks((size_t)L.nx * L.ny * L.nz);
    k_residual_cell<P, PO><<<nb, 256, 0, s>>>(L, u, f, r, partials, done);
    note_launch();
    return nb;
}

template <class P, class PF>
int launch_prolongate_cell(int nxc, int nyc, int nz, const typename P::S* uc, typename PF::S* uf, const int* done,
                           cudaStream_t s) {
    if ((size_t)nxc * nyc > (size_t)PCR_MAX_COLS / 4) return -1;  // fine level at most PCR_MAX_COLS columns
    const int nb = cell_blocks((size_t)4 * nxc * nyc * nz);
    k_prolongate_cell<P, PF><<<nb, 256, 0, s>>>(nxc, nyc, nz, uc, uf, done);
    note_launch();
    return nb;
}

template <class P, class PF>
int launch_prolongate_x4(int nxc, int nyc, int nz, const typename P::S* uc, typename PF::S* uf, const int* done,
                         cudaStream_t s) {
    dim3 blk(32, 4), grd((nxc + 31) / 32, (nyc + 3) / 4, nz);
    k_prolongate_x4<P, PF><<<grd, blk, 0, s>>>(nxc, nyc, nz, uc, uf, done);
    note_launch();
    return (int)(grd.x * grd.y * grd.z);
}

#define TPMG_COARSE_INST(P)                                                                                 \
    template size_t pcr_factor_count<P>(const Lv<P>&, int);                                                  \
    template void launch_pcr_factors<P>(const Lv<P>&, P::S*, int, cudaStream_t);                             \
    template int pcr_blocks<P>(const Lv<P>&);                                                                \
    template int launch_smooth_pcr<P>(const Lv<P>&, double, const P::S*, const P::S*, P::S*, double*,        \
                                      const int*, cudaStream_t);                                             \
    template int launch_line_solve_pcr<P>(const Lv<P>&, const P::S*, P::S*, double, const int*, cudaStream_t); \
    template int launch_restrict_smooth_pcr<P, P>(const Lv<P>&, double, const P::S*, P::S*, P::S*, const int*, \
                                                  cudaStream_t);                                             \
    template int launch_residual_cell<P, P>(const Lv<P>&, const P::S*, const P::S*, P::S*, double*, const int*, \
                                            cudaStream_t);                                                   \
    template int launch_prolongate_cell<P, P>(int, int, int, const P::S*, P::S*, const int*, cudaStream_t);     \
    template int launch_prolongate_x4<P, P>(int, int, int, const P::S*, P::S*, const int*, cudaStream_t);

TPMG_COARSE_INST(PolF64)
TPMG_COARSE_INST(PolF32)
TPMG_COARSE_INST(PolDW)
TPMG_COARSE_INST(PolF32B)
template int launch_restrict_smooth_pcr<PolF32, PolF32B>(const Lv<PolF32B>&, double, const float*, float*, float*,
                                                         const int*, cudaStream_t);
template int launch_prolongate_cell<PolF32B, PolF32>(int, int, int, const float*, float*, const int*, cudaStream_t);
template int launch_prolongate_x4<PolF32B, PolF32>(int, int, int, const float*, float*, const int*, cudaStream_t);
template int launch_restrict_smooth_pcr<PolDW, PolF64>(const Lv<PolF64>&, double, const float2*, double*, double*,
                                                       const int*, cudaStream_t);
template int launch_prolongate_cell<PolF64, PolDW>(int, int, int, const double*, float2*, const int*, cudaStream_t);
template int launch_prolongate_x4<PolF64, PolDW>(int, int, int, const double*, float2*, const int*, cudaStream_t);
template int launch_residual_cell<PolDW, PolF32>(const Lv<PolDW>&, const float2*, const float2*, float*, double*,
                                                 const int*, cudaStream_t);
template int launch_residual_cell<PolF64, PolF32>(const Lv<PolF64>&, const double*, const double*, float*, double*,
                                                  const int*, cudaStream_t);

}  // namespace tpmg
