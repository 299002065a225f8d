// k_mg.cu -- matrix-free operator, vertical line solves and the multigrid kernels.
//
// Every kernel maps one thread to one vertical column (Sec. 3.1: the vertical dependency of the
// tridiagonal solve is kept inside a thread) and 32 consecutive x columns to a warp, so every
// global access of a warp at fixed (j, k) is one contiguous row segment. The vertical neighbours
// live in a three-value register window; the horizontal neighbours are read through the read-only
// cache (the same rows are read by the neighbouring warps of the block and stay in L1/L2).
//
// The Thomas algorithm keeps its forward-eliminated right-hand side d'_k and w_k = v/m_k in a
// per-thread stack in shared memory, so the smoother reads u and f once and writes u' once
// (the paper splits Smooth into two kernels to avoid a race on u, Sec. 3.1; here the output goes
// to a separate buffer and the back substitution happens in the same kernel).
//
// Operator (Sec. 2.1.1, flat-box form of Eq. (6), periodic horizontally, Neumann at k = 0 and
// k = nz-1): (A u)_k = D_k u_k - cx (u_W + u_E) - cy (u_S + u_N) - v (u_{k-1} + u_{k+1}) with
// D_k = 1 + 2cx + 2cy + v * (number of vertical neighbours).
#include "kernels.cuh"

namespace tpmg {

static constexpr int TX = 32;

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Column geometry of one thread.
struct Col {
    int i, j;
    bool act;
    size_t c, w, e, s, n;  // in-plane offsets of the column and its 4 horizontal neighbours
};
__device__ __forceinline__ Col make_col(int nx, int ny) {
    Col q;
    q.i = blockIdx.x * blockDim.x + threadIdx.x;
    q.j = blockIdx.y * blockDim.y + threadIdx.y;
    q.act = q.i < nx && q.j < ny;
    if (q.act) {
        q.c = (size_t)q.j * nx + q.i;
        q.w = (size_t)q.j * nx + wrapi(q.i - 1, nx);
        q.e = (size_t)q.j * nx + wrapi(q.i + 1, nx);
        q.s = (size_t)wrapi(q.j - 1, ny) * nx + q.i;
        q.n = (size_t)wrapi(q.j + 1, ny) * nx + q.i;
    }
    return q;
}

// (A u)_k from the register window (um = u_{k-1} or 0, up = u_{k+1} or 0).
template <class P>
__device__ __forceinline__ typename P::R stencil(typename P::R diag, typename P::R uc,
                                                 typename P::R um, typename P::R up,
                                                 typename P::R hsum_x, typename P::R hsum_y,
                                                 typename P::R cx, typename P::R cy,
                                                 typename P::R vv) {
    typename P::R au = P::mul(diag, uc);
    au = P::sub(au, P::mul(cx, hsum_x));
    au = P::sub(au, P::mul(cy, hsum_y));
    au = P::sub(au, P::mul(vv, P::add(um, up)));
    return au;
}

// Diagonal of row k of the column block.
template <class P>
__device__ __forceinline__ typename P::R diag_k(int k, int nz, typename P::R dh, typename P::R dh1,
                                                typename P::R dh2) {
    if (nz == 1) return dh;
    return (k == 0 || k == nz - 1) ? dh1 : dh2;
}

// ---------------------------------------------------------------- y = A x
template <class P>
__global__ void __launch_bounds__(256) k_apply_A(Lv<P> L, const typename P::S* __restrict__ x,
                                                 typename P::S* __restrict__ y) {
    typedef typename P::R R;
    Col q = make_col(L.nx, L.ny);
    if (!q.act) return;
    const size_t pl = (size_t)L.nx * L.ny;
    const R cx = P::cst(L.cx), cy = P::cst(L.cy), vv = P::ld(L.v, q.c);
    const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
    R um = P::zero(), uc = P::ld(x, q.c);
    for (int k = 0; k < L.nz; ++k) {
        const size_t b = (size_t)k * pl;
        R up = (k + 1 < L.nz) ? P::ld(x, b + pl + q.c) : P::zero();
        R hx = P::add(P::ld(x, b + q.w), P::ld(x, b + q.e));
        R hy = P::add(P::ld(x, b + q.s), P::ld(x, b + q.n));
        R au = stencil<P>(diag_k<P>(k, L.nz, dh, dh1, dh2), uc, um, up, hx, hy, cx, cy, vv);
        P::st(y, b + q.c, au);
        um = uc;
        uc = up;
    }
}

// ---------------------------------------------------------------- Thomas helpers
// Forward elimination step k for the symmetric tridiagonal column block with off-diagonals -v:
// m_k = D_k - v^2 / m_{k-1}, d'_k = (rhs_k + v d'_{k-1}) / m_k, w_k = v / m_k. The pair
// (d'_k, w_k) goes to the thread's stack; the back substitution is x_k = d'_k + w_k x_{k+1}.
template <class P>
struct Thomas {
    typedef typename P::R R;
    R vv, vv2, inv_prev, d_prev;
    R* dp;
    R* w;
    int nt, tid;
    __device__ __forceinline__ void init(R v, R* stack, int nz) {
        vv = v;
        vv2 = P::mul(v, v);
        inv_prev = P::zero();
        d_prev = P::zero();
        nt = blockDim.x * blockDim.y;
        tid = threadIdx.y * blockDim.x + threadIdx.x;
        dp = stack;
        w = stack + (size_t)nz * nt;
    }
    __device__ __forceinline__ void forward(int k, R diag, R rhs) {
        R m = (k == 0) ? diag : P::sub(diag, P::mul(vv2, inv_prev));
        R inv = P::rcp(m);
        R d = P::mul(P::add(rhs, P::mul(vv, d_prev)), inv);
        dp[(size_t)k * nt + tid] = d;
        w[(size_t)k * nt + tid] = P::mul(vv, inv);
        inv_prev = inv;
        d_prev = d;
    }
    // x_k given x_{k+1}
    __device__ __forceinline__ R back(int k, R x_next) const {
        return P::add(dp[(size_t)k * nt + tid], P::mul(w[(size_t)k * nt + tid], x_next));
    }
};

// ---------------------------------------------------------------- x = M^{-1} b
template <class P>
__global__ void __launch_bounds__(256) k_line_solve(Lv<P> L, const typename P::S* __restrict__ b,
                                                    typename P::S* __restrict__ x, double scale_d,
                                                    const int* done) {
    typedef typename P::R R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    Col q = make_col(L.nx, L.ny);
    if (!q.act) return;
    const size_t pl = (size_t)L.nx * L.ny;
    const R vv = P::ld(L.v, q.c);
    const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
    const R scale = P::cst(scale_d);
    const bool scaled = scale_d != 1.0;
    Thomas<P> th;
    th.init(vv, reinterpret_cast<R*>(smem_raw), L.nz);
    for (int k = 0; k < L.nz; ++k)
        th.forward(k, diag_k<P>(k, L.nz, dh, dh1, dh2), P::ld(b, (size_t)k * pl + q.c));
    R xn = P::zero();
    for (int k = L.nz - 1; k >= 0; --k) {
        xn = th.back(k, xn);
        P::st(x, (size_t)k * pl + q.c, scaled ? P::mul(scale, xn) : xn);
    }
}

// ---------------------------------------------------------------- Smooth (Eq. 11)
// uo = u + rho M^{-1}(f - A u); optional block partial sums of ||f - A u||^2 (the residual of the
// incoming iterate, which the solver uses as the convergence test of the previous cycle).
template <class P>
__global__ void __launch_bounds__(256) k_smooth(Lv<P> L, double rho_d,
                                                const typename P::S* __restrict__ u,
                                                const typename P::S* __restrict__ f,
                                                typename P::S* __restrict__ uo, double* partials,
                                                const int* done) {
    typedef typename P::R R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    Col q = make_col(L.nx, L.ny);
    typename P::Acc acc = 0, cmp = 0;
    if (q.act) {
        const size_t pl = (size_t)L.nx * L.ny;
        const R cx = P::cst(L.cx), cy = P::cst(L.cy), vv = P::ld(L.v, q.c);
        const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
        const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        const R rho = P::cst(rho_d);
        Thomas<P> th;
        th.init(vv, reinterpret_cast<R*>(smem_raw), L.nz);
        R um = P::zero(), uc = P::ld(u, q.c);
        for (int k = 0; k < L.nz; ++k) {
            const size_t b = (size_t)k * pl;
            R up = (k + 1 < L.nz) ? P::ld(u, b + pl + q.c) : P::zero();
            R hx = P::add(P::ld(u, b + q.w), P::ld(u, b + q.e));
            R hy = P::add(P::ld(u, b + q.s), P::ld(u, b + q.n));
            R diag = diag_k<P>(k, L.nz, dh, dh1, dh2);
            R r = P::sub(P::ld(f, b + q.c), stencil<P>(diag, uc, um, up, hx, hy, cx, cy, vv));
            P::acc_dot(acc, cmp, r, r);
            th.forward(k, diag, r);
            um = uc;
            uc = up;
        }
        R xn = P::zero();
        for (int k = L.nz - 1; k >= 0; --k) {
            const size_t id = (size_t)k * pl + q.c;
            xn = th.back(k, xn);
            P::st(uo, id, P::add(P::ld(u, id), P::mul(rho, xn)));
        }
    }
    if (partials) {
        double s = block_sum(P::acc_get(acc, cmp));
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------- Residual
template <class P, class PO>
__global__ void __launch_bounds__(256) k_residual(Lv<P> L, const typename P::S* __restrict__ u,
                                                  const typename P::S* __restrict__ f,
                                                  typename PO::S* __restrict__ r, double* partials,
                                                  const int* done) {
    typedef typename P::R R;
    if (done && *(volatile const int*)done) return;
    Col q = make_col(L.nx, L.ny);
    typename P::Acc acc = 0, cmp = 0;
    if (q.act) {
        const size_t pl = (size_t)L.nx * L.ny;
        const R cx = P::cst(L.cx), cy = P::cst(L.cy), vv = P::ld(L.v, q.c);
        const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
        const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        R um = P::zero(), uc = P::ld(u, q.c);
        for (int k = 0; k < L.nz; ++k) {
            const size_t b = (size_t)k * pl;
            R up = (k + 1 < L.nz) ? P::ld(u, b + pl + q.c) : P::zero();
            R hx = P::add(P::ld(u, b + q.w), P::ld(u, b + q.e));
            R hy = P::add(P::ld(u, b + q.s), P::ld(u, b + q.n));
            R rk = P::sub(P::ld(f, b + q.c),
                          stencil<P>(diag_k<P>(k, L.nz, dh, dh1, dh2), uc, um, up, hx, hy, cx, cy, vv));
            P::acc_dot(acc, cmp, rk, rk);
            if (PO::id == P::id)
                P::st(reinterpret_cast<typename P::S*>(r), b + q.c, rk);
            else
                PO::st(r, b + q.c, PO::from_f(P::to_f(rk)));
            um = uc;
            uc = up;
        }
    }
    if (partials) {
        double s = block_sum(P::acc_get(acc, cmp));
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}


// ---------------------------------------------------------------- RestrictSmooth
// Coarse column (I, J): f_c = 1/4 (sum of the 2x2 fine children of r_f), then the first smoothing
// step from a zero guess, u_c = rho M_c^{-1} f_c (Algorithm 1; Sec. 3.1 kernel list). The fine
// level may be stored in another precision (PF) than the coarse one (P).
template <class PF, class P>
__global__ void __launch_bounds__(256) k_restrict_smooth(Lv<P> Lc, double rho_d,
                                                         const typename PF::S* __restrict__ rf,
                                                         typename P::S* __restrict__ fc,
                                                         typename P::S* __restrict__ uc,
                                                         const int* done) {
    typedef typename P::R R;
    typedef Conv<PF, P> CV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    Col q = make_col(Lc.nx, Lc.ny);
    if (!q.act) return;
    const int nxf = 2 * Lc.nx;
    const size_t plc = (size_t)Lc.nx * Lc.ny, plf = 4 * plc;
    const size_t f00 = (size_t)(2 * q.j) * nxf + 2 * q.i, f01 = f00 + nxf;
    const R vv = P::ld(Lc.v, q.c);
    const R dh = P::cst(1.0 + 2.0 * Lc.cx + 2.0 * Lc.cy);
    const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
    const R rho = P::cst(rho_d), quarter = P::cst(0.25);
    Thomas<P> th;
    th.init(vv, reinterpret_cast<R*>(smem_raw), Lc.nz);
    for (int k = 0; k < Lc.nz; ++k) {
        const size_t bf = (size_t)k * plf;
        R s = P::add(P::add(CV::f(PF::ld(rf, bf + f00)), CV::f(PF::ld(rf, bf + f00 + 1))),
                     P::add(CV::f(PF::ld(rf, bf + f01)), CV::f(PF::ld(rf, bf + f01 + 1))));
        R fk = P::mul(quarter, s);
        P::st(fc, (size_t)k * plc + q.c, fk);
        th.forward(k, diag_k<P>(k, Lc.nz, dh, dh1, dh2), fk);
    }
    R xn = P::zero();
    for (int k = Lc.nz - 1; k >= 0; --k) {
        xn = th.back(k, xn);
        P::st(uc, (size_t)k * plc + q.c, P::mul(rho, xn));
    }
}

// ---------------------------------------------------------------- Prolongate
// u_f += P u_c: cell-centred bilinear interpolation, weights 9/16, 3/16, 3/16, 1/16; the fine
// cell 2I+a takes its second x neighbour from coarse I-1 (a = 0) or I+1 (a = 1); periodic.
// The interpolated value is formed in the coarse precision P and added in the fine one PF.
template <class P, class PF>
__global__ void __launch_bounds__(256) k_prolongate(int nxc, int nyc, int nz,
                                                    const typename P::S* __restrict__ uc,
                                                    typename PF::S* __restrict__ uf,
                                                    const int* done) {
    typedef typename P::R R;
    if (done && *(volatile const int*)done) return;
    const int nxf = 2 * nxc, nyf = 2 * nyc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nxf || j >= nyf) return;
    const int I = i >> 1, J = j >> 1;
    const int I2 = wrapi((i & 1) ? I + 1 : I - 1, nxc), J2 = wrapi((j & 1) ? J + 1 : J - 1, nyc);
    const size_t plc = (size_t)nxc * nyc, plf = (size_t)nxf * nyf;
    const size_t a = (size_t)J * nxc + I, bq = (size_t)J * nxc + I2, c = (size_t)J2 * nxc + I,
                 d = (size_t)J2 * nxc + I2, o = (size_t)j * nxf + i;
    const R w9 = P::cst(0.5625), w3 = P::cst(0.1875), w1 = P::cst(0.0625);
    for (int k = 0; k < nz; ++k) {
        const size_t bc = (size_t)k * plc;
        R val = P::mul(w9, P::ld(uc, bc + a));
        val = P::add(val, P::mul(w3, P::ld(uc, bc + bq)));
        val = P::add(val, P::mul(w3, P::ld(uc, bc + c)));
        val = P::add(val, P::mul(w1, P::ld(uc, bc + d)));
        const size_t id = (size_t)k * plf + o;
        PF::st(uf, id, PF::add(PF::ld_plain(uf, id), Conv<P, PF>::f(val)));
    }
}

// ---------------------------------------------------------------- u += e (FP32 correction)
template <class P>
__global__ void k_correct(size_t n, typename P::S* __restrict__ u, const float* __restrict__ e,
                          const int* done) {
    if (done && *(volatile const int*)done) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x)
        P::st(u, t, P::add(P::ld_plain(u, t), P::from_f(__ldg(e + t))));
}

// ---------------------------------------------------------------- launch shapes
static int g_smem_optin = -1;

Shape sweep_shape(int nx, int ny, int nz, int bytes_per_value, bool stack) {
    Shape sh;
    int ty = 4;
    size_t per_thread = stack ? (size_t)2 * nz * bytes_per_value : 0;
    if (stack) {
        // aim for about 72 KB of stack per block so three blocks fit on an SM
        size_t budget = 72 * 1024;
        ty = (int)(budget / (per_thread * TX));
        if (ty < 1) ty = 1;
        if (ty > 8) ty = 8;
    }
    int gx = (nx + TX - 1) / TX;
    // narrow levels: do not leave most of a block idle
    if (ny < ty) ty = ny < 1 ? 1 : ny;
    sh.block = dim3(TX, ty, 1);
    sh.grid = dim3(gx, (ny + ty - 1) / ty, 1);
    sh.smem = per_thread * TX * ty;
    return sh;
}

int max_partials(int nx, int ny) {
    const int col_kernels = ((nx + TX - 1) / TX) * ny;
    const int cell_kernels = nx * ny <= PCR_MAX_COLS ? nx * ny : 0;  // at most one block per column
    return col_kernels > cell_kernels ? col_kernels : cell_kernels;
}

template <class K>
static void allow_smem(K kernel, size_t bytes) {
    if (bytes > 32 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class P>
void launch_apply_A(const Lv<P>& L, const typename P::S* x, typename P::S* y, cudaStream_t s) {
    if (launch_apply_A_x2<P>(L, x, y, s) >= 0) return;
    Shape sh = sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), false);
    k_apply_A<P><<<sh.grid, sh.block, 0, s>>>(L, x, y);
    note_launch();
}
template <class P>
void launch_line_solve(const Lv<P>& L, const typename P::S* b, typename P::S* x, double scale, const int* done,
                       cudaStream_t s) {
    if (launch_line_solve_pcr<P>(L, b, x, scale, done, s) >= 0) return;
    if (launch_line_solve_pp<P>(L, b, x, scale, done, s) >= 0) return;
    Shape sh = sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), true);
    allow_smem(k_line_solve<P>, sh.smem);
    k_line_solve<P><<<sh.grid, sh.block, sh.smem, s>>>(L, b, x, scale, done);
    note_launch();
}
template <class P>
int launch_smooth(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                   typename P::S* uo, double* partials, const int* done, cudaStream_t s) {
    int nparts = launch_smooth_pcr<P>(L, rho, u, f, uo, partials, done, s);
    if (nparts >= 0) return nparts;
    nparts = launch_smooth_pp<P>(L, rho, u, f, uo, partials, done, s);
    if (nparts >= 0) return nparts;
    Shape sh = sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), true);
    allow_smem(k_smooth<P>, sh.smem);
    k_smooth<P><<<sh.grid, sh.block, sh.smem, s>>>(L, rho, u, f, uo, partials, done);
    note_launch();
    return sh.nblocks();
}
template <class P, class PO>
int residual_launch_blocks(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r) {
    // launch_residual's three choices in its order: pointwise, plane-pipelined, one thread per column
    if ((size_t)L.nx * L.ny <= (size_t)PCR_MAX_COLS) return cell_blocks((size_t)L.nx * L.ny * L.nz);
    const int nb = residual_pp_blocks<P, PO>(L, u, f, r);
    if (nb >= 0) return nb;
    return sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), false).nblocks();
}
template <class P, class PO>
int launch_residual(const Lv<P>& L, const typename P::S* u, const typename P::S* f,
                    typename PO::S* r, double* partials, const int* done, cudaStream_t s) {
    int nb = launch_residual_cell<P, PO>(L, u, f, r, partials, done, s);
    if (nb >= 0) return nb;
    nb = launch_residual_pp<P, PO>(L, u, f, r, partials, done, s);
    if (nb >= 0) return nb;
    Shape sh = sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), false);
    k_residual<P, PO><<<sh.grid, sh.block, 0, s>>>(L, u, f, r, partials, done);
    note_launch();
    return sh.nblocks();
}
template <class PF, class P>
void launch_restrict_smooth(const Lv<P>& Lc, double rho, const typename PF::S* rf,
                            typename P::S* fc, typename P::S* uc, const int* done, cudaStream_t s) {
    if (launch_restrict_smooth_pcr<PF, P>(Lc, rho, rf, fc, uc, done, s) >= 0) return;
    // the pipelined kernel copies pairs of fine values: their address must be pair-aligned
    if (((uintptr_t)rf % (2 * sizeof(typename PF::S))) == 0 &&
        launch_restrict_smooth_pp<PF, P>(Lc, rho, rf, fc, uc, done, s) >= 0)
        return;
    Shape sh = sweep_shape(Lc.nx, Lc.ny, Lc.nz, sizeof(typename P::R), true);
    allow_smem(k_restrict_smooth<PF, P>, sh.smem);
    k_restrict_smooth<PF, P><<<sh.grid, sh.block, sh.smem, s>>>(Lc, rho, rf, fc, uc, done);
    note_launch();
}
template <class P, class PF>
void launch_prolongate(int nxc, int nyc, int nz, const typename P::S* uc, typename PF::S* uf,
                       const int* done, cudaStream_t s) {
    if (launch_prolongate_cell<P, PF>(nxc, nyc, nz, uc, uf, done, s) >= 0) return;
    if (launch_prolongate_x4<P, PF>(nxc, nyc, nz, uc, uf, done, s) >= 0) return;
    Shape sh = sweep_shape(2 * nxc, 2 * nyc, nz, sizeof(typename P::R), false);
    k_prolongate<P, PF><<<sh.grid, sh.block, 0, s>>>(nxc, nyc, nz, uc, uf, done);
    note_launch();
}
template <class P>
void launch_correct(size_t n, typename P::S* u, const float* e, const int* done, cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_correct<P><<<(unsigned)blocks, 256, 0, s>>>(n, u, e, done);
    note_launch();
}

#define TPMG_INST(P)                                                                              \
    template void launch_apply_A<P>(const Lv<P>&, const P::S*, P::S*, cudaStream_t);              \
    template void launch_line_solve<P>(const Lv<P>&, const P::S*, P::S*, double, const int*, cudaStream_t); \
    template int launch_smooth<P>(const Lv<P>&, double, const P::S*, const P::S*, P::S*, double*, \
                                   const int*, cudaStream_t);                                      \
    template int residual_launch_blocks<P, P>(const Lv<P>&, const P::S*, const P::S*, P::S*);     \
    template int launch_residual<P, P>(const Lv<P>&, const P::S*, const P::S*, P::S*, double*,     \
                                        const int*, cudaStream_t);                                 \
    template void launch_restrict_smooth<P, P>(const Lv<P>&, double, const P::S*, P::S*, P::S*,   \
                                            const int*, cudaStream_t);                             \
    template void launch_prolongate<P, P>(int, int, int, const P::S*, P::S*, const int*, cudaStream_t);

TPMG_INST(PolF64)
TPMG_INST(PolF32)
TPMG_INST(PolDW)
TPMG_INST(PolF32B)
template void launch_restrict_smooth<PolF32, PolF32B>(const Lv<PolF32B>&, double, const float*, float*, float*,
                                                      const int*, cudaStream_t);
template void launch_prolongate<PolF32B, PolF32>(int, int, int, const float*, float*, const int*, cudaStream_t);
template int launch_residual<PolDW, PolF32>(const Lv<PolDW>&, const float2*, const float2*, float*,
                                             double*, const int*, cudaStream_t);
template int launch_residual<PolF64, PolF32>(const Lv<PolF64>&, const double*, const double*,
                                              float*, double*, const int*, cudaStream_t);
template void launch_correct<PolDW>(size_t, float2*, const float*, const int*, cudaStream_t);
template void launch_restrict_smooth<PolDW, PolF64>(const Lv<PolF64>&, double, const float2*, double*, double*,
                                                    const int*, cudaStream_t);
template void launch_prolongate<PolF64, PolDW>(int, int, int, const double*, float2*, const int*, cudaStream_t);
template void launch_correct<PolF64>(size_t, double*, const float*, const int*, cudaStream_t);

}  // namespace tpmg
