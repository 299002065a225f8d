// k_panel.cu -- the paper's own operator: Eq. (1) on one gnomonic cubed-sphere panel with
// homogeneous Dirichlet conditions on the panel boundary, in the factorised form of Eq. (14)
// "LocalMatrixStencil" (Sec. 3.1), native FP64 (the paper's precision):
//
//   (A u)_{T,k} = (|T| E_k - alpha_T) u_{T,k} + sum_{T'} alpha_{TT'} u_{T',k}
//                 - |T| (B_k u_{T,k-1} + C_k u_{T,k+1}),
//   E_k = a_k - b_k - c_k,  B_k = -b_k,  C_k = -c_k  (B_0 = 0, C_{nz-1} = 0: Neumann),
//
// alpha_{TT'} < 0 the two-point flux coefficients of the four faces of T (a face on the panel
// boundary couples to a ghost value of 0 but still counts in alpha_T = their sum), |T| the cell's
// area. Only the coefficient arithmetic differs from the flat box: per column four face
// coefficients and the area instead of cx, cy and v; per level three radial vectors.
//
// Every kernel maps one thread to one vertical column and 32 consecutive x columns to a warp
// (coalesced rows, Sec. 3.1); horizontal neighbours come through the read-only cache. The Thomas
// factors of the column blocks are computed once per level (k_panel_factors): 1/m_k, the forward
// multiplier |T| B_k / m_k and the backward one |T| C_k / m_k, per cell. The forward-eliminated
// values go into the output field itself, which the back substitution then overwrites, so the
// sweeps need no scratch. These kernels are bound by the FP64 pipe (about 14 FP64 instructions per
// cell for a Smooth; at 54 resident warps per SM the pipe, not the load latency, sets the pace).
#include "kernels.cuh"
#include "panel.cuh"

namespace tpmg {

namespace {

template <class T>
struct PCol {
    int i, j;
    bool act, hw, he, hs, hn;  // in range; which horizontal neighbours lie on the panel
    size_t c;
    T area, aw, ae, as, an, at;
};

template <class T>
__device__ __forceinline__ PCol<T> panel_col(const PanelLvT<T>& L) {
    PCol<T> q;
    q.i = blockIdx.x * blockDim.x + threadIdx.x;
    q.j = blockIdx.y * blockDim.y + threadIdx.y;
    q.act = q.i < L.nx && q.j < L.ny;
    if (!q.act) return q;
    q.c = (size_t)q.j * L.nx + q.i;
    q.hw = q.i > 0;
    q.he = q.i < L.nx - 1;
    q.hs = q.j > 0;
    q.hn = q.j < L.ny - 1;
    q.area = __ldg(L.area + q.c);
    q.aw = __ldg(L.ax + (size_t)q.j * (L.nx + 1) + q.i);
    q.ae = __ldg(L.ax + (size_t)q.j * (L.nx + 1) + q.i + 1);
    q.as = __ldg(L.ay + (size_t)q.j * L.nx + q.i);
    q.an = __ldg(L.ay + (size_t)(q.j + 1) * L.nx + q.i);
    q.at = (q.aw + q.ae) + (q.as + q.an);
    return q;
}

// (A u)_{T,k} given the centre value, its vertical neighbours (0 beyond the column) and
// |T| B_k, |T| C_k; the horizontal neighbours of plane k are read here (0 beyond the panel)
template <class T>
__device__ __forceinline__ T panel_Au(const PanelLvT<T>& L, const PCol<T>& q, const T* __restrict__ x, size_t b, int k,
                                     T uc, T um, T up, T tb, T tc) {
    const T xw = q.hw ? __ldg(x + b + q.c - 1) : T(0);
    const T xe = q.he ? __ldg(x + b + q.c + 1) : T(0);
    const T xs = q.hs ? __ldg(x + b + q.c - L.nx) : T(0);
    const T xn = q.hn ? __ldg(x + b + q.c + L.nx) : T(0);
    T s = fma(q.area, __ldg(L.E + k), -q.at) * uc;  // the diagonal
    s = fma(q.aw, xw, s);
    s = fma(q.ae, xe, s);
    s = fma(q.as, xs, s);
    s = fma(q.an, xn, s);
    s = fma(-tb, um, s);
    return fma(-tc, up, s);
}

}  // namespace

// Thomas factors of every column block of level L: m_0 = D_0, m_k = D_k - (|T| B_k)^2 / m_{k-1}
// with D_k = |T| E_k - alpha_T (the off-diagonals of row k are -|T| B_k below, -|T| C_k above, and
// C_{k-1} = B_k); stored 1/m_k, |T| B_k / m_k and |T| C_k / m_k.
__global__ void __launch_bounds__(128) k_panel_factors(PanelLv L, double* __restrict__ inv, double* __restrict__ fl,
                                                       double* __restrict__ fw) {
    const PCol<double> q = panel_col(L);
    if (!q.act) return;
    const size_t pl = (size_t)L.nx * L.ny;
    double m_prev = 1.0;
    for (int k = 0; k < L.nz; ++k) {
        const double d = fma(q.area, L.E[k], -q.at);
        const double tb = q.area * L.B[k];
        const double m = (k == 0) ? d : d - tb * tb / m_prev;
        const double iv = 1.0 / m;
        inv[(size_t)k * pl + q.c] = iv;
        fl[(size_t)k * pl + q.c] = tb * iv;
        fw[(size_t)k * pl + q.c] = q.area * L.C[k] * iv;
        m_prev = m;
    }
}

// MODE 0 Smooth: out = u + coef M^{-1} (f - A u) (Eq. (11)), partial sums of ||f - A u||^2
// MODE 1 Residual: out = f - A u (stored in TO: the FP64 outer residual of the mixed solve is stored
//        in FP32), partial sums of ||f - A u||^2
// MODE 2 line solve: out = coef M^{-1} u (u is the right-hand side)
// MODE 3 apply: out = A u
// T is the arithmetic (double or float); the norm's partial sums are accumulated in T.
template <int MODE, class T, class TO>
__global__ void __launch_bounds__(128) k_panel_sweep(PanelLvT<T> L, T coef, const T* __restrict__ u,
                                                     const T* __restrict__ f, TO* out, double* partials,
                                                     const int* done) {
    if (done && *(volatile const int*)done) return;
    const PCol<T> q = panel_col(L);
    const size_t pl = (size_t)L.nx * L.ny;
    const int nz = L.nz;
    T acc = 0;
    if (q.act) {
        T um = 0, uc = (MODE != 2) ? __ldg(u + q.c) : T(0), dp = 0;
        T tb = 0;  // |T| B_k (B_0 = 0); |T| C_k = |T| B_{k+1} is carried to the next plane
#pragma unroll 2
        for (int k = 0; k < nz; ++k) {
            const size_t b = (size_t)k * pl;
            const T tc = (k + 1 < nz) ? q.area * __ldg(L.B + k + 1) : T(0);
            T r;
            if (MODE != 2) {
                const T up = (k + 1 < nz) ? __ldg(u + b + pl + q.c) : T(0);
                const T au = panel_Au(L, q, u, b, k, uc, um, up, tb, tc);
                r = (MODE == 3) ? au : __ldg(f + b + q.c) - au;
                um = uc;
                uc = up;
            } else {
                r = __ldg(u + b + q.c);
            }
            if (MODE == 0 || MODE == 1) {
                if (partials) acc = fma(r, r, acc);
            }
            if (MODE == 0 || MODE == 2) {
                dp = fma(__ldg(L.fl + b + q.c), dp, r * __ldg(L.inv + b + q.c));  // forward elimination
                out[b + q.c] = dp;  // the output field holds d'_k until the back substitution
            } else {
                out[b + q.c] = (TO)r;
            }
            tb = tc;
        }
        if (MODE == 0 || MODE == 2) {
            T x = 0;
            for (int k = nz - 1; k >= 0; --k) {
                const size_t id = (size_t)k * pl + q.c;
                x = fma(__ldg(L.fw + id), x, (T)out[id]);
                out[id] = (MODE == 0) ? fma(coef, x, __ldg(u + id)) : coef * x;
            }
        }
    }
    if ((MODE == 0 || MODE == 1) && partials) {
        const double s = block_sum((double)acc);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// RestrictSmooth onto level Lc: f_c = sum of the 2 x 2 children's residuals r_f (the equations are
// integrated over the cells), u_c = rho M_c^{-1} f_c (the first smoothing step from zero).
template <class T>
__global__ void __launch_bounds__(128) k_panel_restrict_smooth(PanelLvT<T> Lc, T rho, const T* __restrict__ rf,
                                                               T* __restrict__ fc, T* uc, const int* done) {
    if (done && *(volatile const int*)done) return;
    const PCol<T> q = panel_col(Lc);
    if (!q.act) return;
    const size_t plc = (size_t)Lc.nx * Lc.ny, nxf = 2 * (size_t)Lc.nx, plf = 4 * plc;
    const size_t f0 = (size_t)(2 * q.j) * nxf + 2 * q.i;
    T dp = 0;
    for (int k = 0; k < Lc.nz; ++k) {
        const T* r = rf + (size_t)k * plf + f0;
        const T s = (__ldg(r) + __ldg(r + 1)) + (__ldg(r + nxf) + __ldg(r + nxf + 1));
        const size_t id = (size_t)k * plc + q.c;
        fc[id] = s;
        dp = fma(__ldg(Lc.fl + id), dp, s * __ldg(Lc.inv + id));
        uc[id] = dp;
    }
    T x = 0;
    for (int k = Lc.nz - 1; k >= 0; --k) {
        const size_t id = (size_t)k * plc + q.c;
        x = fma(__ldg(Lc.fw + id), x, uc[id]);
        uc[id] = rho * x;
    }
}

// u_f += P u_c: bilinear in the logical grid (weights 3/4 and 1/4 per direction), a coarse
// neighbour beyond the panel boundary contributing 0. One thread per fine column.
template <class T>
__global__ void __launch_bounds__(128) k_panel_prolongate(int nxc, int nyc, int nz, const T* __restrict__ uc,
                                                          T* __restrict__ uf, const int* done) {
    if (done && *(volatile const int*)done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nxf = 2 * nxc, nyf = 2 * nyc;
    if (i >= nxf || j >= nyf) return;
    const int I = i >> 1, J = j >> 1;
    const int I2 = (i & 1) ? I + 1 : I - 1, J2 = (j & 1) ? J + 1 : J - 1;
    const bool in2 = I2 >= 0 && I2 < nxc, jn2 = J2 >= 0 && J2 < nyc;
    const size_t plc = (size_t)nxc * nyc, plf = (size_t)nxf * nyf;
    const size_t c0 = (size_t)J * nxc + I, cx = (size_t)J * nxc + I2, cy = (size_t)J2 * nxc + I,
                 cxy = (size_t)J2 * nxc + I2, fo = (size_t)j * nxf + i;
    for (int k = 0; k < nz; ++k) {
        const T* p = uc + (size_t)k * plc;
        T v = T(0.5625) * __ldg(p + c0);
        if (in2) v = fma(T(0.1875), __ldg(p + cx), v);
        if (jn2) v = fma(T(0.1875), __ldg(p + cy), v);
        if (in2 && jn2) v = fma(T(0.0625), __ldg(p + cxy), v);
        uf[(size_t)k * plf + fo] += v;
    }
}

// ---------------------------------------------------------------- fused CG kernels (Sec. 3.1)
// SpMV: u += alpha p; p = z + beta p; q = A z + beta q; sigma = <p, q> (alpha, beta from the previous
// iteration in the device scalars; the u update lags one iteration, as in the flat-box CG)
__global__ void __launch_bounds__(128) k_panel_cg_spmv(PanelLv L, const Scalars* __restrict__ sc, double* u,
                                                       double* p, const double* __restrict__ z, double* q,
                                                       double* partials) {
    if (*(volatile const int*)&sc->done) return;
    const PCol<double> c = panel_col(L);
    const size_t pl = (size_t)L.nx * L.ny;
    const double alpha = sc->alpha, beta = sc->beta;
    double acc = 0.0;
    if (c.act) {
        double zm = 0.0, zc = __ldg(z + c.c), tb = 0.0;
        for (int k = 0; k < L.nz; ++k) {
            const size_t b = (size_t)k * pl, id = b + c.c;
            const double tc = (k + 1 < L.nz) ? c.area * __ldg(L.B + k + 1) : 0.0;
            const double zp = (k + 1 < L.nz) ? __ldg(z + id + pl) : 0.0;
            const double az = panel_Au(L, c, z, b, k, zc, zm, zp, tb, tc);
            const double po = p[id];
            u[id] = fma(alpha, po, u[id]);
            const double pn = fma(beta, po, zc);
            const double qn = fma(beta, q[id], az);
            p[id] = pn;
            q[id] = qn;
            acc = fma(pn, qn, acc);
            zm = zc;
            zc = zp;
            tb = tc;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Tridiag: r -= alpha q; z = M^{-1} r; partial sums of <r, r> (first nparts slots) and <r, z> (next)
__global__ void __launch_bounds__(128) k_panel_cg_tridiag(PanelLv L, const Scalars* __restrict__ sc, double* r,
                                                          const double* __restrict__ q, double* z, double* partials,
                                                          int nparts) {
    if (*(volatile const int*)&sc->done) return;
    const PCol<double> c = panel_col(L);
    const size_t pl = (size_t)L.nx * L.ny;
    const double alpha = sc->alpha;
    double rr = 0.0, rz = 0.0;
    if (c.act) {
        double dp = 0.0;
        for (int k = 0; k < L.nz; ++k) {
            const size_t id = (size_t)k * pl + c.c;
            const double rk = fma(-alpha, __ldg(q + id), r[id]);
            r[id] = rk;
            rr = fma(rk, rk, rr);
            dp = fma(__ldg(L.fl + id), dp, rk * __ldg(L.inv + id));
            z[id] = dp;
        }
        double x = 0.0;
        for (int k = L.nz - 1; k >= 0; --k) {
            const size_t id = (size_t)k * pl + c.c;
            x = fma(__ldg(L.fw + id), x, z[id]);
            z[id] = x;
            rz = fma(r[id], x, rz);
        }
    }
    const double s1 = block_sum(rr);
    __syncthreads();
    const double s2 = block_sum(rz);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        partials[blockIdx.y * gridDim.x + blockIdx.x] = s1;
        partials[nparts + blockIdx.y * gridDim.x + blockIdx.x] = s2;
    }
}

static dim3 panel_grid(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 3) / 4); }

int panel_blocks(int nx, int ny) {
    const dim3 g = panel_grid(nx, ny);
    return (int)(g.x * g.y);
}

void launch_panel_cg_spmv(const PanelLv& L, const Scalars* sc, double* u, double* p, const double* z, double* q,
                          double* partials, cudaStream_t s) {
    k_panel_cg_spmv<<<panel_grid(L.nx, L.ny), dim3(32, 4), 0, s>>>(L, sc, u, p, z, q, partials);
    note_launch();
}

void launch_panel_cg_tridiag(const PanelLv& L, const Scalars* sc, double* r, const double* q, double* z,
                             double* partials, cudaStream_t s) {
    k_panel_cg_tridiag<<<panel_grid(L.nx, L.ny), dim3(32, 4), 0, s>>>(L, sc, r, q, z, partials,
                                                                        panel_blocks(L.nx, L.ny));
    note_launch();
}

void launch_panel_factors(const PanelLv& L, double* inv, double* fl, double* fw, cudaStream_t s) {
    k_panel_factors<<<panel_grid(L.nx, L.ny), dim3(32, 4), 0, s>>>(L, inv, fl, fw);
    note_launch();
}

template <class T>
int launch_panel_sweep(int mode, const PanelLvT<T>& L, double coef, const T* u, const T* f, T* out, double* partials,
                       const int* done, cudaStream_t s) {
    const dim3 g = panel_grid(L.nx, L.ny), b(32, 4);
    const T c = (T)coef;
    switch (mode) {
        case PANEL_SMOOTH: k_panel_sweep<0, T, T><<<g, b, 0, s>>>(L, c, u, f, out, partials, done); break;
        case PANEL_RESIDUAL: k_panel_sweep<1, T, T><<<g, b, 0, s>>>(L, c, u, f, out, partials, done); break;
        case PANEL_LINESOLVE: k_panel_sweep<2, T, T><<<g, b, 0, s>>>(L, c, u, f, out, nullptr, done); break;
        default: k_panel_sweep<3, T, T><<<g, b, 0, s>>>(L, c, u, f, out, nullptr, done); break;
    }
    note_launch();
    return (int)(g.x * g.y);
}

int launch_panel_residual_to_f32(const PanelLv& L, const double* u, const double* f, float* r, double* partials,
                                 const int* done, cudaStream_t s) {
    const dim3 g = panel_grid(L.nx, L.ny);
    k_panel_sweep<1, double, float><<<g, dim3(32, 4), 0, s>>>(L, 1.0, u, f, r, partials, done);
    note_launch();
    return (int)(g.x * g.y);
}

template <class T>
void launch_panel_restrict_smooth(const PanelLvT<T>& Lc, double rho, const T* rf, T* fc, T* uc, const int* done,
                                  cudaStream_t s) {
    k_panel_restrict_smooth<T><<<panel_grid(Lc.nx, Lc.ny), dim3(32, 4), 0, s>>>(Lc, (T)rho, rf, fc, uc, done);
    note_launch();
}

template <class T>
void launch_panel_prolongate(int nxc, int nyc, int nz, const T* uc, T* uf, const int* done, cudaStream_t s) {
    k_panel_prolongate<T><<<panel_grid(2 * nxc, 2 * nyc), dim3(32, 4), 0, s>>>(nxc, nyc, nz, uc, uf, done);
    note_launch();
}

#define TPMG_PANEL_INST(T)                                                                                       \
    template int launch_panel_sweep<T>(int, const PanelLvT<T>&, double, const T*, const T*, T*, double*, const int*, \
                                       cudaStream_t);                                                            \
    template void launch_panel_restrict_smooth<T>(const PanelLvT<T>&, double, const T*, T*, T*, const int*,        \
                                                  cudaStream_t);                                                  \
    template void launch_panel_prolongate<T>(int, int, int, const T*, T*, const int*, cudaStream_t);
TPMG_PANEL_INST(double)
TPMG_PANEL_INST(float)

}  // namespace tpmg
