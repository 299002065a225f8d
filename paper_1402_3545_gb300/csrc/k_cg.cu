// k_cg.cu -- the two fused kernels of the line-preconditioned CG iteration (Sec. 3.1, kernel list
// "Conjugate Gradient"), with the BLAS-1 updates and the dot products folded into the sweeps.
//
// Fused SpMV (iteration j, scalars of iteration j-1):
//   u <- u + alpha_{j-1} p ; p <- z + beta_{j-1} p ; q <- A z + beta_{j-1} q ; sigma = <p, q>
// which uses A p_j = A z_j + beta_{j-1} A p_{j-1}, so the stencil is applied to z and the
// solution update lags one iteration behind (finished by k_cg_finish).
// Fused Tridiag:
//   r <- r - alpha_j q ; z <- M^{-1} r ; <r, r> ; <r, z>
// One thread owns one vertical column; the sums are reduced per block and summed in a fixed order
// by the finalize kernels (k_util.cu), which also compute alpha and beta on the device.
#include "kernels.cuh"
#include "sweep_x2.cuh"

namespace tpmg {

static constexpr int TX = 32;
__device__ __forceinline__ int wrapc(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <class P>
__global__ void __launch_bounds__(256) k_cg_spmv(Lv<P> L, const Scalars* __restrict__ sc,
                                                 typename P::S* __restrict__ u,
                                                 typename P::S* __restrict__ p,
                                                 const typename P::S* __restrict__ z,
                                                 typename P::S* __restrict__ q, double* partials) {
    typedef typename P::R R;
    if (*(volatile const int*)&sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool act = i < L.nx && j < L.ny;
    typename P::Acc acc = 0, cmp = 0;
    if (act) {
        const size_t pl = (size_t)L.nx * L.ny, c = (size_t)j * L.nx + i;
        const size_t cw = (size_t)j * L.nx + wrapc(i - 1, L.nx), ce = (size_t)j * L.nx + wrapc(i + 1, L.nx);
        const size_t cs = (size_t)wrapc(j - 1, L.ny) * L.nx + i, cn = (size_t)wrapc(j + 1, L.ny) * L.nx + i;
        const R alpha = P::cst(sc->alpha), beta = P::cst(sc->beta);
        const R cx = P::cst(L.cx), cy = P::cst(L.cy), vv = P::ld(L.v, c);
        const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
        const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        R zm = P::zero(), zc = P::ld(z, c);
        for (int k = 0; k < L.nz; ++k) {
            const size_t b = (size_t)k * pl, id = b + c;
            R zp = (k + 1 < L.nz) ? P::ld(z, b + pl + c) : P::zero();
            R hx = P::add(P::ld(z, b + cw), P::ld(z, b + ce));
            R hy = P::add(P::ld(z, b + cs), P::ld(z, b + cn));
            R diag = (L.nz == 1) ? dh : ((k == 0 || k == L.nz - 1) ? dh1 : dh2);
            R az = P::mul(diag, zc);
            az = P::sub(az, P::mul(cx, hx));
            az = P::sub(az, P::mul(cy, hy));
            az = P::sub(az, P::mul(vv, P::add(zm, zp)));
            R pold = P::ld_plain(p, id);
            P::st(u, id, P::add(P::ld_plain(u, id), P::mul(alpha, pold)));
            R pn = P::add(zc, P::mul(beta, pold));
            R qn = P::add(az, P::mul(beta, P::ld_plain(q, id)));
            P::st(p, id, pn);
            P::st(q, id, qn);
            P::acc_dot(acc, cmp, pn, qn);
            zm = zc;
            zc = zp;
        }
    }
    double s = block_sum(P::acc_get(acc, cmp));
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// The fused SpMV pointwise: the stencil has no recurrence along the column, so every pair of
// x-adjacent cells of a plane is a thread (grid-stride over the pairs, a fixed number of blocks for
// the partial sums); neighbours come through the read-only cache. Requires nx even.
template <class P>
__global__ void __launch_bounds__(256) k_cg_spmv_cell(Lv<P> L, const Scalars* __restrict__ sc,
                                                      typename P::S* __restrict__ u, typename P::S* __restrict__ p,
                                                      const typename P::S* __restrict__ z,
                                                      typename P::S* __restrict__ q, double* partials) {
    typedef typename P::R R;
    if (*(volatile const int*)&sc->done) return;
    const int nx = L.nx, ny = L.ny, nz = L.nz, hx2 = nx / 2;
    const size_t pl = (size_t)nx * ny, npairs = (size_t)hx2 * ny * nz;
    const R alpha = P::cst(sc->alpha), beta = P::cst(sc->beta);
    const R cx = P::cst(L.cx), cy = P::cst(L.cy);
    const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    const bool iso = L.cx == L.cy;
    typename P::Acc acc = 0, cmp = 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < npairs; t += (size_t)gridDim.x * blockDim.x) {
        const int ip = (int)(t % hx2), j = (int)((t / hx2) % ny), k = (int)(t / ((size_t)hx2 * ny));
        const int i = 2 * ip;
        const size_t c = (size_t)j * nx + i, b = (size_t)k * pl, id = b + c;
        const size_t rs = (size_t)wrapc(j - 1, ny) * nx + i, rn = (size_t)wrapc(j + 1, ny) * nx + i;
        const R z0 = P::ld(z, id), z1 = P::ld(z, id + 1);
        const R zw = P::ld(z, b + (size_t)j * nx + wrapc(i - 1, nx)), ze = P::ld(z, b + (size_t)j * nx + wrapc(i + 2, nx));
        const R zs0 = P::ld(z, b + rs), zs1 = P::ld(z, b + rs + 1), zn0 = P::ld(z, b + rn), zn1 = P::ld(z, b + rn + 1);
        R zm0 = P::zero(), zm1 = P::zero(), zp0 = P::zero(), zp1 = P::zero();
        if (k > 0) {
            zm0 = P::ld(z, id - pl);
            zm1 = P::ld(z, id - pl + 1);
        }
        if (k + 1 < nz) {
            zp0 = P::ld(z, id + pl);
            zp1 = P::ld(z, id + pl + 1);
        }
        const R v0 = P::ld(L.v, c), v1 = P::ld(L.v, c + 1);
        R d0 = dh, d1 = dh;
        if (k > 0) {
            d0 = P::add(d0, v0);
            d1 = P::add(d1, v1);
        }
        if (k + 1 < nz) {
            d0 = P::add(d0, v0);
            d1 = P::add(d1, v1);
        }
        // A z = -(f - A z) with f = 0: the sweep residual of a zero right-hand side, negated
        const R az0 = P::neg(sweep_residual<P>(P::zero(), d0, z0, zw, z1, zs0, zn0, zm0, zp0, cx, cy, v0, iso));
        const R az1 = P::neg(sweep_residual<P>(P::zero(), d1, z1, z0, ze, zs1, zn1, zm1, zp1, cx, cy, v1, iso));
        const R po0 = P::ld_plain(p, id), po1 = P::ld_plain(p, id + 1);
        P::st(u, id, P::fma(alpha, po0, P::ld_plain(u, id)));
        P::st(u, id + 1, P::fma(alpha, po1, P::ld_plain(u, id + 1)));
        const R pn0 = P::fma(beta, po0, z0), pn1 = P::fma(beta, po1, z1);
        const R qn0 = P::fma(beta, P::ld_plain(q, id), az0), qn1 = P::fma(beta, P::ld_plain(q, id + 1), az1);
        P::st(p, id, pn0);
        P::st(p, id + 1, pn1);
        P::st(q, id, qn0);
        P::st(q, id + 1, qn1);
        P::acc_dot(acc, cmp, pn0, qn0);
        P::acc_dot(acc, cmp, pn1, qn1);
    }
    const double s = block_sum(P::acc_get(acc, cmp));
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <class P>
__global__ void __launch_bounds__(256) k_cg_tridiag(Lv<P> L, const Scalars* __restrict__ sc,
                                                    typename P::S* __restrict__ r,
                                                    const typename P::S* __restrict__ q,
                                                    typename P::S* __restrict__ z, double* partials) {
    typedef typename P::R R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (*(volatile const int*)&sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool act = i < L.nx && j < L.ny;
    typename P::Acc arr = 0, crr = 0, arz = 0, crz = 0;
    if (act) {
        const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
        R* dp = reinterpret_cast<R*>(smem_raw);
        R* w = dp + (size_t)L.nz * nt;
        const size_t pl = (size_t)L.nx * L.ny, c = (size_t)j * L.nx + i;
        const R alpha = P::cst(sc->alpha);
        const R vv = P::ld(L.v, c), vv2 = P::mul(vv, vv);
        const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
        const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        R inv_prev = P::zero(), d_prev = P::zero();
        for (int k = 0; k < L.nz; ++k) {
            const size_t id = (size_t)k * pl + c;
            R rn = P::sub(P::ld_plain(r, id), P::mul(alpha, P::ld(q, id)));
            P::st(r, id, rn);
            P::acc_dot(arr, crr, rn, rn);
            R diag = (L.nz == 1) ? dh : ((k == 0 || k == L.nz - 1) ? dh1 : dh2);
            R m = (k == 0) ? diag : P::sub(diag, P::mul(vv2, inv_prev));
            R inv = P::rcp(m);
            R d = P::mul(P::add(rn, P::mul(vv, d_prev)), inv);
            dp[(size_t)k * nt + tid] = d;
            w[(size_t)k * nt + tid] = P::mul(vv, inv);
            inv_prev = inv;
            d_prev = d;
        }
        R xn = P::zero();
        for (int k = L.nz - 1; k >= 0; --k) {
            const size_t id = (size_t)k * pl + c;
            xn = P::add(dp[(size_t)k * nt + tid], P::mul(w[(size_t)k * nt + tid], xn));
            P::st(z, id, xn);
            P::acc_dot(arz, crz, P::ld_plain(r, id), xn);
        }
    }
    double s1 = block_sum(P::acc_get(arr, crr));
    double s2 = block_sum(P::acc_get(arz, crz));
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int b = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
        partials[b] = s1;
        partials[nb + b] = s2;
    }
}

// The same fused Tridiag with the level's precomputed Thomas factors (1/m_k, v/m_k) and the
// forward-eliminated values on a per-block stack in the global scratch (L.gstack): a persistent
// grid of a few blocks per SM loops over tiles of 32 x 4 columns. No reciprocal per cell and no
// shared-memory stack, so the SM holds as many warps as its registers allow.
template <class P>
__global__ void __launch_bounds__(128) k_cg_tridiag_gs(Lv<P> L, const Scalars* __restrict__ sc,
                                                       typename P::S* __restrict__ r,
                                                       const typename P::S* __restrict__ q,
                                                       typename P::S* __restrict__ z, double* partials) {
    typedef typename P::R R;
    typedef typename P::S S;
    if (*(volatile const int*)&sc->done) return;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int tiles_x = (nx + 31) / 32, ntiles = tiles_x * ((ny + 3) / 4);
    const size_t pl = (size_t)nx * ny;
    const bool percol = L.fac_percol != 0;
    S* gst = reinterpret_cast<S*>(L.gstack) + (size_t)blockIdx.x * nz * 128;
    const R nalpha = P::neg(P::cst(sc->alpha));
    typename P::Acc arr = 0, crr = 0, arz = 0, crz = 0;
    // q, the factors and z stream through L2 evict-first; the stack is stored evict-last and each
    // of its lines is dropped once read (see the persistent Smooth)
    const unsigned long long pol_first = l2_evict_first(), pol_last = l2_evict_last();
    constexpr int LANES_PER_LINE = 128 / (int)sizeof(S);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = (tile % tiles_x) * 32 + threadIdx.x, j = (tile / tiles_x) * 4 + threadIdx.y;
        const bool active = i < nx && j < ny;
        const size_t c = (size_t)j * nx + i;
        const R vv = active ? P::ld(L.v, c) : P::zero();
        R d_prev = P::zero();
        for (int k = 0; k < nz && active; ++k) {
            const size_t id = (size_t)k * pl + c;
            const R rn = P::fma(nalpha, ld_pol(q + id, pol_first), P::ld_plain(r, id));
            P::st(r, id, rn);
            P::acc_dot(arr, crr, rn, rn);
            const R inv = percol ? ld_pol(L.finv + id, pol_first) : P::ld(L.finv, k);
            d_prev = P::mul(P::fma(vv, d_prev, rn), inv);
            st_pol(gst + (size_t)k * 128 + tid, d_prev, pol_last);
        }
        R xn = P::zero();
        for (int k = nz - 1; k >= 0; --k) {
            const size_t id = (size_t)k * pl + c;
            if (active) {
                const R w = percol ? ld_pol(L.fw + id, pol_first) : P::ld(L.fw, k);
                xn = P::fma(w, xn, P::ld_plain(gst, (size_t)k * 128 + tid));
                st_pol(z + id, xn, pol_first);
                P::acc_dot(arz, crz, P::ld_plain(r, id), xn);
            }
            // every lane of the warp has consumed its stack value of plane k: drop the dead lines
            __syncwarp();
            if (tid % LANES_PER_LINE == 0) l2_discard(gst + (size_t)k * 128 + tid);
        }
    }
    double s1 = block_sum(P::acc_get(arr, crr));
    double s2 = block_sum(P::acc_get(arz, crz));
    if (tid == 0) {
        partials[blockIdx.x] = s1;
        partials[gridDim.x + blockIdx.x] = s2;
    }
}

// The fused Tridiag on two columns per thread, plane-pipelined like the two-column Smooth
// (sweep_x2.cuh): each plane's r, q and (where the elimination has not converged) 1/m_k pairs
// arrive by cp.async PD planes ahead; the forward-eliminated values go to the block's scratch slot
// (evict-last, each line dropped from L2 once read back). <r, z> is taken in the forward sweep: with
// the column block M = U^T D U (D = diag(m_k), U unit upper bidiagonal), the elimination gives
// yh = U^{-T} r (yh_k = r_k + v d'_{k-1}) and d'_k = yh_k / m_k, so <r, M^{-1} r> = sum_k yh_k d'_k,
// a sum of non-negative terms, and the back substitution does not read r again.
// Tiles of 64 x TY columns; requires nx % 64 == 0, ny % TY == 0, 16-byte aligned fields.
template <class P, int TY, int PD>
__global__ void __launch_bounds__(32 * TY) k_cg_tridiag_x2(Lv<P> L, const Scalars* __restrict__ sc,
                                                           typename P::S* __restrict__ r,
                                                           const typename P::S* __restrict__ q,
                                                           typename P::S* __restrict__ z, double* partials) {
    typedef typename P::S S;
    typedef typename P::R R;
    constexpr int NT = 32 * TY, SL = 2 * NT;  // values per ring slot and array
    constexpr int PB = 2 * (int)sizeof(S);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (*(volatile const int*)&sc->done) return;
    const int nx = L.nx, ny = L.ny, nz = L.nz, tid = threadIdx.y * 32 + threadIdx.x;
    const size_t pl = (size_t)nx * ny;
    const int tiles_x = nx / 64, ntiles = tiles_x * (ny / TY);
    const bool percol = L.fac_percol != 0;
    const int k0 = L.fac_k0;
    S* ringR = reinterpret_cast<S*>(smem_raw);
    S* ringQ = ringR + PD * SL;
    S* ringI = ringQ + PD * SL;
    S* gst = reinterpret_cast<S*>(L.gstack) + (size_t)blockIdx.x * nz * SL;
    const R nalpha = P::neg(P::cst(sc->alpha));
    const unsigned long long pol_first = l2_evict_first(), pol_last = l2_evict_last();
    typename P::Acc arr = 0, crr = 0, arz = 0, crz = 0;
    const R vzero = P::zero();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i0 = (tile % tiles_x) * 64, j0 = (tile / tiles_x) * TY;
        const size_t c = (size_t)(j0 + threadIdx.y) * nx + i0 + 2 * threadIdx.x;
        __syncthreads();  // the previous tile's rings are no longer read
        auto issue_plane = [&](int k, int slot) {
            if (k < nz) {
                const size_t id = (size_t)k * pl + c;
                cp_async<PB>(&ringR[slot * SL + 2 * tid], r + id);
                cp_async_pol<PB>(&ringQ[slot * SL + 2 * tid], q + id, pol_first);
                if (percol && !(k >= k0 && k <= nz - 2))
                    cp_async_pol<PB>(&ringI[slot * SL + 2 * tid], L.finv + id, pol_first);
            }
            cp_commit();
        };
        for (int sl = 0; sl < PD; ++sl) issue_plane(sl, sl);
        const R v0 = P::ld(L.v, c), v1 = P::ld(L.v, c + 1);
        R ci0 = vzero, ci1 = vzero, cw0 = vzero, cw1 = vzero;
        if (percol && k0 <= nz - 2) {
            const size_t rr = (size_t)(nz - 2) * pl + c;
            ci0 = P::ld(L.finv, rr);
            ci1 = P::ld(L.finv, rr + 1);
            cw0 = P::ld(L.fw, rr);
            cw1 = P::ld(L.fw, rr + 1);
        }
        R dp0 = vzero, dp1 = vzero;
        int slot = 0;
        for (int k = 0; k < nz; ++k) {
            cp_wait<PD - 1>();  // this thread's copies of plane k
            const int o = slot * SL + 2 * tid;
            const R rn0 = P::fma(nalpha, P::ld_plain(ringQ, o), P::ld_plain(ringR, o));
            const R rn1 = P::fma(nalpha, P::ld_plain(ringQ, o + 1), P::ld_plain(ringR, o + 1));
            const size_t id = (size_t)k * pl + c;
            st_pair_pol(r + id, rn0, rn1, pol_first);
            P::acc_dot(arr, crr, rn0, rn0);
            P::acc_dot(arr, crr, rn1, rn1);
            R i0v, i1v;
            if (!percol) {
                i0v = i1v = P::ld(L.finv, k);
            } else if (k >= k0 && k <= nz - 2) {
                i0v = ci0;
                i1v = ci1;
            } else {
                i0v = P::ld_plain(ringI, o);
                i1v = P::ld_plain(ringI, o + 1);
            }
            const R yh0 = P::fma(v0, dp0, rn0), yh1 = P::fma(v1, dp1, rn1);
            dp0 = P::mul(yh0, i0v);
            dp1 = P::mul(yh1, i1v);
            P::acc_dot(arz, crz, yh0, dp0);
            P::acc_dot(arz, crz, yh1, dp1);
            st_pair_pol(gst + ((size_t)k * NT + tid) * 2, dp0, dp1, pol_last);
            issue_plane(k + PD, slot);
            slot = (slot + 1 == PD) ? 0 : slot + 1;
        }
        cp_wait<0>();
        __syncthreads();  // the backward ring reuses the forward ring's shared memory
        S* bW = reinterpret_cast<S*>(smem_raw);
        S* bD = bW + PD * SL;
        auto issue_back = [&](int k, int s2) {
            if (k >= 0) {
                if (percol && !(k >= k0 && k <= nz - 2))
                    cp_async_pol<PB>(&bW[s2 * SL + 2 * tid], L.fw + (size_t)k * pl + c, pol_first);
                cp_async<PB>(&bD[s2 * SL + 2 * tid], gst + ((size_t)k * NT + tid) * 2);
            }
            cp_commit();
        };
        for (int sl = 0; sl < PD; ++sl) issue_back(nz - 1 - sl, sl);
        R x0 = vzero, x1 = vzero;
        slot = 0;
        for (int k = nz - 1; k >= 0; --k) {
            cp_wait<PD - 1>();
            {
                // plane k of the stack has landed for every lane of the warp: its lines are dead
                constexpr int LANES_PER_LINE = 128 / PB;
                __syncwarp();
                if (tid % LANES_PER_LINE == 0) l2_discard(gst + ((size_t)k * NT + tid) * 2);
            }
            const int o = slot * SL + 2 * tid;
            R w0, w1;
            if (!percol) {
                w0 = w1 = P::ld(L.fw, k);
            } else if (k >= k0 && k <= nz - 2) {
                w0 = cw0;
                w1 = cw1;
            } else {
                w0 = P::ld_plain(bW, o);
                w1 = P::ld_plain(bW, o + 1);
            }
            x0 = P::fma(w0, x0, P::ld_plain(bD, o));
            x1 = P::fma(w1, x1, P::ld_plain(bD, o + 1));
            st_pair_pol(z + (size_t)k * pl + c, x0, x1, pol_first);
            issue_back(k - PD, slot);
            slot = (slot + 1 == PD) ? 0 : slot + 1;
        }
        cp_wait<0>();
    }
    const double s1 = block_sum(P::acc_get(arr, crr));
    const double s2 = block_sum(P::acc_get(arz, crz));
    if (tid == 0) {
        partials[blockIdx.x] = s1;
        partials[gridDim.x + blockIdx.x] = s2;
    }
}

static constexpr int CGX_TY = 2, CGX_PD = 4;
template <class P>
static bool cg_x2_fits(const Lv<P>& L) {
    return P::id != 0 && L.gstack && L.finv && L.fw && L.nx % 64 == 0 && L.ny % CGX_TY == 0;
}
template <class P>
static size_t cg_x2_smem() {
    return (size_t)CGX_PD * 3 * 2 * 32 * CGX_TY * sizeof(typename P::S);
}
template <class P>
static int cg_x2_blocks(const Lv<P>& L) {
    static int per_sm = 0, nsm = 0;
    if (per_sm == 0) {
        auto kern = k_cg_tridiag_x2<P, CGX_TY, CGX_PD>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cg_x2_smem<P>());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * CGX_TY, cg_x2_smem<P>());
        if (per_sm > 10) per_sm = 10;
        if (per_sm < 1) per_sm = 1;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    int nb = nsm * per_sm;
    // the scratch slots: 64 TY columns per block out of gstack_bytes
    const int slots = nsm * GS_BLOCKS_PER_SM * GS_MAX_NT / (2 * 32 * CGX_TY);
    if (nb > slots) nb = slots;
    const int ntiles = (L.nx / 64) * (L.ny / CGX_TY);
    return nb < ntiles ? nb : ntiles;
}

// u <- u + alpha p : the lagged solution update after the last iteration.
template <class P>
__global__ void k_cg_finish(size_t n, const Scalars* __restrict__ sc, typename P::S* __restrict__ u,
                            const typename P::S* __restrict__ p) {
    const typename P::R alpha = P::cst(sc->alpha);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        P::st(u, t, P::add(P::ld_plain(u, t), P::mul(alpha, P::ld(p, t))));
}

// the pointwise SpMV for the FP32-pipe policies (native FP64 keeps the column kernel, which reuses
// the vertical neighbours from registers and runs faster on the slow FP64 pipe)
template <class P>
int cg_spmv_blocks(const Lv<P>& L) {
    if (L.nx % 2 == 0 && P::id != 0) {
        const size_t b = ((size_t)L.nx / 2 * L.ny * L.nz + 255) / 256;
        return (int)(b < 152 * 8 ? (b ? b : 1) : 152 * 8);
    }
    return sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), false).nblocks();
}
template <class P>
int launch_cg_spmv(const Lv<P>& L, const Scalars* sc, typename P::S* u, typename P::S* p,
                   const typename P::S* z, typename P::S* q, double* partials, cudaStream_t s) {
    if (L.nx % 2 == 0 && P::id != 0) {
        const int nb = cg_spmv_blocks(L);
        k_cg_spmv_cell<P><<<nb, 256, 0, s>>>(L, sc, u, p, z, q, partials);
        note_launch();
        return nb;
    }
    Shape sh = sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), false);
    k_cg_spmv<P><<<sh.grid, sh.block, 0, s>>>(L, sc, u, p, z, q, partials);
    note_launch();
    return sh.nblocks();
}
// blocks of the fused Tridiag (= partial sums per quantity); the persistent form when the level has
// its factors and the scratch
template <class P>
int cg_tridiag_blocks(const Lv<P>& L) {
    if (cg_x2_fits(L)) return cg_x2_blocks(L);
    if (L.gstack && L.finv && L.fw) {
        static int per_sm = 0;
        if (per_sm == 0) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_tridiag_gs<P>, 128, 0);
            if (per_sm > GS_BLOCKS_PER_SM) per_sm = GS_BLOCKS_PER_SM;
            if (per_sm < 1) per_sm = 1;
        }
        int nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int ntiles = ((L.nx + 31) / 32) * ((L.ny + 3) / 4);
        const int nb = nsm * per_sm;
        return nb < ntiles ? nb : ntiles;
    }
    return sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), true).nblocks();
}
template <class P>
int launch_cg_tridiag(const Lv<P>& L, const Scalars* sc, typename P::S* r, const typename P::S* q,
                      typename P::S* z, double* partials, cudaStream_t s) {
    if (cg_x2_fits(L)) {
        const int nb = cg_x2_blocks(L);
        k_cg_tridiag_x2<P, CGX_TY, CGX_PD><<<nb, dim3(32, CGX_TY), cg_x2_smem<P>(), s>>>(L, sc, r, q, z, partials);
        note_launch();
        return nb;
    }
    if (L.gstack && L.finv && L.fw) {
        const int nb = cg_tridiag_blocks(L);
        k_cg_tridiag_gs<P><<<nb, dim3(32, 4), 0, s>>>(L, sc, r, q, z, partials);
        note_launch();
        return nb;
    }
    Shape sh = sweep_shape(L.nx, L.ny, L.nz, sizeof(typename P::R), true);
    if (sh.smem > 32 * 1024)
        cudaFuncSetAttribute(k_cg_tridiag<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    k_cg_tridiag<P><<<sh.grid, sh.block, sh.smem, s>>>(L, sc, r, q, z, partials);
    note_launch();
    return sh.nblocks();
}
template <class P>
void launch_cg_finish(size_t n, const Scalars* sc, typename P::S* u, const typename P::S* p,
                      cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_cg_finish<P><<<(unsigned)blocks, 256, 0, s>>>(n, sc, u, p);
    note_launch();
}

#define TPMG_CG_INST(P)                                                                             \
    template int cg_spmv_blocks<P>(const Lv<P>&);                                                   \
    template int cg_tridiag_blocks<P>(const Lv<P>&);                                                \
    template int launch_cg_spmv<P>(const Lv<P>&, const Scalars*, P::S*, P::S*, const P::S*, P::S*,  \
                                   double*, cudaStream_t);                                         \
    template int launch_cg_tridiag<P>(const Lv<P>&, const Scalars*, P::S*, const P::S*, P::S*,      \
                                      double*, cudaStream_t);                                      \
    template void launch_cg_finish<P>(size_t, const Scalars*, P::S*, const P::S*, cudaStream_t);

TPMG_CG_INST(PolF64)
TPMG_CG_INST(PolF32)
TPMG_CG_INST(PolDW)

}  // namespace tpmg
