// sweep_x2.cuh -- the two-column plane-pipelined column sweep as a device function, used by the
// persistent sweep kernels (k_sweep.cu) and, one tile per task, by the batched persistent solver
// (k_batched.cu); plus the cp.async helpers and sweep modes they share.
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace tpmg {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES));
}
// the same with an L2 eviction-priority policy (createpolicy) attached to the global read
template <int BYTES>
__device__ __forceinline__ void cp_async_pol(void* dst, const void* src, unsigned long long pol) {
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                     "l"(pol));
    else
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)), "l"(src),
                     "n"(BYTES), "l"(pol));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// MODE_APPLY: out = A u (f unused), formed as -(0 - A u) by the residual's stencil: negation is exact
enum { MODE_SMOOTH = 0, MODE_RESIDUAL = 1, MODE_LINESOLVE = 2, MODE_RESTRICT = 3, MODE_APPLY = 4 };
// modes whose per-column Thomas stack lives in the block's scratch slot (MODE_RESTRICT keeps the
// stack of the coarse column there)
__host__ __device__ constexpr bool x2_stack(int mode) { return mode == MODE_SMOOTH || mode == MODE_LINESOLVE; }
__host__ __device__ constexpr bool x2_slot(int mode) { return mode != MODE_RESIDUAL && mode != MODE_APPLY; }

// MODE_RESTRICT: the fine level's residual r = f - A u is not stored; each 2 x 2 group of fine
// columns is restricted on the fly to the coarse right-hand side f_c = 1/4 (sum of the children)
// and the coarse level's first smoothing step from a zero guess, u_c = rho M_c^{-1} f_c, follows
// (Residual and RestrictSmooth of Algorithm 1 in one pass over the fine level). The coarse level
// and the two outputs:
template <class P>
struct XRestrict {
    Lv<P> Lc;
    typename P::R rho;      // converted on the host (P::hcst)
    typename P::R quarter;  // 1/4, likewise
    typename P::S* fc;
    typename P::S* uc;
};

// L2 eviction hints of the persistent sweeps (bit mask). The Thomas scratch of a persistent block
// is written in the forward sweep and read back in the backward sweep a whole column later; the
// fields stream through L2 in between and, at the default priority, push the scratch out to DRAM
// (written back, then read again). HINT_STREAM marks the single-use reads (f, 1/m_k, v/m_k, the
// backward re-read of u) and the result store evict-first; HINT_KEEP stores the scratch
// evict-last; HINT_DISCARD drops each scratch line from L2 once the backward sweep has read it, so
// dead scratch is never written back. On the mid workload these cut DRAM traffic of the DW Smooth
// from 2.03 to 1.76 GB per launch.
constexpr int HINT_STREAM = 1, HINT_KEEP = 2, HINT_DISCARD = 4, HINT_ALL = 7;

// ---------------------------------------------------------------- two columns per thread
// Tiles tile0, tile0 + tile_step, ... < tile_end of 64 x TY columns (tile t covers x from
// (t % (nx/64)) * 64, y from (t / (nx/64)) * TY), each thread owning two adjacent columns: every
// per-thread load, store and cp.async moves a 16-byte pair (8 bytes in FP32), and the two
// independent Thomas recurrences interleave. gstack is this block's scratch slot of nz x 64 TY
// values (unused in residual and apply modes; the coarse columns' stack in restrict mode); smem_raw
// its dynamic shared memory (sweep_x2_smem bytes); K the level's constants and the mode's
// coefficient (rho for Smooth, the line solve's scale, 1 otherwise). Every thread of the block must
// call it (barriers). Shared ring per slot: u rows of stride UW = 68 (pad, left halo, 64 columns, right
// halo, pad), rows j0-1 .. j0+TY; f pairs; 1/m_k pairs (restrict mode: the coarse columns' 1/m_k,
// then a two-plane buffer of the odd rows' pair sums). xr: the coarse level and outputs of restrict
// mode (unused otherwise). Requires nx % 64 == 0, ny % TY == 0 and 16-byte aligned fields.
template <class P, class PO, int TY, int PD, int MODE, int HINT = 0>
__device__ __forceinline__ double sweep_x2_tiles(const Lv<P>& L, const SweepK<P>& K, const typename P::S* __restrict__ u,
                                                 const typename P::S* __restrict__ f,
                                                 typename PO::S* __restrict__ out, bool want_norm, int tile0,
                                                 int tile_end, int tile_step, typename P::S* gstack,
                                                 unsigned char* smem_raw, const XRestrict<P>* xr = nullptr) {
    typedef typename P::S S;
    typedef typename P::R R;
    constexpr int NT = 32 * TY;
    constexpr int UW = 68;
    constexpr bool STACK = x2_stack(MODE);
    constexpr bool HALO = MODE != MODE_LINESOLVE;
    constexpr bool RESTR = MODE == MODE_RESTRICT;
    static_assert(!RESTR || TY % 2 == 0, "the fused restriction pairs the block's rows");
    constexpr int CR = TY / 2;  // RESTR: coarse rows per tile
    constexpr bool GFORM = MODE == MODE_SMOOTH && P::id == 1;  // as in k_sweep_pp
    constexpr int UPL = HALO ? (TY + 2) * UW : 0;
    constexpr int FPL = 2 * NT;
    constexpr int IPL = STACK ? 2 * NT : 0;
    constexpr int PB = 2 * (int)sizeof(S);  // bytes of a column pair

    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const bool percol = L.fac_percol != 0;
    S* ringU = reinterpret_cast<S*>(smem_raw);
    S* ringF = ringU + PD * UPL;
    S* ringI = ringF + PD * FPL;
    S* ringIc = ringI + PD * IPL;  // RESTR: 1/m_k of the coarse columns, 32 CR per plane
    S* xs = ringIc + (RESTR ? PD * 32 * CR : 0);  // RESTR: row pair sums of the odd rows, 2 planes

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    // RESTR: rows 2q and 2q+1 of a tile are the children of coarse row q; the even row's thread
    // owns coarse column ci of the tile
    const int cr = TY == 2 ? 0 : ty >> 1, ci = cr * 32 + tx;  // (threadIdx.y < TY: constant when TY = 2)
    const bool even = TY == 2 ? ty == 0 : (ty & 1) == 0;
    const size_t pl = (size_t)nx * ny;
    const int tiles_x = nx / 64;
    const S* rhs = (MODE == MODE_LINESOLVE) ? u : f;
    const R vzero = P::zero();
    typename P::Acc acc = 0, cmp = 0;
    const bool iso = K.iso != 0;
    const int k0 = L.fac_k0;
    unsigned long long pol_first = 0, pol_last = 0;
    if constexpr (HINT != 0) {
        pol_first = l2_evict_first();
        pol_last = l2_evict_last();
    }

    for (int tile = tile0; tile < tile_end; tile += tile_step) {
        const int i0 = (tile % tiles_x) * 64, j0 = (tile / tiles_x) * TY;
        const size_t c = (size_t)(j0 + ty) * nx + (i0 + 2 * tx);  // the thread's first column
        // RESTR: the coarse column over this thread's pair and the pair of the row pair's other row
        const size_t plc = pl / 4;
        const size_t cc = (size_t)(j0 / 2 + cr) * (nx / 2) + (i0 / 2 + tx);
        __syncthreads();  // the previous tile's rings are no longer read

        // halo of the u plane: 2 rows x 32 pairs (one pair per thread when TY = 2) and 2 TY side
        // singles; ring offsets and in-plane sources are the same for every plane
        constexpr int NPAIR = 64, NSIDE = 2 * TY;
        constexpr int PPT = (NPAIR + NT - 1) / NT;
        int hp_dst[PPT];
        size_t hp_src[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int it = tid + q * NT;
            const int top = it < 32, p = it & 31;
            const int gj = top ? (j0 == 0 ? ny - 1 : j0 - 1) : (j0 + TY == ny ? 0 : j0 + TY);
            hp_dst[q] = it < NPAIR ? (top ? 0 : (TY + 1) * UW) + 2 + 2 * p : -1;
            hp_src[q] = (size_t)gj * nx + i0 + 2 * p;
        }
        int hs_dst = -1;
        size_t hs_src = 0;
        if (tid < NSIDE) {
            const int r = tid >> 1, right = tid & 1;
            hs_dst = (r + 1) * UW + (right ? 66 : 1);
            hs_src = (size_t)(j0 + r) * nx + (right ? (i0 + 64 == nx ? 0 : i0 + 64) : (i0 == 0 ? nx - 1 : i0 - 1));
        }

        auto issue_plane = [&](int k, int slot) {
            if (k < nz) {
                const size_t b = (size_t)k * pl;
                S* Us = ringU + slot * UPL;
                const bool fac = STACK && percol && !(k >= k0 && k <= nz - 2);  // factors of plane k needed
                if constexpr ((HINT & HINT_STREAM) != 0) {
                    if (MODE != MODE_APPLY) cp_async_pol<PB>(&ringF[slot * FPL + 2 * tid], rhs + b + c, pol_first);
                    if (fac) cp_async_pol<PB>(&ringI[slot * FPL + 2 * tid], L.finv + b + c, pol_first);
                } else {
                    if (MODE != MODE_APPLY) cp_async<PB>(&ringF[slot * FPL + 2 * tid], rhs + b + c);
                    if (fac) cp_async<PB>(&ringI[slot * FPL + 2 * tid], L.finv + b + c);
                }
                if constexpr (RESTR) {
                    const int kc0 = xr->Lc.fac_k0;
                    if (even && xr->Lc.fac_percol && !(k >= kc0 && k <= nz - 2))
                        cp_async<sizeof(S)>(&ringIc[slot * 32 * CR + ci], xr->Lc.finv + (size_t)k * plc + cc);
                }
                if (HALO) {
                    cp_async<PB>(&Us[(ty + 1) * UW + 2 + 2 * tx], u + b + c);
#pragma unroll
                    for (int q = 0; q < PPT; ++q)
                        if (hp_dst[q] >= 0) cp_async<PB>(&Us[hp_dst[q]], u + b + hp_src[q]);
                    if (hs_dst >= 0) cp_async<sizeof(S)>(&Us[hs_dst], u + b + hs_src);
                }
            }
            cp_commit();
        };
        for (int s = 0; s < PD; ++s) issue_plane(s, s);

        const R v0 = P::ld(L.v, c), v1 = P::ld(L.v, c + 1);
        // the converged factors (plane nz-2) of this thread's columns, used on planes k0 .. nz-2
        R ci0 = vzero, ci1 = vzero, cw0 = vzero, cw1 = vzero;
        if (STACK && percol && k0 <= nz - 2) {
            const size_t r = (size_t)(nz - 2) * pl + c;
            ci0 = P::ld(L.finv, r);
            ci1 = P::ld(L.finv, r + 1);
            cw0 = P::ld(L.fw, r);
            cw1 = P::ld(L.fw, r + 1);
        }
        const R cx = K.cx, cy = K.cy, cf = K.coef, dh = K.dh;
        const R dh1a = P::add(dh, v0), dh2a = P::add(dh1a, v0);
        const R dh1b = P::add(dh, v1), dh2b = P::add(dh1b, v1);
        R um0 = vzero, um1 = vzero, uc0 = vzero, uc1 = vzero, dp0 = vzero, dp1 = vzero;
        // RESTR: coupling and converged factors of the coarse column, its forward-eliminated value
        R vcc = vzero, cic = vzero, cwc = vzero, dpc = vzero, qv = vzero;
        if constexpr (RESTR) {
            if (even) {
                vcc = P::ld(xr->Lc.v, cc);
                if (xr->Lc.fac_percol && xr->Lc.fac_k0 <= nz - 2) {
                    cic = P::ld(xr->Lc.finv, (size_t)(nz - 2) * plc + cc);
                    cwc = P::ld(xr->Lc.fw, (size_t)(nz - 2) * plc + cc);
                }
            }
        }
        int slot = 0;
        const int ctr = (ty + 1) * UW + 2 + 2 * tx;
        for (int k = 0; k < nz; ++k) {
            const int nslot = (slot + 1 == PD) ? 0 : slot + 1;
            R r0, r1;
            if constexpr (!HALO) {
                cp_wait<PD - 1>();  // only this thread's own copies are read: no barrier needed
                r0 = P::ld_plain(ringF, slot * FPL + 2 * tid);
                r1 = P::ld_plain(ringF, slot * FPL + 2 * tid + 1);
            } else {
                cp_wait<PD - 2>();  // planes k and k+1 have landed
                __syncthreads();    // ... including the halo values other threads fetched
                const S* Us = ringU + slot * UPL;
                if (k == 0) {
                    uc0 = P::ld_plain(Us, ctr);
                    uc1 = P::ld_plain(Us, ctr + 1);
                }
                R up0 = vzero, up1 = vzero;
                if (k + 1 < nz) {
                    up0 = P::ld_plain(ringU + nslot * UPL, ctr);
                    up1 = P::ld_plain(ringU + nslot * UPL, ctr + 1);
                }
                const R wv = P::ld_plain(Us, ctr - 1), ev = P::ld_plain(Us, ctr + 2);
                const R s0 = P::ld_plain(Us, ctr - UW), s1 = P::ld_plain(Us, ctr - UW + 1);
                const R n0 = P::ld_plain(Us, ctr + UW), n1 = P::ld_plain(Us, ctr + UW + 1);
                const bool end = nz == 1 || k == 0 || k == nz - 1;
                const R dga = nz == 1 ? dh : (end ? dh1a : dh2a), dgb = nz == 1 ? dh : (end ? dh1b : dh2b);
                const R f0 = MODE == MODE_APPLY ? vzero : P::ld_plain(ringF, slot * FPL + 2 * tid);
                const R f1 = MODE == MODE_APPLY ? vzero : P::ld_plain(ringF, slot * FPL + 2 * tid + 1);
                r0 = sweep_residual<P>(f0, dga, uc0, wv, uc1, s0, n0, um0, up0,
                                       cx, cy, v0, iso);
                r1 = sweep_residual<P>(f1, dgb, uc1, uc0, ev, s1, n1, um1,
                                       up1, cx, cy, v1, iso);
                if (want_norm) {
                    P::acc_dot(acc, cmp, r0, r0);
                    P::acc_dot(acc, cmp, r1, r1);
                }
                um0 = uc0;
                um1 = uc1;
                uc0 = up0;
                uc1 = up1;
                if constexpr (RESTR) {
                    qv = P::add(r0, r1);  // the row pair's sum; the odd row hands it over
                    if (!even) P::st(xs, (k & 1) * 32 * CR + ci, qv);
                }
            }
            if constexpr (MODE == MODE_APPLY) {
                const size_t id = (size_t)k * pl + c;
                P::st(out, id, P::neg(r0));
                P::st(out, id + 1, P::neg(r1));
            }
            if constexpr (MODE == MODE_RESIDUAL) {
                const size_t id = (size_t)k * pl + c;
                if constexpr (std::is_same<P, PO>::value) {
                    P::st(out, id, r0);
                    P::st(out, id + 1, r1);
                } else {
                    PO::st(out, id, PO::from_f(P::to_f(r0)));
                    PO::st(out, id + 1, PO::from_f(P::to_f(r1)));
                }
            }
            if constexpr (STACK) {
                R i0v, i1v;
                if (percol && k >= k0 && k <= nz - 2) {
                    i0v = ci0;
                    i1v = ci1;
                } else if (percol) {
                    i0v = P::ld_plain(ringI, slot * FPL + 2 * tid);
                    i1v = P::ld_plain(ringI, slot * FPL + 2 * tid + 1);
                } else {
                    i0v = i1v = P::ld(L.finv, k);
                }
                dp0 = P::mul_u(P::fma_u(v0, dp0, r0), i0v);
                dp1 = P::mul_u(P::fma_u(v1, dp1, r1), i1v);
                R g0 = dp0, g1 = dp1;
                if constexpr (GFORM) {
                    // g_k = u_k + rho d'_k - w_k u_{k+1} (um*, uc* now hold u_k, u_{k+1})
                    R w0, w1;
                    if (percol) {
                        w0 = P::mul(v0, i0v);
                        w1 = P::mul(v1, i1v);
                    } else {
                        w0 = w1 = P::ld(L.fw, k);
                    }
                    g0 = P::fma(P::neg(w0), uc0, P::fma(cf, dp0, um0));
                    g1 = P::fma(P::neg(w1), uc1, P::fma(cf, dp1, um1));
                }
                if constexpr ((HINT & HINT_KEEP) != 0) {
                    st_pair_pol(gstack + ((size_t)k * NT + tid) * 2, g0, g1, pol_last);
                } else {
                    P::sts(gstack, ((size_t)k * NT + tid) * 2, g0);
                    P::sts(gstack, ((size_t)k * NT + tid) * 2 + 1, g1);
                }
            }
            if (HALO) __syncthreads();  // the slot is reused by the next issue
            if constexpr (RESTR) {
                if (even) {
                    // f_c = 1/4 (even row pair + odd row pair), then the coarse forward elimination
                    const R fk = P::mul(xr->quarter, P::add(qv, P::ld_plain(xs, (k & 1) * 32 * CR + ci)));
                    P::st(xr->fc, (size_t)k * plc + cc, fk);
                    R ic;
                    if (xr->Lc.fac_percol && k >= xr->Lc.fac_k0 && k <= nz - 2)
                        ic = cic;
                    else if (xr->Lc.fac_percol)
                        ic = P::ld_plain(ringIc, slot * 32 * CR + ci);
                    else
                        ic = P::ld(xr->Lc.finv, k);
                    dpc = P::mul(P::fma(vcc, dpc, fk), ic);
                    P::sts(gstack, (size_t)k * 32 * CR + ci, dpc);
                }
            }
            issue_plane(k + PD, slot);
            slot = nslot;
        }
        cp_wait<0>();

        if constexpr (STACK) {
            // back substitution from the stacked values and v/m_k (and u_k unless GFORM)
            constexpr bool NEED_U = MODE == MODE_SMOOTH && !GFORM;
            __syncthreads();  // the backward ring reuses the forward ring's shared memory
            S* bW = reinterpret_cast<S*>(smem_raw);
            S* bD = bW + PD * 2 * NT;
            S* bU = bD + PD * 2 * NT;
            auto issue_back = [&](int k, int s2) {
                if (k >= 0) {
                    const size_t id = (size_t)k * pl + c;
                    const bool fac = percol && !(k >= k0 && k <= nz - 2);
                    if constexpr ((HINT & HINT_STREAM) != 0) {
                        if (NEED_U) cp_async_pol<PB>(&bU[(s2 * NT + tid) * 2], u + id, pol_first);
                        if (fac) cp_async_pol<PB>(&bW[(s2 * NT + tid) * 2], L.fw + id, pol_first);
                    } else {
                        if (NEED_U) cp_async<PB>(&bU[(s2 * NT + tid) * 2], u + id);
                        if (fac) cp_async<PB>(&bW[(s2 * NT + tid) * 2], L.fw + id);
                    }
                    cp_async<PB>(&bD[(s2 * NT + tid) * 2], gstack + ((size_t)k * NT + tid) * 2);
                }
                cp_commit();
            };
            for (int s = 0; s < PD; ++s) issue_back(nz - 1 - s, s);
            R x0 = vzero, x1 = vzero;
            slot = 0;
            for (int k = nz - 1; k >= 0; --k) {
                cp_wait<PD - 1>();
                if constexpr ((HINT & HINT_DISCARD) != 0) {
                    // plane k of the stack has landed for every lane of the warp: its lines are dead
                    constexpr int LANES_PER_LINE = 128 / PB;
                    __syncwarp();
                    if (tid % LANES_PER_LINE == 0) l2_discard(gstack + ((size_t)k * NT + tid) * 2);
                }
                const int o = (slot * NT + tid) * 2;
                R w0, w1;
                if (percol && k >= k0 && k <= nz - 2) {
                    w0 = cw0;
                    w1 = cw1;
                } else if (percol) {
                    w0 = P::ld_plain(bW, o);
                    w1 = P::ld_plain(bW, o + 1);
                } else {
                    w0 = w1 = P::ld(L.fw, k);
                }
                x0 = P::fma_u(w0, x0, P::ld_plain(bD, o));  // the recurrence carries unnormalised pairs
                x1 = P::fma_u(w1, x1, P::ld_plain(bD, o + 1));
                const size_t id = (size_t)k * pl + c;
                if constexpr (MODE == MODE_SMOOTH) {
                    R o0 = x0, o1 = x1;  // GFORM: the recurrence already yields u'
                    if constexpr (NEED_U) {
                        o0 = P::fma(cf, x0, P::ld_plain(bU, o));  // u' = u + rho x
                        o1 = P::fma(cf, x1, P::ld_plain(bU, o + 1));
                    }
                    if constexpr ((HINT & HINT_STREAM) != 0) {
                        st_pair_pol(reinterpret_cast<S*>(out) + id, P::rnd(o0), P::rnd(o1), pol_first);
                    } else {
                        P::st(reinterpret_cast<S*>(out), id, o0);
                        P::st(reinterpret_cast<S*>(out), id + 1, o1);
                    }
                } else {
                    // the product also renormalises the pair the recurrence carried
                    P::st(reinterpret_cast<S*>(out), id, P::mul(cf, x0));
                    P::st(reinterpret_cast<S*>(out), id + 1, P::mul(cf, x1));
                }
                issue_back(k - PD, slot);
                slot = (slot + 1 == PD) ? 0 : slot + 1;
            }
            cp_wait<0>();
        }
        if constexpr (RESTR) {
            // coarse back substitution by the even rows: u_c = rho x, x_k = d'_k + (v/m_k) x_{k+1}
            __syncthreads();  // the backward ring reuses the forward ring's shared memory
            if (even) {
                S* bW = reinterpret_cast<S*>(smem_raw);
                S* bD = bW + PD * 32 * CR;
                const bool pcc = xr->Lc.fac_percol != 0;
                const int kc0 = xr->Lc.fac_k0;
                auto issue_back = [&](int k, int s2) {
                    if (k >= 0) {
                        if (pcc && !(k >= kc0 && k <= nz - 2))
                            cp_async<sizeof(S)>(&bW[s2 * 32 * CR + ci], xr->Lc.fw + (size_t)k * plc + cc);
                        cp_async<sizeof(S)>(&bD[s2 * 32 * CR + ci], gstack + (size_t)k * 32 * CR + ci);
                    }
                    cp_commit();
                };
                for (int s = 0; s < PD; ++s) issue_back(nz - 1 - s, s);
                const R rho = xr->rho;
                R xn = vzero;
                slot = 0;
                for (int k = nz - 1; k >= 0; --k) {
                    cp_wait<PD - 1>();
                    R w;
                    if (pcc && k >= kc0 && k <= nz - 2)
                        w = cwc;
                    else if (pcc)
                        w = P::ld_plain(bW, slot * 32 * CR + ci);
                    else
                        w = P::ld(xr->Lc.fw, k);
                    xn = P::fma(w, xn, P::ld_plain(bD, slot * 32 * CR + ci));
                    P::st(xr->uc, (size_t)k * plc + cc, P::mul(rho, xn));
                    issue_back(k - PD, slot);
                    slot = (slot + 1 == PD) ? 0 : slot + 1;
                }
                cp_wait<0>();
            }
        }
    }
    return want_norm ? block_sum(P::acc_get(acc, cmp)) : 0.0;  // the block's sum, valid in thread 0
}


template <class P, int TY, int PD, int MODE>
constexpr size_t sweep_x2_smem() {
    constexpr bool STACK = x2_stack(MODE);
    constexpr bool HALO = MODE != MODE_LINESOLVE;
    constexpr size_t fwd = ((size_t)PD * ((HALO ? (TY + 2) * 68 : 0) + 2 * 32 * TY + (STACK ? 2 * 32 * TY : 0)) +
                            (MODE == MODE_RESTRICT ? (size_t)(PD + 2) * 32 * (TY / 2) : 0)) *
                           sizeof(typename P::S);
    constexpr size_t back = STACK ? (size_t)PD * 3 * 2 * 32 * TY * sizeof(typename P::S)
                                  : (MODE == MODE_RESTRICT ? (size_t)PD * 2 * 32 * (TY / 2) * sizeof(typename P::S) : 0);
    return fwd > back ? fwd : back;
}

}  // namespace tpmg
