// k_sweep.cu -- plane-pipelined column sweeps for the large levels (Smooth, Residual, line solve,
// RestrictSmooth), the Thomas factors, and the tile variants the autotuner chooses from.
//
// A block owns 32 x TY vertical columns (one thread each, 32 consecutive x per warp). It walks the
// planes k = 0..nz-1 of its tile; each plane of its inputs -- u with its one-cell periodic halo in
// x and y when a stencil is applied, f or the right-hand side, and, when lambda^2 varies over the
// level, the Thomas factor 1/m_k -- is fetched with cp.async into a ring of PD shared-memory slots,
// PD planes ahead of the computation, so many planes' loads are in flight while the recurrence of
// the current plane runs. The forward-eliminated values d'_k go to a per-thread stack in shared
// memory; the back substitution streams u_k and v/m_k through the ring in reverse order and writes
// each output value once.
//
// Per cell the kernels move the algorithmic minimum of their operation plus the factor arrays when
// lambda^2 varies over the level (constant lambda^2: one table of nz factors, read through L1).
#include <type_traits>

#include "kernels.cuh"
#include "sweep_x2.cuh"
#include "tpmg.h"

namespace tpmg {

__device__ __forceinline__ int wrap_p(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------- Thomas factors
template <class P>
__global__ void k_factors(Lv<P> L, typename P::S* __restrict__ finv, typename P::S* __restrict__ fw,
                          int percol) {
    typedef typename P::R R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (percol ? (i >= L.nx || j >= L.ny) : (i != 0 || j != 0)) return;
    const size_t pl = (size_t)L.nx * L.ny, c = (size_t)j * L.nx + i;
    const R vv = P::ld(L.v, c), vv2 = P::mul(vv, vv);
    const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
    R inv_prev = P::zero();
    for (int k = 0; k < L.nz; ++k) {
        R diag = (L.nz == 1) ? dh : ((k == 0 || k == L.nz - 1) ? dh1 : dh2);
        R m;
        if constexpr (P::id == 1)  // FP32: one rounding, as the four-column sweep forms it in registers
            m = (k == 0) ? diag : fmaf(-vv2, inv_prev, diag);
        else
            m = (k == 0) ? diag : P::sub(diag, P::mul(vv2, inv_prev));
        R inv = P::rcp(m);
        const size_t id = percol ? (size_t)k * pl + c : (size_t)k;
        P::st(finv, id, inv);
        P::st(fw, id, P::mul(vv, inv));
        inv_prev = inv;
    }
}

template <class P>
void launch_factors(const Lv<P>& L, typename P::S* finv, typename P::S* fw, int percol, cudaStream_t s) {
    dim3 blk(32, 4), grd((L.nx + 31) / 32, (L.ny + 3) / 4);
    if (!percol) grd = dim3(1, 1);
    k_factors<P><<<grd, blk, 0, s>>>(L, finv, fw, percol);
    note_launch();
}

// per column: the first plane k0 such that the stored factors of planes k0 .. nz-2 all equal (bit
// for bit) those of plane nz-2; *k0 = the maximum over the columns
template <class P>
__global__ void k_factor_k0(Lv<P> L, const typename P::S* __restrict__ finv, const typename P::S* __restrict__ fw,
                            int* k0) {
    typedef typename P::S S;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= L.nx || j >= L.ny || L.nz < 3) return;
    const size_t pl = (size_t)L.nx * L.ny, c = (size_t)j * L.nx + i;
    const int ref = L.nz - 2;
    const S ri = finv[(size_t)ref * pl + c], rw = fw[(size_t)ref * pl + c];
    auto same = [](const S& a, const S& b) {
        static_assert(sizeof(S) % 4 == 0, "32-bit words");
        const unsigned* x = reinterpret_cast<const unsigned*>(&a);
        const unsigned* y = reinterpret_cast<const unsigned*>(&b);
        for (int q = 0; q < (int)(sizeof(S) / 4); ++q)
            if (x[q] != y[q]) return false;
        return true;
    };
    int k = ref;
    while (k > 0 && same(finv[(size_t)(k - 1) * pl + c], ri) && same(fw[(size_t)(k - 1) * pl + c], rw)) --k;
    atomicMax(k0, k);
}

template <class P>
void launch_factor_k0(const Lv<P>& L, const typename P::S* finv, const typename P::S* fw, int* k0, cudaStream_t s) {
    dim3 blk(32, 4), grd((L.nx + 31) / 32, (L.ny + 3) / 4);
    k_factor_k0<P><<<grd, blk, 0, s>>>(L, finv, fw, k0);
    note_launch();
}

// ---------------------------------------------------------------- generic pipelined sweep

// MODE_SMOOTH:    out = u + coef M^{-1}(f - A u), partial sums of ||f - A u||^2      (Eq. 11)
// MODE_RESIDUAL:  out = f - A u (stored in PO's precision), partial sums of ||f - A u||^2
// MODE_LINESOLVE: out = coef M^{-1} u (u is the right-hand side; f unused)            (Eq. 9)
//
// GS = false: one tile per block, the forward-eliminated values d'_k on a shared-memory stack
// (nz values per thread: shared memory, not registers, then limits the SM to a few warps).
// GS = true: the stack lives in a global scratch of gridDim.x * nz * NT values that the blocks
// reuse tile after tile (a persistent loop over the tiles with a grid of a few blocks per SM), so
// the scratch stays resident in L2 and shared memory holds only the rings; d'_k is written with
// plain stores in the forward sweep and streamed back through the backward ring.
template <class P, class PO, int TY, int PD, int MODE, bool GS>
__global__ void __launch_bounds__(32 * TY) k_sweep_pp(Lv<P> L, SweepK<P> K, const typename P::S* __restrict__ u,
                                                      const typename P::S* __restrict__ f,
                                                      typename PO::S* __restrict__ out, double* partials,
                                                      const int* done) {
    typedef typename P::S S;
    typedef typename P::R R;
    constexpr int NT = 32 * TY;
    constexpr bool HALO = MODE != MODE_LINESOLVE;  // the stencil needs the u plane with its halo
    constexpr bool STACK = MODE != MODE_RESIDUAL;  // a Thomas solve follows
    constexpr int UPL = HALO ? (TY + 2) * 34 : 0;
    constexpr int FPL = NT;
    // FP32 Smooth stacks g_k = u_k + rho d'_k - w_k u_{k+1} and back-substitutes u'_k = g_k + w_k
    // u'_{k+1} (u'_k - u_k = rho x_k, x_k = d'_k + w_k x_{k+1}), so u is not read a second time;
    // the double-word and FP64 sweeps, bound by their arithmetic, stack d'_k and re-read u instead
    constexpr bool GFORM = MODE == MODE_SMOOTH && P::id == 1;
    constexpr int IPL = STACK ? NT : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;

    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const bool percol = L.fac_percol != 0;
    S* ringU = reinterpret_cast<S*>(smem_raw);
    S* ringF = ringU + PD * UPL;
    S* ringI = ringF + PD * FPL;
    const size_t ring_bytes = ((size_t)PD * (UPL + FPL + IPL) * sizeof(S) + 15) & ~(size_t)15;
    R* stack = reinterpret_cast<R*>(smem_raw + ring_bytes);
    S* gstack = GS ? reinterpret_cast<S*>(L.gstack) + (size_t)blockIdx.x * nz * NT : nullptr;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const size_t pl = (size_t)nx * ny;
    const int tiles_x = nx / 32;
    const int ntiles = GS ? tiles_x * (ny / TY) : 1;
    const S* rhs = (MODE == MODE_LINESOLVE) ? u : f;
    const R vzero = P::zero();
    typename P::Acc acc = 0, cmp = 0;

    for (int tile = GS ? blockIdx.x : 0; tile < ntiles; tile += GS ? gridDim.x : 1) {
        const int i0 = GS ? (tile % tiles_x) * 32 : blockIdx.x * 32;
        const int j0 = GS ? (tile / tiles_x) * TY : blockIdx.y * TY;
        const size_t c = (size_t)(j0 + ty) * nx + (i0 + tx);
        if (GS) __syncthreads();  // the previous tile's backward ring is no longer read

        // halo of the u plane: rows j0-1 and j0+TY (32 each), columns i0-1 and i0+32 (TY+2 each);
        // thread tid fetches items tid, tid + NT, ...: their ring offsets and in-plane sources are
        // the same for every plane, so they are computed once per tile
        constexpr int NHALO = 64 + 2 * (TY + 2);
        constexpr int HPT = (NHALO + NT - 1) / NT;
        int h_dst[HPT];
        size_t h_src[HPT];
        if constexpr (HALO) {
#pragma unroll
            for (int q = 0; q < HPT; ++q) {
                const int it = tid + q * NT;
                int rr = 0, cc = 0, gj = j0, gi = i0;
                if (it < 64) {
                    rr = (it < 32) ? 0 : TY + 1;
                    cc = (it & 31) + 1;
                    gj = (it < 32) ? j0 - 1 : j0 + TY;
                    gi = i0 + (it & 31);
                } else if (it < NHALO) {
                    const int e = it - 64;
                    rr = e >> 1;
                    cc = (e & 1) ? 33 : 0;
                    gj = j0 - 1 + rr;
                    gi = (e & 1) ? i0 + 32 : i0 - 1;
                }
                h_dst[q] = it < NHALO ? rr * 34 + cc : -1;
                h_src[q] = (size_t)wrap_p(gj, ny) * nx + wrap_p(gi, nx);
            }
        }

        auto issue_plane = [&](int k, int slot) {
            if (k < nz) {
                const size_t b = (size_t)k * pl;
                cp_async<sizeof(S)>(&ringF[slot * FPL + tid], rhs + b + c);
                if (STACK && percol) cp_async<sizeof(S)>(&ringI[slot * FPL + tid], L.finv + b + c);
                if (HALO) {
                    S* Us = ringU + slot * UPL;
                    cp_async<sizeof(S)>(&Us[(ty + 1) * 34 + tx + 1], u + b + c);
#pragma unroll
                    for (int q = 0; q < HPT; ++q)
                        if (h_dst[q] >= 0) cp_async<sizeof(S)>(&Us[h_dst[q]], u + b + h_src[q]);
                }
            }
            cp_commit();
        };

        for (int s = 0; s < PD; ++s) issue_plane(s, s);

        const R vv = P::ld(L.v, c);
        const R cx = K.cx, cy = K.cy, dh = K.dh;
        const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        const bool iso = K.iso != 0;  // square cells: one product for the four horizontal neighbours
        const bool want_norm = partials != nullptr;
        const R cf = K.coef;
        R um = vzero, uc = vzero, d_prev = vzero;
        int slot = 0;
        const int ctr = (ty + 1) * 34 + tx + 1;
        for (int k = 0; k < nz; ++k) {
            const int nslot = (slot + 1 == PD) ? 0 : slot + 1;
            R r;
            if constexpr (HALO) {
                cp_wait<PD - 2>();  // planes k and k+1 (the upper neighbour) have landed
                __syncthreads();    // ... including the halo values other threads fetched
                const S* Us = ringU + slot * UPL;
                if (k == 0) uc = P::ld_plain(Us, ctr);
                const R up = (k + 1 < nz) ? P::ld_plain(ringU + nslot * UPL, ctr) : vzero;
                const R diag = (nz == 1) ? dh : ((k == 0 || k == nz - 1) ? dh1 : dh2);
                r = sweep_residual<P>(P::ld_plain(ringF, slot * FPL + tid), diag, uc, P::ld_plain(Us, ctr - 1),
                                      P::ld_plain(Us, ctr + 1), P::ld_plain(Us, ctr - 34), P::ld_plain(Us, ctr + 34),
                                      um, up, cx, cy, vv, iso);
                if (want_norm) P::acc_dot(acc, cmp, r, r);
                um = uc;
                uc = up;
            } else {
                cp_wait<PD - 1>();  // only this thread's own copies are read: no barrier needed
                r = P::ld_plain(ringF, slot * FPL + tid);
            }
            if constexpr (MODE == MODE_RESIDUAL) {
                const size_t id = (size_t)k * pl + c;
                if constexpr (std::is_same<P, PO>::value)
                    P::st(out, id, r);
                else
                    PO::st(out, id, PO::from_f(P::to_f(r)));
            }
            if constexpr (STACK) {
                const R inv = percol ? P::ld_plain(ringI, slot * FPL + tid) : P::ld(L.finv, k);
                const R d = P::mul_u(P::fma_u(vv, d_prev, r), inv);
                R g = d;
                if constexpr (GFORM) {
                    // g_k = u_k + rho d'_k - w_k u_{k+1} (um, uc now hold u_k, u_{k+1})
                    const R w = percol ? P::mul(vv, inv) : P::ld(L.fw, k);
                    g = P::fma(P::neg(w), uc, P::fma(cf, d, um));
                }
                if constexpr (GS)
                    P::sts(gstack, (size_t)k * NT + tid, g);
                else
                    stack[(size_t)k * NT + tid] = g;
                d_prev = d;
            }
            if constexpr (HALO) __syncthreads();  // the slot is reused by the next issue
            issue_plane(k + PD, slot);
            slot = nslot;
        }
        cp_wait<0>();

        if constexpr (STACK) {
            __syncthreads();  // the backward ring reuses the forward ring's shared memory
            // back substitution, streaming v/m_k, (GS) the stacked values and (Smooth, unless
            // GFORM) u_k through the ring in reverse order; every thread reads only its own copies
            constexpr bool NEED_U = MODE == MODE_SMOOTH && !GFORM;
            S* bW = reinterpret_cast<S*>(smem_raw);
            S* bD = bW + PD * NT;
            S* bU = bD + PD * NT;
            auto issue_back = [&](int k, int s2) {
                if (k >= 0) {
                    const size_t id = (size_t)k * pl + c;
                    if (NEED_U) cp_async<sizeof(S)>(&bU[s2 * NT + tid], u + id);
                    if (percol) cp_async<sizeof(S)>(&bW[s2 * NT + tid], L.fw + id);
                    if (GS) cp_async<sizeof(S)>(&bD[s2 * NT + tid], gstack + (size_t)k * NT + tid);
                }
                cp_commit();
            };
            for (int s = 0; s < PD; ++s) issue_back(nz - 1 - s, s);
            R xn = vzero;
            slot = 0;
            for (int k = nz - 1; k >= 0; --k) {
                cp_wait<PD - 1>();
                const R w = percol ? P::ld_plain(bW, slot * NT + tid) : P::ld(L.fw, k);
                const R dk = GS ? P::ld_plain(bD, slot * NT + tid) : stack[(size_t)k * NT + tid];
                xn = P::fma_u(w, xn, dk);  // the recurrence carries unnormalised pairs
                const size_t id = (size_t)k * pl + c;
                if constexpr (GFORM)
                    P::st(reinterpret_cast<S*>(out), id, xn);
                else if constexpr (MODE == MODE_SMOOTH)
                    P::st(reinterpret_cast<S*>(out), id, P::fma(cf, xn, P::ld_plain(bU, slot * NT + tid)));
                else
                    P::st(reinterpret_cast<S*>(out), id, P::mul(cf, xn));  // also renormalises the pair
                issue_back(k - PD, slot);
                slot = (slot + 1 == PD) ? 0 : slot + 1;
            }
            cp_wait<0>();
        }
    }
    if (MODE != MODE_LINESOLVE && partials) {
        double sm = block_sum(P::acc_get(acc, cmp));
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = sm;
    }
}

template <class P, int TY, int PD, int MODE, bool GS = false>
static size_t sweep_pp_smem(int nz) {
    typedef typename P::S S;
    const int UPL = MODE != MODE_LINESOLVE ? (TY + 2) * 34 : 0;
    const int IPL = MODE != MODE_RESIDUAL ? 32 * TY : 0;
    const size_t ring = ((size_t)PD * (UPL + 32 * TY + IPL) * sizeof(S) + 15) & ~(size_t)15;
    const size_t stack = (MODE != MODE_RESIDUAL && !GS) ? (size_t)nz * 32 * TY * sizeof(typename P::R) : 0;
    // the backward ring (u, v/m and, GS, the stacked values) reuses the forward ring: take the larger
    const size_t back = (size_t)PD * 32 * TY * sizeof(S) * 3;
    return (GS && back > ring ? back : ring) + stack;
}

template <class P, int TY, bool FACTORS = true>
static bool pp_fits(const Lv<P>& L) {
    return L.nx % 32 == 0 && L.ny % TY == 0 && L.nx >= 32 && (!FACTORS || (L.finv && L.fw));
}

static int g_num_sms = 0;
static int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

size_t gstack_bytes(int nz) { return (size_t)num_sms() * GS_BLOCKS_PER_SM * GS_MAX_NT * nz * 8; }

template <class P, class PO, int TY, int PD, int MODE, bool GS = false>
static int run_sweep_pp(const Lv<P>& L, double coef, const typename P::S* u, const typename P::S* f,
                        typename PO::S* out, double* partials, const int* done, cudaStream_t s,
                        int cap = GS_BLOCKS_PER_SM) {
    static_assert(!GS || 32 * TY <= GS_MAX_NT, "persistent variants own GS_MAX_NT-thread stack slots");
    const size_t smem = sweep_pp_smem<P, TY, PD, MODE, GS>(L.nz);
    auto kern = k_sweep_pp<P, PO, TY, PD, MODE, GS>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grd(L.nx / 32, L.ny / TY), blk(32, TY);
    if (GS) {
        // persistent: at most GS_BLOCKS_PER_SM resident blocks per SM, each owning a stack slot
        const int ntiles = (L.nx / 32) * (L.ny / TY);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * TY, smem);
        if (cap > GS_BLOCKS_PER_SM) cap = GS_BLOCKS_PER_SM;
        if (per_sm > cap) per_sm = cap;
        if (per_sm < 1) per_sm = 1;
        int nb = num_sms() * per_sm;
        if (nb > ntiles) nb = ntiles;
        grd = dim3(nb, 1);
    }
    kern<<<grd, blk, smem, s>>>(L, sweep_k<P>(L.cx, L.cy, coef), u, f, out, partials, done);
    note_launch();
    return (int)(grd.x * grd.y);
}

// ---------------------------------------------------------------- two columns per thread
// The body is sweep_x2_tiles (sweep_x2.cuh), shared with the batched persistent kernel.
template <class P, class PO, int TY, int PD, int MODE, int MINB = 1, int HINT = 0>
__global__ void __launch_bounds__(32 * TY, MINB) k_sweep_x2(Lv<P> L, SweepK<P> K, const typename P::S* __restrict__ u,
                                                      const typename P::S* __restrict__ f,
                                                      typename PO::S* __restrict__ out, double* partials,
                                                      const int* done) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    typename P::S* slot = x2_slot(MODE)
                              ? reinterpret_cast<typename P::S*>(L.gstack) + (size_t)blockIdx.x * L.nz * 2 * 32 * TY
                              : nullptr;
    const int ntiles = (L.nx / 64) * (L.ny / TY);
    const double sm = sweep_x2_tiles<P, PO, TY, PD, MODE, HINT>(L, K, u, f, out, partials != nullptr, blockIdx.x,
                                                                 ntiles, gridDim.x, slot, smem_raw);
    if (partials && threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.x] = sm;
}

// Grid (number of persistent blocks) of the two-column sweep on level L with these fields, or -1
// where the level or the fields do not take it. run_sweep_x2 launches exactly this many blocks, and
// residual_launch_blocks reports it without launching.
template <class P, class PO, int TY, int PD, int MODE, int MINB = 1, int HINT = 0>
static int sweep_x2_grid(const Lv<P>& L, const void* u, const void* f, const void* out, int cap) {
    constexpr bool STACK = x2_stack(MODE);
    constexpr bool HALO = MODE != MODE_LINESOLVE;
    if (L.nx % 64 || L.ny % TY || (STACK && (!L.gstack || !L.finv || !L.fw))) return -1;
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    if (!al(u) || (HALO && MODE != MODE_APPLY && !al(f)) || !al(out) || (STACK && (!al(L.finv) || !al(L.fw))))
        return -1;
    const size_t smem = sweep_x2_smem<P, TY, PD, MODE>();
    auto kern = k_sweep_x2<P, PO, TY, PD, MODE, MINB, HINT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int ntiles = (L.nx / 64) * (L.ny / TY);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * TY, smem);
    if (cap > GS_BLOCKS_PER_SM) cap = GS_BLOCKS_PER_SM;
    if (per_sm > cap) per_sm = cap;
    if (per_sm < 1) per_sm = 1;
    int nb = num_sms() * per_sm;
    // the stack slots: 2 * 32 * TY columns per block out of gstack_bytes
    const int slots = num_sms() * GS_BLOCKS_PER_SM * GS_MAX_NT / (2 * 32 * TY);
    if (STACK && nb > slots) nb = slots;
    if (nb > ntiles) nb = ntiles;
    return nb;
}

template <class P, class PO, int TY, int PD, int MODE, int MINB = 1, int HINT = 0>
static int run_sweep_x2(const Lv<P>& L, double coef, const typename P::S* u, const typename P::S* f,
                        typename PO::S* out, double* partials, const int* done, cudaStream_t s, int cap) {
    const int nb = sweep_x2_grid<P, PO, TY, PD, MODE, MINB, HINT>(L, u, f, out, cap);
    if (nb < 0) return -1;
    const size_t smem = sweep_x2_smem<P, TY, PD, MODE>();
    k_sweep_x2<P, PO, TY, PD, MODE, MINB, HINT><<<nb, dim3(32, TY), smem, s>>>(L, sweep_k<P>(L.cx, L.cy, coef), u, f,
                                                                             out, partials, done);
    note_launch();
    return nb;
}

// ---------------------------------------------------------------- Residual + RestrictSmooth, fused
// One pass over the fine level L: r = f - A u per fine cell (not stored), f_c = R r and
// u_c = rho M_c^{-1} f_c on the coarse level Lc (sweep_x2_tiles in MODE_RESTRICT). Per fine cell it
// reads u and f once; per coarse cell it writes f_c and u_c -- 2.5 instead of 4.5 memory references
// per fine cell for the two kernels. The arithmetic is that of the separate kernels, operation for
// operation, so the results are the same bit for bit.
template <class P, int PD>
__global__ void __launch_bounds__(64) k_residual_restrict_x2(Lv<P> L, SweepK<P> K, XRestrict<P> xr,
                                                               const typename P::S* __restrict__ u,
                                                               const typename P::S* __restrict__ f, const int* done) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    typename P::S* slot = reinterpret_cast<typename P::S*>(L.gstack) + (size_t)blockIdx.x * L.nz * 2 * 32 * 2;
    const int ntiles = (L.nx / 64) * (L.ny / 2);
    sweep_x2_tiles<P, P, 2, PD, MODE_RESTRICT, 0>(L, K, u, f, nullptr, false, blockIdx.x, ntiles, gridDim.x, slot,
                                                 smem_raw, &xr);
}

template <class P>
int launch_residual_restrict(const Lv<P>& L, const Lv<P>& Lc, double rho, const typename P::S* u,
                             const typename P::S* f, typename P::S* fc, typename P::S* uc, const int* done,
                             cudaStream_t s) {
    constexpr int PD = 4;
    if (L.nx % 64 || L.ny % 2 || !L.gstack || !Lc.finv || !Lc.fw || !Lc.v) return -1;
    if (Lc.nx * 2 != L.nx || Lc.ny * 2 != L.ny || Lc.nz != L.nz) return -1;
    // small coarse levels solve their columns by cyclic reduction (k_coarse.cu)
    if (Lc.pcr && (size_t)Lc.nx * Lc.ny <= (size_t)PCR_MAX_COLS && Lc.nz <= 256) return -1;
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    if (!al(u) || !al(f)) return -1;
    const size_t smem = sweep_x2_smem<P, 2, PD, MODE_RESTRICT>();
    auto kern = k_residual_restrict_x2<P, PD>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int ntiles = (L.nx / 64) * (L.ny / 2);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64, smem);
    if (per_sm > GS_BLOCKS_PER_SM) per_sm = GS_BLOCKS_PER_SM;
    if (per_sm < 1) per_sm = 1;
    int nb = num_sms() * per_sm;
    const int slots = num_sms() * GS_BLOCKS_PER_SM * GS_MAX_NT / (2 * 32 * 2);
    if (nb > slots) nb = slots;
    if (nb > ntiles) nb = ntiles;
    XRestrict<P> xr{Lc, P::hcst(rho), P::hcst(0.25), fc, uc};
    kern<<<nb, dim3(32, 2), smem, s>>>(L, sweep_k<P>(L.cx, L.cy, 1.0), xr, u, f, done);
    note_launch();
    return nb;
}

// ---------------------------------------------------------------- tile variants
// Smooth: eight variants per precision -- three (TY, PD) tile shapes with the shared-memory stack
// (0-2), two persistent ones with the stack in global scratch (3, 4), and three persistent ones with
// two columns per thread and L2 eviction hints (k_sweep_x2; 5-7); the autotuner (tpmg_autotune)
// times them per level and stores its choice in Lv::variant. An untuned level takes variant 6
// (double-word) or 5 (FP32) where the two-column form applies (nx % 64 == 0, aligned fields), else
// variant 3; in native FP64, variant 0.
template <class P>
struct SmoothVariants;
template <>
struct SmoothVariants<PolF32> {
    static constexpr int TY[3] = {2, 4, 1};
};
template <>
struct SmoothVariants<PolF64> {
    static constexpr int TY[3] = {1, 2, 2};
};
template <>
struct SmoothVariants<PolDW> {
    static constexpr int TY[3] = {1, 2, 2};
};

template <class P>
static int smooth_dispatch(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                           typename P::S* uo, double* partials, const int* done, cudaStream_t s) {
    int v = L.variant;
    if constexpr (std::is_same<P, PolF32>::value) {  // one tile of 128 x 2 columns per warp where the level takes it
        if ((v < 0 || v >= TPMG_NUM_VARIANTS || v >= 8) && L.gstack) {
            const int nb = launch_smooth_x4(L, rho, u, f, uo, partials, done, s, v >= 8 && v < TPMG_NUM_VARIANTS ? v - 8 : 0);
            if (nb >= 0) return nb;
        }
    }
    if (v < 0 || v >= TPMG_NUM_VARIANTS || v >= 8) {
        v = 0;
        if (L.gstack && P::id != 0) {  // native FP64 is bound by its slow pipe: one column per thread
            const int nb = P::id == 1
                               ? run_sweep_x2<P, P, 2, 4, MODE_SMOOTH, 1, HINT_ALL>(L, rho, u, f, uo, partials, done, s, 8)
                               : run_sweep_x2<P, P, 2, 4, MODE_SMOOTH, 10, HINT_ALL>(L, rho, u, f, uo, partials, done, s, 12);
            if (nb >= 0) return nb;
            v = 3;
        }
    }
    if (v >= 5 && L.gstack) {
        int nb = -1;
        if (v == 5) nb = run_sweep_x2<P, P, 2, 4, MODE_SMOOTH, 1, HINT_ALL>(L, rho, u, f, uo, partials, done, s, 8);
        if (v == 6) nb = run_sweep_x2<P, P, 2, 4, MODE_SMOOTH, 10, HINT_ALL>(L, rho, u, f, uo, partials, done, s, 12);
        if (v == 7) nb = run_sweep_x2<P, P, 2, 6, MODE_SMOOTH, 10, HINT_ALL>(L, rho, u, f, uo, partials, done, s, 12);
        if (nb >= 0) return nb;
    }
    if (P::id == 1) {  // FP32
        if (v == 0 && pp_fits<P, 2>(L)) return run_sweep_pp<P, P, 2, 8, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
        if (v == 1 && pp_fits<P, 4>(L)) return run_sweep_pp<P, P, 4, 6, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
        if (v == 2 && pp_fits<P, 1>(L)) return run_sweep_pp<P, P, 1, 8, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
        if (L.gstack && v == 3 && pp_fits<P, 2>(L))
            return run_sweep_pp<P, P, 2, 8, MODE_SMOOTH, true>(L, rho, u, f, uo, partials, done, s, 8);
        if (L.gstack && v == 4 && pp_fits<P, 2>(L))
            return run_sweep_pp<P, P, 2, 8, MODE_SMOOTH, true>(L, rho, u, f, uo, partials, done, s, 16);
        if (pp_fits<P, 2>(L)) return run_sweep_pp<P, P, 2, 8, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
    } else {  // 8-byte values
        if (v == 1 && pp_fits<P, 2>(L)) return run_sweep_pp<P, P, 2, 4, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
        if (v == 2 && pp_fits<P, 2>(L)) return run_sweep_pp<P, P, 2, 6, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
        if (L.gstack && v == 3 && pp_fits<P, 2>(L))
            return run_sweep_pp<P, P, 2, 4, MODE_SMOOTH, true>(L, rho, u, f, uo, partials, done, s, 8);
        if (L.gstack && v == 4 && pp_fits<P, 2>(L))
            return run_sweep_pp<P, P, 2, 4, MODE_SMOOTH, true>(L, rho, u, f, uo, partials, done, s, 16);
        if (pp_fits<P, 1>(L)) return run_sweep_pp<P, P, 1, 6, MODE_SMOOTH>(L, rho, u, f, uo, partials, done, s);
    }
    return -1;
}

template <class P>
int launch_smooth_pp(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                     typename P::S* uo, double* partials, const int* done, cudaStream_t s) {
    if (L.nz * 32 * 8 > 160 * 1024) return -1;  // stack too deep for shared memory
    return smooth_dispatch<P>(L, rho, u, f, uo, partials, done, s);
}

template <class P, class PO>
int launch_residual_pp(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r,
                       double* partials, const int* done, cudaStream_t s) {
    // two columns per thread when the level allows it (nx % 64 == 0, 16-byte aligned fields)
    const int nb = run_sweep_x2<P, PO, 2, 4, MODE_RESIDUAL>(L, 1.0, u, f, r, partials, done, s, 16);
    if (nb >= 0) return nb;
    if (!pp_fits<P, 4, false>(L)) return -1;
    return run_sweep_pp<P, PO, 4, 6, MODE_RESIDUAL>(L, 1.0, u, f, r, partials, done, s);
}

template <class P, class PO>
int residual_pp_blocks(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r) {
    // the same decisions as launch_residual_pp: the two-column grid, else the one-column pipelined
    // kernel's (nx / 32) x (ny / 4) blocks (run_sweep_pp without the persistent stack)
    const int nb = sweep_x2_grid<P, PO, 2, 4, MODE_RESIDUAL>(L, u, f, r, 16);
    if (nb >= 0) return nb;
    if (!pp_fits<P, 4, false>(L)) return -1;
    return (L.nx / 32) * (L.ny / 4);
}

template <class P>
int launch_apply_A_x2(const Lv<P>& L, const typename P::S* x, typename P::S* y, cudaStream_t s) {
    return run_sweep_x2<P, P, 2, 4, MODE_APPLY>(L, 1.0, x, nullptr, y, nullptr, nullptr, s, 16);
}

template <class P>
int launch_line_solve_pp(const Lv<P>& L, const typename P::S* b, typename P::S* x, double scale, const int* done,
                         cudaStream_t s) {
    if constexpr (std::is_same<P, PolF32>::value) {
        if (L.gstack) {
            const int nb = launch_line_solve_x4(L, b, x, scale, done, s);
            if (nb >= 0) return nb;
        }
    }
    // two columns per thread with the stack in the L2-steered scratch where the level allows it
    if (L.gstack && P::id != 0) {
        const int nb = run_sweep_x2<P, P, 2, 4, MODE_LINESOLVE, 1, HINT_ALL>(L, scale, b, nullptr, x, nullptr, done, s, 8);
        if (nb >= 0) return nb;
    }
    if (L.nz * 32 * 8 > 160 * 1024) return -1;
    if (P::id == 1) {
        if (!pp_fits<P, 2>(L)) return -1;
        return run_sweep_pp<P, P, 2, 8, MODE_LINESOLVE>(L, scale, b, nullptr, x, nullptr, done, s);
    }
    if (!pp_fits<P, 1>(L)) return -1;
    return run_sweep_pp<P, P, 1, 8, MODE_LINESOLVE>(L, scale, b, nullptr, x, nullptr, done, s);
}


// ---------------------------------------------------------------- RestrictSmooth, pipelined
// Coarse tile of 32 x TY columns; per coarse plane each thread fetches its 2 x 2 fine children
// (two contiguous pairs) and, when lambda^2 varies, 1/m_k; f_c = 1/4 (sum of the children) is
// written in the forward sweep, u_c = rho M_c^{-1} f_c in the backward sweep.
template <class PF, class P, int TY, int PD, bool GS>
__global__ void __launch_bounds__(32 * TY) k_restrict_smooth_pp(Lv<P> Lc, double rho_d,
                                                                const typename PF::S* __restrict__ rf,
                                                                typename P::S* __restrict__ fc,
                                                                typename P::S* __restrict__ uc, const int* done) {
    typedef typename PF::S SF;
    typedef typename P::S S;
    typedef typename P::R R;
    constexpr int NT = 32 * TY;
    constexpr int CPL = 4 * NT;  // fine children per coarse plane tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;
    const int nxc = Lc.nx, nyc = Lc.ny, nz = Lc.nz, nxf = 2 * nxc;
    const bool percol = Lc.fac_percol != 0;
    SF* ringC = reinterpret_cast<SF*>(smem_raw);
    S* ringI = reinterpret_cast<S*>(smem_raw + (size_t)PD * CPL * sizeof(SF));
    const size_t ring_bytes = (((size_t)PD * CPL * sizeof(SF) + (size_t)PD * NT * sizeof(S)) + 15) & ~(size_t)15;
    R* stack = reinterpret_cast<R*>(smem_raw + ring_bytes);
    S* gstack = GS ? reinterpret_cast<S*>(Lc.gstack) + (size_t)blockIdx.x * nz * NT : nullptr;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const size_t plc = (size_t)nxc * nyc, plf = 4 * plc;
    const int tiles_x = nxc / 32;
    const int ntiles = GS ? tiles_x * (nyc / TY) : 1;
    for (int tile = GS ? blockIdx.x : 0; tile < ntiles; tile += GS ? gridDim.x : 1) {
        const int I = (GS ? (tile % tiles_x) : blockIdx.x) * 32 + tx;
        const int J = (GS ? (tile / tiles_x) : blockIdx.y) * TY + ty;
        const size_t c = (size_t)J * nxc + I;
        const size_t f0 = (size_t)(2 * J) * nxf + 2 * I, f1 = f0 + nxf;
        if (GS) __syncthreads();  // the previous tile's backward ring is no longer read
        auto issue_plane = [&](int k, int slot) {
            if (k < nz) {
                const size_t bf = (size_t)k * plf;
                cp_async<2 * sizeof(SF)>(&ringC[slot * CPL + 4 * tid], rf + bf + f0);
                cp_async<2 * sizeof(SF)>(&ringC[slot * CPL + 4 * tid + 2], rf + bf + f1);
                if (percol) cp_async<sizeof(S)>(&ringI[slot * NT + tid], Lc.finv + (size_t)k * plc + c);
            }
            cp_commit();
        };
        for (int s = 0; s < PD; ++s) issue_plane(s, s);
        const R vv = P::ld(Lc.v, c), quarter = P::cst(0.25);
        R d_prev = P::zero();
        int slot = 0;
        for (int k = 0; k < nz; ++k) {
            cp_wait<PD - 1>();
            const SF* ch = ringC + slot * CPL + 4 * tid;
            R s4;
            if constexpr (std::is_same<PF, P>::value) {
                s4 = P::add(P::add(P::ld_plain(ch, 0), P::ld_plain(ch, 1)), P::add(P::ld_plain(ch, 2), P::ld_plain(ch, 3)));
            } else {
                auto cv = [&](int q) { return P::cst(PF::to_d(PF::ld_plain(ch, q))); };
                s4 = P::add(P::add(cv(0), cv(1)), P::add(cv(2), cv(3)));
            }
            const R fk = P::mul(quarter, s4);
            P::st(fc, (size_t)k * plc + c, fk);
            const R inv = percol ? P::ld_plain(ringI, slot * NT + tid) : P::ld(Lc.finv, k);
            const R d = P::mul(P::fma(vv, d_prev, fk), inv);
            if constexpr (GS)
                P::sts(gstack, (size_t)k * NT + tid, d);
            else
                stack[(size_t)k * NT + tid] = d;
            d_prev = d;
            issue_plane(k + PD, slot);
            slot = (slot + 1 == PD) ? 0 : slot + 1;
        }
        cp_wait<0>();
        // the backward ring reuses shared memory that other threads' forward slots occupied: wait
        // until every thread of the block has finished its forward sweep
        __syncthreads();
        // back substitution with v/m_k and (GS) d'_k streamed in reverse (each thread reads only
        // its own copies)
        S* bW = reinterpret_cast<S*>(smem_raw);
        S* bD = bW + PD * NT;
        auto issue_back = [&](int k, int s2) {
            if (k >= 0) {
                if (percol) cp_async<sizeof(S)>(&bW[s2 * NT + tid], Lc.fw + (size_t)k * plc + c);
                if (GS) cp_async<sizeof(S)>(&bD[s2 * NT + tid], gstack + (size_t)k * NT + tid);
            }
            cp_commit();
        };
        for (int s = 0; s < PD; ++s) issue_back(nz - 1 - s, s);
        const R rho = P::cst(rho_d);
        R xn = P::zero();
        slot = 0;
        for (int k = nz - 1; k >= 0; --k) {
            cp_wait<PD - 1>();
            const R w = percol ? P::ld_plain(bW, slot * NT + tid) : P::ld(Lc.fw, k);
            const R dk = GS ? P::ld_plain(bD, slot * NT + tid) : stack[(size_t)k * NT + tid];
            xn = P::fma(w, xn, dk);
            P::st(uc, (size_t)k * plc + c, P::mul(rho, xn));
            issue_back(k - PD, slot);
            slot = (slot + 1 == PD) ? 0 : slot + 1;
        }
        cp_wait<0>();
    }
}

template <class PF, class P>
int launch_restrict_smooth_pp(const Lv<P>& Lc, double rho, const typename PF::S* rf, typename P::S* fc,
                              typename P::S* uc, const int* done, cudaStream_t s) {
    constexpr int TY = (P::id == 1) ? 2 : 1;
    constexpr int PD = 6;
    if (!pp_fits<P, TY>(Lc) || Lc.nz * 32 * 8 > 160 * 1024) return -1;
    const size_t ring = (((size_t)PD * 4 * 32 * TY * sizeof(typename PF::S) + (size_t)PD * 32 * TY * sizeof(typename P::S)) + 15) & ~(size_t)15;
    if (Lc.gstack) {
        // persistent, the stack in global scratch (the backward ring of v/m and d' fits the ring)
        auto kern = k_restrict_smooth_pp<PF, P, TY, PD, true>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
        const int ntiles = (Lc.nx / 32) * (Lc.ny / TY);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * TY, ring);
        if (per_sm > GS_BLOCKS_PER_SM) per_sm = GS_BLOCKS_PER_SM;
        if (per_sm < 1) per_sm = 1;
        int nb = num_sms() * per_sm;
        if (nb > ntiles) nb = ntiles;
        kern<<<nb, dim3(32, TY), ring, s>>>(Lc, rho, rf, fc, uc, done);
        note_launch();
        return 1;
    }
    const size_t smem = ring + (size_t)Lc.nz * 32 * TY * sizeof(typename P::R);
    auto kern = k_restrict_smooth_pp<PF, P, TY, PD, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grd(Lc.nx / 32, Lc.ny / TY), blk(32, TY);
    kern<<<grd, blk, smem, s>>>(Lc, rho, rf, fc, uc, done);
    note_launch();
    return 1;
}

#define TPMG_SWEEP_INST(P)                                                                                  \
    template void launch_factors<P>(const Lv<P>&, P::S*, P::S*, int, cudaStream_t);                         \
    template void launch_factor_k0<P>(const Lv<P>&, const P::S*, const P::S*, int*, cudaStream_t);          \
    template int launch_smooth_pp<P>(const Lv<P>&, double, const P::S*, const P::S*, P::S*, double*, const int*, \
                                     cudaStream_t);                                                          \
    template int residual_pp_blocks<P, P>(const Lv<P>&, const P::S*, const P::S*, P::S*);                    \
    template int launch_residual_pp<P, P>(const Lv<P>&, const P::S*, const P::S*, P::S*, double*, const int*,  \
                                          cudaStream_t);                                                     \
    template int launch_line_solve_pp<P>(const Lv<P>&, const P::S*, P::S*, double, const int*, cudaStream_t); \
    template int launch_apply_A_x2<P>(const Lv<P>&, const P::S*, P::S*, cudaStream_t);                        \
    template int launch_restrict_smooth_pp<P, P>(const Lv<P>&, double, const P::S*, P::S*, P::S*, const int*, \
                                                 cudaStream_t);                                                \
    template int launch_residual_restrict<P>(const Lv<P>&, const Lv<P>&, double, const P::S*, const P::S*, P::S*, \
                                             P::S*, const int*, cudaStream_t);

TPMG_SWEEP_INST(PolF64)
TPMG_SWEEP_INST(PolF32)
TPMG_SWEEP_INST(PolDW)
TPMG_SWEEP_INST(PolF32B)
template int launch_restrict_smooth_pp<PolF32, PolF32B>(const Lv<PolF32B>&, double, const float*, float*, float*,
                                                        const int*, cudaStream_t);
template int launch_residual_pp<PolF64, PolF32>(const Lv<PolF64>&, const double*, const double*, float*, double*,
                                                const int*, cudaStream_t);
template int launch_residual_pp<PolDW, PolF32>(const Lv<PolDW>&, const float2*, const float2*, float*, double*,
                                               const int*, cudaStream_t);
template int launch_restrict_smooth_pp<PolDW, PolF64>(const Lv<PolF64>&, double, const float2*, double*, double*,
                                                      const int*, cudaStream_t);

}  // namespace tpmg
