// k_sweep.cu -- plane-pipelined column sweeps for the large levels, and the Thomas factors.
//
// A block owns 32 x TY vertical columns (one thread each, 32 consecutive x per warp). It walks the
// planes k = 0..nz-1 of its tile; each plane of u (with its one-cell periodic halo in x and y), of
// f and, when lambda^2 varies, of the factor 1/m_k is fetched with cp.async into a ring of PD
// shared-memory slots, PD planes ahead of the computation, so the loads of many planes are in
// flight while the Thomas recurrence of the current plane runs. The forward-eliminated values d'_k
// go to a per-thread stack in shared memory; the back substitution streams u_k (and v/m_k) through
// the same ring in reverse order and writes u' = u + rho x once per cell.
//
// Per cell the kernel moves the algorithmic minimum of the smoother -- read u and f, write u' --
// plus the factor arrays when lambda^2 varies over the level, and u once more in the backward pass
// (an L2 hit: the block's tile was read a few microseconds earlier).
#include "kernels.cuh"

namespace tpmg {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

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
        R m = (k == 0) ? diag : P::sub(diag, P::mul(vv2, inv_prev));
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

// ---------------------------------------------------------------- Smooth, plane pipelined
// uo = u + rho M^{-1}(f - A u) (Eq. 11) with block partial sums of ||f - A u||^2.
template <class P, int TY, int PD>
__global__ void __launch_bounds__(32 * TY) k_smooth_pp(Lv<P> L, double rho_d, const typename P::S* __restrict__ u,
                                                       const typename P::S* __restrict__ f,
                                                       typename P::S* __restrict__ uo, double* partials,
                                                       const int* done) {
    typedef typename P::S S;
    typedef typename P::R R;
    constexpr int NT = 32 * TY;
    constexpr int UPL = (TY + 2) * 34;  // u plane tile with halo
    constexpr int FPL = NT;             // f (and 1/m) plane tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (done && *(volatile const int*)done) return;

    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const bool percol = L.fac_percol != 0;
    S* ringU = reinterpret_cast<S*>(smem_raw);
    S* ringF = ringU + PD * UPL;
    S* ringI = ringF + PD * FPL;
    const size_t ring_bytes = ((size_t)PD * (UPL + 2 * FPL) * sizeof(S) + 15) & ~(size_t)15;
    R* stack = reinterpret_cast<R*>(smem_raw + ring_bytes);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY;
    const size_t pl = (size_t)nx * ny;
    const size_t c = (size_t)(j0 + ty) * nx + (i0 + tx);

    auto issue_plane = [&](int k, int slot) {
        if (k < nz) {
            const size_t b = (size_t)k * pl;
            S* Us = ringU + slot * UPL;
            cp_async<sizeof(S)>(&Us[(ty + 1) * 34 + tx + 1], u + b + c);
            cp_async<sizeof(S)>(&ringF[slot * FPL + tid], f + b + c);
            if (percol) cp_async<sizeof(S)>(&ringI[slot * FPL + tid], L.finv + b + c);
            // halo: rows j0-1 and j0+TY (32 each), columns i0-1 and i0+32 (TY+2 each)
            for (int it = tid; it < 64 + 2 * (TY + 2); it += NT) {
                int rr, cc, gj, gi;
                if (it < 64) {
                    rr = (it < 32) ? 0 : TY + 1;
                    cc = (it & 31) + 1;
                    gj = (it < 32) ? j0 - 1 : j0 + TY;
                    gi = i0 + (it & 31);
                } else {
                    const int q = it - 64;
                    rr = q >> 1;
                    cc = (q & 1) ? 33 : 0;
                    gj = j0 - 1 + rr;
                    gi = (q & 1) ? i0 + 32 : i0 - 1;
                }
                gj = wrap_p(gj, ny);
                gi = wrap_p(gi, nx);
                cp_async<sizeof(S)>(&Us[rr * 34 + cc], u + b + (size_t)gj * nx + gi);
            }
        }
        cp_commit();
    };

    for (int s = 0; s < PD; ++s) issue_plane(s, s);

    const R cx = P::cst(L.cx), cy = P::cst(L.cy), vv = P::ld(L.v, c);
    const R dh = P::cst(1.0 + 2.0 * L.cx + 2.0 * L.cy);
    const R dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
    typename P::Acc acc = 0, cmp = 0;
    R um = P::zero(), uc = P::zero(), d_prev = P::zero();
    int slot = 0;
    for (int k = 0; k < nz; ++k) {
        cp_wait<PD - 2>();
        __syncthreads();
        const S* Us = ringU + slot * UPL;
        const int nslot = (slot + 1 == PD) ? 0 : slot + 1;
        const int ctr = (ty + 1) * 34 + tx + 1;
        if (k == 0) uc = P::ld_plain(Us, ctr);
        const R up = (k + 1 < nz) ? P::ld_plain(ringU + nslot * UPL, ctr) : P::zero();
        const R hx = P::add(P::ld_plain(Us, ctr - 1), P::ld_plain(Us, ctr + 1));
        const R hy = P::add(P::ld_plain(Us, ctr - 34), P::ld_plain(Us, ctr + 34));
        const R diag = (nz == 1) ? dh : ((k == 0 || k == nz - 1) ? dh1 : dh2);
        R au = P::mul(diag, uc);
        au = P::sub(au, P::mul(cx, hx));
        au = P::sub(au, P::mul(cy, hy));
        au = P::sub(au, P::mul(vv, P::add(um, up)));
        const R r = P::sub(P::ld_plain(ringF, slot * FPL + tid), au);
        P::acc_dot(acc, cmp, r, r);
        const R inv = percol ? P::ld_plain(ringI, slot * FPL + tid) : P::ld(L.finv, k);
        const R d = P::mul(P::add(r, P::mul(vv, d_prev)), inv);
        stack[(size_t)k * NT + tid] = d;
        d_prev = d;
        um = uc;
        uc = up;
        __syncthreads();
        issue_plane(k + PD, slot);
        slot = nslot;
    }
    cp_wait<0>();
    __syncthreads();

    // back substitution, streaming u_k (and v/m_k) through the ring in reverse order
    S* bU = reinterpret_cast<S*>(smem_raw);
    S* bW = bU + PD * NT;
    auto issue_back = [&](int k, int s2) {
        if (k >= 0) {
            const size_t id = (size_t)k * pl + c;
            cp_async<sizeof(S)>(&bU[s2 * NT + tid], u + id);
            if (percol) cp_async<sizeof(S)>(&bW[s2 * NT + tid], L.fw + id);
        }
        cp_commit();
    };
    for (int s = 0; s < PD; ++s) issue_back(nz - 1 - s, s);
    const R rho = P::cst(rho_d);
    R xn = P::zero();
    slot = 0;
    for (int k = nz - 1; k >= 0; --k) {
        cp_wait<PD - 1>();
        const R w = percol ? P::ld_plain(bW, slot * NT + tid) : P::ld(L.fw, k);
        xn = P::add(stack[(size_t)k * NT + tid], P::mul(w, xn));
        const R uk = P::ld_plain(bU, slot * NT + tid);
        P::st(uo, (size_t)k * pl + c, P::add(uk, P::mul(rho, xn)));
        issue_back(k - PD, slot);
        slot = (slot + 1 == PD) ? 0 : slot + 1;
    }
    cp_wait<0>();
    if (partials) {
        double sm = block_sum(P::acc_get(acc, cmp));
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = sm;
    }
}

template <class P, int TY, int PD>
static size_t smooth_pp_smem(int nz) {
    typedef typename P::S S;
    const size_t ring = ((size_t)PD * ((TY + 2) * 34 + 2 * 32 * TY) * sizeof(S) + 15) & ~(size_t)15;
    return ring + (size_t)nz * 32 * TY * sizeof(typename P::R);
}

template <class P, int TY, int PD>
static bool try_smooth_pp(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                          typename P::S* uo, double* partials, const int* done, cudaStream_t s, int* nparts) {
    if (L.nx % 32 != 0 || L.ny % TY != 0 || L.nx < 32 || !L.finv || !L.fw) return false;
    const size_t smem = smooth_pp_smem<P, TY, PD>(L.nz);
    if (smem > 200 * 1024) return false;
    auto kern = k_smooth_pp<P, TY, PD>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grd(L.nx / 32, L.ny / TY), blk(32, TY);
    kern<<<grd, blk, smem, s>>>(L, rho, u, f, uo, partials, done);
    note_launch();
    if (nparts) *nparts = (int)(grd.x * grd.y);
    return true;
}

// Tile shapes: FP32 uses 64-column blocks (two 32-wide rows) and an 8-plane ring; the 8-byte
// types use 32-column blocks and a 6-plane ring so that two or more blocks share an SM.
template <>
bool launch_smooth_pp<PolF32>(const Lv<PolF32>& L, double rho, const float* u, const float* f, float* uo,
                              double* partials, const int* done, cudaStream_t s, int* nparts) {
    return try_smooth_pp<PolF32, 2, 8>(L, rho, u, f, uo, partials, done, s, nparts);
}
template <>
bool launch_smooth_pp<PolF64>(const Lv<PolF64>& L, double rho, const double* u, const double* f, double* uo,
                              double* partials, const int* done, cudaStream_t s, int* nparts) {
    return try_smooth_pp<PolF64, 1, 6>(L, rho, u, f, uo, partials, done, s, nparts);
}
template <>
bool launch_smooth_pp<PolDW>(const Lv<PolDW>& L, double rho, const float2* u, const float2* f, float2* uo,
                             double* partials, const int* done, cudaStream_t s, int* nparts) {
    return try_smooth_pp<PolDW, 1, 6>(L, rho, u, f, uo, partials, done, s, nparts);
}

template void launch_factors<PolF64>(const Lv<PolF64>&, double*, double*, int, cudaStream_t);
template void launch_factors<PolF32>(const Lv<PolF32>&, float*, float*, int, cudaStream_t);
template void launch_factors<PolDW>(const Lv<PolDW>&, float2*, float2*, int, cudaStream_t);

}  // namespace tpmg
