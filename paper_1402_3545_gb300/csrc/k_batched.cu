// k_batched.cu -- the batched persistent solver: many independent problems of different sizes in
// one cooperative launch.
//
// Each problem runs mixed-precision iterative refinement: r = f - A u in double-word arithmetic
// (stored FP32), one FP32 V-cycle of Algorithm 1 on A e = r from e = 0, u += e. The host turns the
// cycle of every problem into a list of phases; phase p holds one task per problem (the problem's
// p-th step: a Smooth, Residual, RestrictSmooth, Prolongate, ... on one of its levels), each task cut
// into tiles of 32 x BTY columns. The persistent blocks stride over the tiles of a phase and then
// meet at a grid barrier; problems of fewer levels simply have no task in the late phases. The
// barrier is a counter plus generation word; every wait is bounded by a time limit after which
// the kernel raises an error flag and all blocks return (TPMG_ERR_TIMEOUT on the host).
//
// One thread per column sweeps k with the Thomas recurrence (precomputed factors: a table of nz
// entries when lambda^2 is constant on the level, which is the batched workload's case), the
// forward-eliminated values on a per-block stack in global scratch (L2-resident; a stack in shared
// memory would leave room for only three blocks per SM).
#include "kernels.cuh"
#include "sweep_x2.cuh"

namespace tpmg {

__device__ __forceinline__ int bwrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier with a time limit. Returns false (and raises *error) if the wait gave up.
__device__ bool grid_barrier(const BatchDesc& d) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ok = 1;
        volatile unsigned* gen = d.bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(d.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            *d.bar_count = 0;
            __threadfence();
            atomicAdd(d.bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (*(volatile int*)d.error) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > d.timeout_ns) {
                    atomicExch(d.error, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------- FP32 tile operations
struct TileIdx {
    int i, j, tid, nt;
    bool act;
};
__device__ __forceinline__ TileIdx tile_idx(int i0, int j0, int nx, int ny) {
    TileIdx t;
    t.i = i0 + threadIdx.x;
    t.j = j0 + threadIdx.y;
    t.tid = threadIdx.y * 32 + threadIdx.x;
    t.nt = 32 * BTY;
    t.act = t.i < nx && t.j < ny;
    return t;
}

__device__ __forceinline__ float fac(const float* a, int percol, int k, size_t pl, size_t c) {
    return __ldg(a + (percol ? (size_t)k * pl + c : (size_t)k));
}

// MODE 0: out = u + rho M^{-1}(f - A u); MODE 1: out = f - A u; MODE 2: out = rho M^{-1} f (u unused)
template <int MODE>
__device__ void t_sweep(const BLevelDesc& L, float rho, const float* __restrict__ u, const float* __restrict__ f,
                        float* __restrict__ out, int i0, int j0, float* stack) {
    TileIdx t = tile_idx(i0, j0, L.nx, L.ny);
    if (!t.act) return;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const size_t pl = (size_t)nx * ny, c = (size_t)t.j * nx + t.i;
    const size_t cw = (size_t)t.j * nx + bwrap(t.i - 1, nx), ce = (size_t)t.j * nx + bwrap(t.i + 1, nx);
    const size_t cs = (size_t)bwrap(t.j - 1, ny) * nx + t.i, cn = (size_t)bwrap(t.j + 1, ny) * nx + t.i;
    const float cx = L.k1.cx, cy = L.k1.cy, vv = __ldg(L.v + c);  // converted on the host
    const float dh = L.k1.dh, dh1 = dh + vv, dh2 = dh1 + vv;
    float um = 0.f, uc = (MODE != 2) ? __ldg(u + c) : 0.f, d_prev = 0.f;
    float fnext = __ldg(f + c);
    #pragma unroll 2
    for (int k = 0; k < nz; ++k) {
        const size_t b = (size_t)k * pl;
        const float fk = fnext;
        if (k + 1 < nz) fnext = __ldg(f + b + pl + c);
        float r;
        if (MODE == 2) {
            r = fk;
        } else {
            const float up = (k + 1 < nz) ? __ldg(u + b + pl + c) : 0.f;
            const float diag = (nz == 1) ? dh : ((k == 0 || k == nz - 1) ? dh1 : dh2);
            const float hx = __ldg(u + b + cw) + __ldg(u + b + ce), hy = __ldg(u + b + cs) + __ldg(u + b + cn);
            r = fk - (diag * uc - cx * hx - cy * hy - vv * (um + up));
            um = uc;
            uc = up;
        }
        if (MODE == 1) {
            out[b + c] = r;
        } else {
            const float d = (r + vv * d_prev) * fac(L.finv, L.percol, k, pl, c);
            stack[(size_t)k * t.nt + t.tid] = d;
            d_prev = d;
        }
    }
    if (MODE == 1) return;
    float xn = 0.f;
    #pragma unroll 4
    for (int k = nz - 1; k >= 0; --k) {
        const size_t id = (size_t)k * pl + c;
        xn = stack[(size_t)k * t.nt + t.tid] + fac(L.fw, L.percol, k, pl, c) * xn;
        out[id] = (MODE == 0) ? __ldg(u + id) + rho * xn : rho * xn;
    }
}

// coarse level Lc from the fine residual rf: f_c = R r_f, u_c = rho M_c^{-1} f_c
__device__ void t_restrict_smooth(const BLevelDesc& Lc, float rho, const float* __restrict__ rf, float* __restrict__ fc,
                                  float* __restrict__ uc, int i0, int j0, float* stack) {
    TileIdx t = tile_idx(i0, j0, Lc.nx, Lc.ny);
    if (!t.act) return;
    const int nxc = Lc.nx, nz = Lc.nz, nxf = 2 * nxc;
    const size_t plc = (size_t)nxc * Lc.ny, plf = 4 * plc, c = (size_t)t.j * nxc + t.i;
    const size_t f00 = (size_t)(2 * t.j) * nxf + 2 * t.i, f01 = f00 + nxf;
    const float vv = __ldg(Lc.v + c);
    float d_prev = 0.f;
    auto fine = [&](int k) {
        const size_t bf = (size_t)k * plf;
        return 0.25f * ((__ldg(rf + bf + f00) + __ldg(rf + bf + f00 + 1)) +
                        (__ldg(rf + bf + f01) + __ldg(rf + bf + f01 + 1)));
    };
    auto fwd = [&](int k, float fk) {
        fc[(size_t)k * plc + c] = fk;
        const float d = (fk + vv * d_prev) * fac(Lc.finv, Lc.percol, k, plc, c);
        stack[(size_t)k * t.nt + t.tid] = d;
        d_prev = d;
    };
    // the children of four planes are loaded before their recurrence steps
    int k = 0;
    for (; k + 4 <= nz; k += 4) {
        float fk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) fk[q] = fine(k + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) fwd(k + q, fk[q]);
    }
    for (; k < nz; ++k) fwd(k, fine(k));
    float xn = 0.f;
    k = nz - 1;
    for (; k >= 3; k -= 4) {
        float st[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) st[q] = stack[(size_t)(k - q) * t.nt + t.tid];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xn = st[q] + fac(Lc.fw, Lc.percol, k - q, plc, c) * xn;
            uc[(size_t)(k - q) * plc + c] = rho * xn;
        }
    }
    for (; k >= 0; --k) {
        xn = stack[(size_t)k * t.nt + t.tid] + fac(Lc.fw, Lc.percol, k, plc, c) * xn;
        uc[(size_t)k * plc + c] = rho * xn;
    }
}

// fine level Lf: u_f += P u_c (bilinear, cell centred, periodic)
__device__ void t_prolongate(const BLevelDesc& Lf, const float* __restrict__ ucrs, float* __restrict__ uf, int i0, int j0) {
    TileIdx t = tile_idx(i0, j0, Lf.nx, Lf.ny);
    if (!t.act) return;
    const int nxc = Lf.nx / 2, nyc = Lf.ny / 2, nz = Lf.nz;
    const int I = t.i >> 1, J = t.j >> 1;
    const int I2 = bwrap((t.i & 1) ? I + 1 : I - 1, nxc), J2 = bwrap((t.j & 1) ? J + 1 : J - 1, nyc);
    const size_t plc = (size_t)nxc * nyc, plf = (size_t)Lf.nx * Lf.ny;
    const size_t a = (size_t)J * nxc + I, bq = (size_t)J * nxc + I2, cq = (size_t)J2 * nxc + I,
                 dq = (size_t)J2 * nxc + I2, o = (size_t)t.j * Lf.nx + t.i;
    auto pv = [&](int k) {
        const size_t bc = (size_t)k * plc;
        return 0.5625f * __ldg(ucrs + bc + a) + 0.1875f * __ldg(ucrs + bc + bq) + 0.1875f * __ldg(ucrs + bc + cq) +
               0.0625f * __ldg(ucrs + bc + dq);
    };
    // four planes per step: all loads issued before the stores (the planes are disjoint)
    int k = 0;
    for (; k + 4 <= nz; k += 4) {
        float val[4], old[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            val[q] = pv(k + q);
            old[q] = uf[(size_t)(k + q) * plf + o];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) uf[(size_t)(k + q) * plf + o] = old[q] + val[q];
    }
    for (; k < nz; ++k) uf[(size_t)k * plf + o] += pv(k);
}

// ---------------------------------------------------------------- double-word outer steps
// r32 = f - A u in double-word arithmetic (finest level), partial sum of ||r||^2 per tile
__device__ double t_outres(const BProbDesc& pb, int i0, int j0) {
    typedef PolDW P;
    typedef P::R R;
    const BLevelDesc& L = pb.lev[pb.L];
    TileIdx t = tile_idx(i0, j0, L.nx, L.ny);
    P::Acc acc = 0, cmp = 0;
    if (t.act) {
        const int nx = L.nx, ny = L.ny, nz = L.nz;
        const size_t pl = (size_t)nx * ny, c = (size_t)t.j * nx + t.i;
        const size_t cw = (size_t)t.j * nx + bwrap(t.i - 1, nx), ce = (size_t)t.j * nx + bwrap(t.i + 1, nx);
        const size_t cs = (size_t)bwrap(t.j - 1, ny) * nx + t.i, cn = (size_t)bwrap(t.j + 1, ny) * nx + t.i;
        const R cx = pb.kD.cx, cy = pb.kD.cy, vv = P::ld(pb.vD, c);  // converted on the host
        const R dh = pb.kD.dh, dh1 = P::add(dh, vv), dh2 = P::add(dh1, vv);
        R um = P::zero(), uc = P::ld_plain(pb.uD, c);
        for (int k = 0; k < nz; ++k) {
            const size_t b = (size_t)k * pl;
            const R up = (k + 1 < nz) ? P::ld_plain(pb.uD, b + pl + c) : P::zero();
            const R hx = P::add(P::ld_plain(pb.uD, b + cw), P::ld_plain(pb.uD, b + ce));
            const R hy = P::add(P::ld_plain(pb.uD, b + cs), P::ld_plain(pb.uD, b + cn));
            const R diag = (nz == 1) ? dh : ((k == 0 || k == nz - 1) ? dh1 : dh2);
            R au = P::mul(diag, uc);
            au = P::sub(au, P::mul(cx, hx));
            au = P::sub(au, P::mul(cy, hy));
            au = P::sub(au, P::mul(vv, P::add(um, up)));
            const R r = P::sub(P::ld(pb.fD, b + c), au);
            P::acc_dot(acc, cmp, r, r);
            pb.r32[b + c] = P::to_f(r);
            um = uc;
            uc = up;
        }
    }
    return P::acc_get(acc, cmp);
}

// u += e (double-word plus FP32), finest level
__device__ void t_correct(const BProbDesc& pb, const float* __restrict__ e, int i0, int j0) {
    const BLevelDesc& L = pb.lev[pb.L];
    TileIdx t = tile_idx(i0, j0, L.nx, L.ny);
    if (!t.act) return;
    const size_t pl = (size_t)L.nx * L.ny, c = (size_t)t.j * L.nx + t.i;
    // four planes per step: all loads issued before the stores (the planes are disjoint)
    int k = 0;
    for (; k + 4 <= L.nz; k += 4) {
        PolDW::R uv[4];
        float ev[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uv[q] = PolDW::ld_plain(pb.uD, (size_t)(k + q) * pl + c);
            ev[q] = __ldg(e + (size_t)(k + q) * pl + c);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) PolDW::st(pb.uD, (size_t)(k + q) * pl + c, PolDW::add(uv[q], PolDW::from_f(ev[q])));
    }
    for (; k < L.nz; ++k) {
        const size_t id = (size_t)k * pl + c;
        PolDW::st(pb.uD, id, PolDW::add(PolDW::ld_plain(pb.uD, id), PolDW::from_f(__ldg(e + id))));
    }
}

// per-problem convergence decision after the outer residual (Eq. 10), fixed-order sum
__device__ void t_final(const BatchDesc& d, int prob, int it) {
    const BProbDesc& pb = d.probs[prob];
    // a problem that has finished keeps its iteration count, residual and place in the count of
    // active problems (only this block writes this problem's state, before the next barrier)
    if (!*(volatile int*)&d.state[prob].active) return;
    __shared__ double buf[32 * BTY];
    const int tid = threadIdx.y * 32 + threadIdx.x, nt = 32 * BTY;
    double s = 0.0;
    for (int q = tid; q < pb.fine_tiles; q += nt) s += d.partials[pb.part_base + q];
    buf[tid] = s;
    __syncthreads();
    for (int h = nt / 2; h > 0; h >>= 1) {
        if (tid < h) buf[tid] += buf[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        BState& st = d.state[prob];
        const double nrm = sqrt(buf[0]);
        if (!isfinite(nrm)) {
            st.nonfinite = 1;
            st.active = 0;
            atomicSub(d.n_active, 1);
        } else if (it == 0) {
            st.r0 = nrm;
            st.rel = 1.0;
            st.iters = 0;
            if (pb.history) pb.history[0] = 1.0;
            if (nrm == 0.0) st.converged = 1;
            if (nrm == 0.0 || d.max_iter <= 0) {
                st.active = 0;
                atomicSub(d.n_active, 1);
            }
        } else {
            st.iters = it;
            st.rel = nrm / st.r0;
            if (pb.history) pb.history[it] = st.rel;
            if (st.rel < d.tol) st.converged = 1;
            if (st.rel < d.tol || it >= d.max_iter) {
                st.active = 0;
                atomicSub(d.n_active, 1);
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- two-column tiles
// Levels whose nx is a multiple of 64 (and ny of BTY) run their Smooth, Residual and first line
// solve, and the outer double-word residual, on tiles of 64 x BTY columns with the plane-pipelined
// two-column sweep of the single-problem solver (sweep_x2.cuh): the block's dynamic shared memory
// holds the rings, its scratch slot the Thomas stack.
constexpr int BPD = 4;  // ring depth of the two-column sweeps

__device__ __forceinline__ Lv<PolF32> lv32(const BLevelDesc& b) {
    Lv<PolF32> L;
    L.nx = b.nx;
    L.ny = b.ny;
    L.nz = b.nz;
    L.cx = b.cx;
    L.cy = b.cy;
    L.v = b.v;
    L.finv = b.finv;
    L.fw = b.fw;
    L.fac_percol = b.percol;
    L.variant = -1;
    return L;
}

bool batched_x2_fits(int nx, int ny, const void* a, const void* b, const void* out) {
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return nx % 64 == 0 && ny % BTY == 0 && al(a) && al(b) && al(out);
}

size_t batched_smem_bytes() {
    size_t m = sweep_x2_smem<PolDW, BTY, BPD, MODE_RESIDUAL>();
    const size_t s1 = sweep_x2_smem<PolF32, BTY, BPD, MODE_SMOOTH>();
    const size_t s2 = sweep_x2_smem<PolF32, BTY, BPD, MODE_LINESOLVE>();
    const size_t s3 = sweep_x2_smem<PolF32, BTY, BPD, MODE_RESTRICT>();
    m = s1 > m ? s1 : m;
    m = s3 > m ? s3 : m;
    return s2 > m ? s2 : m;
}

// ---------------------------------------------------------------- the persistent kernel
__global__ void __launch_bounds__(32 * BTY, 4) k_batched(BatchDesc d) {
    extern __shared__ __align__(16) unsigned char bsmem[];
    float* stack = d.scratch + (size_t)blockIdx.x * d.nz_max * 64 * BTY;
    __shared__ double red[32];
    const float rho = (float)d.rho;
    for (int it = 0; it <= d.max_iter; ++it) {
        for (int ph = 0; ph < d.nphase; ++ph) {
            const int tb = d.phase_begin[ph], te = d.phase_begin[ph + 1];
            const int ntiles = d.phase_tiles[ph];
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                // the task owning tile t (tasks of a phase are sorted by tile_base)
                int lo = tb, hi = te - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (d.tasks[mid].tile_base <= t) lo = mid;
                    else hi = mid - 1;
                }
                const BTask& tk = d.tasks[lo];
                if (tk.type == BT_FINAL) {
                    t_final(d, tk.prob, it);
                    continue;
                }
                if (!*(volatile int*)&d.state[tk.prob].active) continue;
                const int loc = t - tk.tile_base;
                const int i0 = (loc % tk.tiles_x) * 32, j0 = (loc / tk.tiles_x) * BTY;
                const BProbDesc& pb = d.probs[tk.prob];
                if (tk.x2) {
                    switch (tk.type) {
                        case BT_OUTRES: {
                            Lv<PolDW> LD;
                            const BLevelDesc& bl = pb.lev[pb.L];
                            LD.nx = bl.nx;
                            LD.ny = bl.ny;
                            LD.nz = bl.nz;
                            LD.cx = bl.cx;
                            LD.cy = bl.cy;
                            LD.v = pb.vD;
                            LD.finv = LD.fw = nullptr;
                            LD.fac_percol = 0;
                            LD.variant = -1;
                            const double s = sweep_x2_tiles<PolDW, PolF32, BTY, BPD, MODE_RESIDUAL, 0>(
                                LD, pb.kD, pb.uD, pb.fD, pb.r32, true, loc, loc + 1, 1, nullptr, bsmem);
                            if (threadIdx.x == 0 && threadIdx.y == 0) d.partials[pb.part_base + loc] = s;
                            break;
                        }
                        case BT_LS0:
                            sweep_x2_tiles<PolF32, PolF32, BTY, BPD, MODE_LINESOLVE, HINT_ALL>(
                                lv32(pb.lev[tk.level]), pb.lev[tk.level].krho, (const float*)tk.b, nullptr, (float*)tk.out, false, loc,
                                loc + 1, 1, stack, bsmem);
                            break;
                        case BT_SMOOTH:
                            sweep_x2_tiles<PolF32, PolF32, BTY, BPD, MODE_SMOOTH, HINT_ALL>(
                                lv32(pb.lev[tk.level]), pb.lev[tk.level].krho, (const float*)tk.a, (const float*)tk.b, (float*)tk.out,
                                false, loc, loc + 1, 1, stack, bsmem);
                            break;
                        case BT_RESID:
                            sweep_x2_tiles<PolF32, PolF32, BTY, BPD, MODE_RESIDUAL, 0>(
                                lv32(pb.lev[tk.level]), pb.lev[tk.level].k1, (const float*)tk.a, (const float*)tk.b, (float*)tk.out,
                                false, loc, loc + 1, 1, nullptr, bsmem);
                            break;
                        case BT_RRS: {
                            const XRestrict<PolF32> xr{lv32(pb.lev[tk.level - 1]), pb.lev[tk.level - 1].krho.coef,
                                                       0.25f, (float*)tk.out, (float*)tk.out2};
                            sweep_x2_tiles<PolF32, PolF32, BTY, BPD, MODE_RESTRICT, 0>(
                                lv32(pb.lev[tk.level]), pb.lev[tk.level].k1, (const float*)tk.a, (const float*)tk.b, nullptr, false,
                                loc, loc + 1, 1, stack, bsmem, &xr);
                            break;
                        }
                        default:
                            break;
                    }
                    continue;
                }
                switch (tk.type) {
                    case BT_OUTRES: {
                        double s = t_outres(pb, i0, j0);
                        s = block_sum(s);
                        if (threadIdx.x == 0 && threadIdx.y == 0) d.partials[pb.part_base + loc] = s;
                        (void)red;
                        break;
                    }
                    case BT_LS0:
                        t_sweep<2>(pb.lev[tk.level], rho, nullptr, (const float*)tk.b, (float*)tk.out, i0, j0, stack);
                        break;
                    case BT_SMOOTH:
                        t_sweep<0>(pb.lev[tk.level], rho, (const float*)tk.a, (const float*)tk.b, (float*)tk.out, i0, j0,
                                   stack);
                        break;
                    case BT_RESID:
                        t_sweep<1>(pb.lev[tk.level], rho, (const float*)tk.a, (const float*)tk.b, (float*)tk.out, i0, j0,
                                   stack);
                        break;
                    case BT_RS:
                        t_restrict_smooth(pb.lev[tk.level], rho, (const float*)tk.a, (float*)tk.out, (float*)tk.out2, i0,
                                          j0, stack);
                        break;
                    case BT_PROL:
                        t_prolongate(pb.lev[tk.level], (const float*)tk.a, (float*)tk.out, i0, j0);
                        break;
                    case BT_CORR:
                        t_correct(pb, (const float*)tk.a, i0, j0);
                        break;
                    default:
                        break;
                }
            }
            if (!grid_barrier(d)) return;
            // after the convergence phase every block sees the same count of active problems
            if (ph == 1 && *(volatile int*)d.n_active == 0) return;
        }
    }
}

int batched_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched, 32 * BTY, batched_smem_bytes()) != cudaSuccess)
        return 0;
    return nb < 8 ? nb : 8;  // 8 x 128 threads per SM; more only grows the scratch
}

size_t batched_scratch_floats(int grid, int nz_max) { return (size_t)grid * nz_max * 64 * BTY; }

cudaError_t launch_batched(const BatchDesc& d, int grid, size_t smem, cudaStream_t s) {
    BatchDesc arg = d;
    void* args[] = {&arg};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_batched, dim3(grid), dim3(32, BTY), args, smem, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

}  // namespace tpmg
