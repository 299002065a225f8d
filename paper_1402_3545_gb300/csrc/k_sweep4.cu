// k_sweep4.cu -- the FP32 line smoother (Eq. 11) and line solve (Eq. 9) with one tile of 128 x ROWS
// columns per warp (ROWS = 1 or 2), four columns x ROWS rows per thread.
//
// Per plane a thread copies its own 16-byte pieces of the u rows j0-1 .. j0+ROWS and of the
// right-hand side rows j0 .. j0+ROWS-1 into its part of the warp's ring and later reads only those,
// so no block or warp barrier orders the ring; the x-neighbours across thread boundaries come from
// the adjacent lanes by shuffles (lanes 0 and 31 copy the tile's periodic edge values). Four or eight
// cells share every per-plane cost (copies, addresses, ring bookkeeping) that the two-column sweep
// spends on two, and
// the planes go in pairs: the two planes' residuals are independent, so their loads and arithmetic
// interleave (a warp has few neighbours on its scheduler to hide latencies behind).
//
// A warp runs its tiles t_0, t_1, ... as a pipeline of stages: stage s sweeps tile t_s forward and,
// plane for plane alongside, tile t_{s-1} backward, so each warp holds the Thomas stack of one tile
// at a time (two scratch slots, alternating) and the forward reads and the backward writes share
// the memory system in a steady mix; with one tile per warp the stages are the plain forward and
// backward sweeps.
//
// RECOMP: the Thomas factors 1/m_k are formed in registers by the forward sweep (m_0 = D_0,
// m_k = D_k - v^2/m_{k-1}, the same operations as k_factors, so the same bits) up to the plane
// fac_k0 from which they have reached their fixed point, instead of being read. The backward sweep
// reads the stored v/m_k below fac_k0 and the converged value above. The forward-eliminated values
// go to the warp's slot of the global scratch (L2 evict-last, dropped from L2 once read back), the
// result is written evict-first. The per-cell arithmetic is that of the two-column sweep, operation
// for operation: the outputs are the same bits.
#include <type_traits>

#include "kernels.cuh"
#include "sweep_x2.cuh"

namespace tpmg {

namespace {

constexpr int XW = 128;  // columns of a tile row (32 lanes x 4)

// the ring's copies and waits are ordered against the ring's loads by the compiler ("memory")
__device__ __forceinline__ void cp16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp16_pol(float* dst, const float* src, unsigned long long pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_groups() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// global stores of the scratch and the result: no ring memory is touched, so no "memory" clobber
// (the ring loads of both planes of a pair may be scheduled around them)
__device__ __forceinline__ void st4_pol(float* p, const float (&a)[4], unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(p), "f"(a[0]), "f"(a[1]),
                 "f"(a[2]), "f"(a[3]), "l"(pol));
}
__device__ __forceinline__ void lds4(float (&a)[4], const float* p) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a[0] = t.x;
    a[1] = t.y;
    a[2] = t.z;
    a[3] = t.w;
}
__device__ __forceinline__ void ldg4(float (&a)[4], const float* p) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = t.x;
    a[1] = t.y;
    a[2] = t.z;
    a[3] = t.w;
}

// Forward ring slot in floats for a tile of ROWS rows. Smooth: u rows j0-1 .. j0+ROWS (0 .. ROWS+1),
// f rows j0 .. j0+ROWS-1, without RECOMP 1/m_k of the same rows, then the edge values (left of each
// tile row, then right, padded to four). Line solve: the right-hand side rows, without RECOMP 1/m_k.
// Backward ring slot: the stacked values of the tile's rows, then their v/m_k.
template <int MODE, bool RECOMP, int ROWS>
__host__ __device__ constexpr int x4_frows() {
    return MODE == MODE_SMOOTH ? (ROWS + 2) + ROWS + (RECOMP ? 0 : ROWS) : ROWS + (RECOMP ? 0 : ROWS);
}
template <int MODE, bool RECOMP, int ROWS>
__host__ __device__ constexpr int x4_fslot() {
    return x4_frows<MODE, RECOMP, ROWS>() * XW + (MODE == MODE_SMOOTH ? 4 : 0);
}
template <int ROWS>
__host__ __device__ constexpr int x4_bslot() {
    return 2 * ROWS * XW;
}

}  // namespace



template <int MODE, int PD, bool RECOMP, int ROWS, bool PIPE>
__global__ void __launch_bounds__(32) k_sweep_x4(Lv<PolF32> L, SweepK<PolF32> K, const float* __restrict__ u,
                                                 const float* __restrict__ f, float* __restrict__ out,
                                                 double* partials, const int* done) {
    static_assert(MODE == MODE_SMOOTH || MODE == MODE_LINESOLVE, "Smooth and line solve only");
    static_assert(PD >= 4, "a pair of planes and the plane after it are read while two more land");
    static_assert(ROWS == 1 || ROWS == 2, "tiles of one or two rows");
    constexpr bool SM = MODE == MODE_SMOOTH;
    constexpr int FS = x4_fslot<MODE, RECOMP, ROWS>(), BS = x4_bslot<ROWS>();
    constexpr int FROW = SM ? ROWS + 2 : 0;  // first right-hand-side row of a forward slot
    constexpr int IROW = FROW + ROWS;        // first 1/m_k row (without RECOMP)
    constexpr int EDGE = x4_frows<MODE, RECOMP, ROWS>() * XW;
    constexpr int TW = ROWS * XW;        // values of a tile plane
    constexpr int LINES = ROWS * 4;      // 128-byte lines of a tile plane of the stack
    extern __shared__ __align__(16) float ring[];
    if (done && *(volatile const int*)done) return;

    const int lane = threadIdx.x;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const size_t pl = (size_t)nx * ny;
    const int tiles_x = nx / XW, ntiles = tiles_x * (ny / ROWS);
    const bool percol = L.fac_percol != 0;
    const int k0 = L.fac_k0;
    float* const gs0 = reinterpret_cast<float*>(L.gstack) + (size_t)blockIdx.x * 2 * nz * TW;
    const unsigned long long pol_first = l2_evict_first(), pol_last = l2_evict_last();
    const float cx = K.cx, cy = K.cy, cf = K.coef, dh = K.dh;
    const bool iso = K.iso != 0;
    const bool want_norm = SM && partials != nullptr;
    const float* rhs = SM ? f : u;
    float* fmy = ring + 4 * lane;            // this lane's four columns in every forward ring row
    // ... and backward ring row: a region of its own when the stages overlap, else the forward ring's
    float* bmy = ring + (PIPE ? PD * FS : 0) + 4 * lane;
    float acc = 0.f, cmp = 0.f;
    const int m = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (!PIPE && m > 1) return;  // the launcher gives a non-overlapping sweep one tile per warp

    int bo0 = 0;  // row offset of the backward tile (the previous stage's forward tile)
    float y[ROWS][4] = {}, cw[ROWS][4] = {};
    for (int st = 0; st <= m; ++st) {
        const bool FW = st < m, BW = st > 0;
        const int tile = (int)blockIdx.x + st * (int)gridDim.x;
        const int i0 = FW ? (tile % tiles_x) * XW : 0, j0 = FW ? (tile / tiles_x) * ROWS : 0;
        const int x = i0 + 4 * lane;
        const int jm = j0 == 0 ? ny - 1 : j0 - 1, jp = j0 + ROWS == ny ? 0 : j0 + ROWS;
        const int o0 = j0 * nx + x, om = jm * nx + x, op = jp * nx + x;  // row r of the tile: o0 + r nx
        // lane 0 copies the periodic left neighbours of the tile rows, lane 31 the right ones
        const bool edge = lane == 0 || lane == 31;
        const int xe = lane == 0 ? (i0 == 0 ? nx - 1 : i0 - 1) : (i0 + XW == nx ? 0 : i0 + XW);
        const int e0 = j0 * nx + xe;
        const int eo = EDGE + (lane == 0 ? 0 : ROWS);
        float* gsF = gs0 + (size_t)(st & 1) * nz * TW;              // the forward tile's stack
        const float* gsB = gs0 + (size_t)((st + 1) & 1) * nz * TW;  // the backward tile's
        __syncwarp();

        auto issue_f = [&](int k, int s) {
            if (FW && k < nz) {
                const size_t b = (size_t)k * pl;
                float* d = fmy + s * FS;
                if constexpr (SM) {
                    cp16(d, u + b + om);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) cp16(d + (1 + r) * XW, u + b + o0 + r * nx);
                    cp16(d + (ROWS + 1) * XW, u + b + op);
                    if (edge) {
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) cp4(ring + s * FS + eo + r, u + b + e0 + r * nx);
                    }
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r) cp16_pol(d + (FROW + r) * XW, rhs + b + o0 + r * nx, pol_first);
                if constexpr (!RECOMP) {
                    if (percol && !(k >= k0 && k <= nz - 2)) {
#pragma unroll
                        for (int r = 0; r < ROWS; ++r)
                            cp16_pol(d + (IROW + r) * XW, L.finv + b + o0 + r * nx, pol_first);
                    }
                }
            }
        };
        auto issue_b = [&](int k, int s) {
            if (BW && k >= 0) {
                float* d = bmy + s * BS;
                const float* gk = gsB + (size_t)k * TW + 4 * lane;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) cp16(d + r * XW, gk + r * XW);
                if (percol && !(k >= k0 && k <= nz - 2)) {
                    const size_t b = (size_t)k * pl;
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) cp16_pol(d + (ROWS + r) * XW, L.fw + b + bo0 + r * nx, pol_first);
                }
            }
        };

        float v[ROWS][4] = {}, vv2[ROWS][4] = {}, dh2[ROWS][4] = {}, ci[ROWS][4] = {};
        if (FW) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) ldg4(v[r], L.v + o0 + r * nx);
            if (!RECOMP && percol && k0 <= nz - 2) {  // the converged 1/m_k, used on planes k0 .. nz-2
#pragma unroll
                for (int r = 0; r < ROWS; ++r) ldg4(ci[r], L.finv + (size_t)(nz - 2) * pl + o0 + r * nx);
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    vv2[r][q] = __fmul_rn(v[r][q], v[r][q]);
                    dh2[r][q] = __fadd_rn(__fadd_rn(dh, v[r][q]), v[r][q]);
                }
        }
        if (BW) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) y[r][q] = 0.f;
            if (percol && k0 <= nz - 2) {  // the converged v/m_k of the backward tile
#pragma unroll
                for (int r = 0; r < ROWS; ++r) ldg4(cw[r], L.fw + (size_t)(nz - 2) * pl + bo0 + r * nx);
            }
        }
        float um[ROWS][4] = {}, uc[ROWS][4] = {}, dp[ROWS][4] = {}, inv[ROWS][4] = {};

        // one plane of the forward sweep from ring slot sa (plane k) and sb (plane k+1); psum
        // receives the plane's sum of squared residuals
        auto plane = [&](int k, int sa, int sb, float& psum) {
            const float* S0 = fmy + sa * FS;
            const bool end = nz == 1 || k == 0 || k == nz - 1;
            float iv[ROWS][4], wk = 0.f;
            if (percol) {
                if constexpr (RECOMP) {
                    if (k <= k0 || k == nz - 1) {
#pragma unroll
                        for (int r = 0; r < ROWS; ++r)
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float dg = nz == 1 ? dh : (end ? __fadd_rn(dh, v[r][q]) : dh2[r][q]);
                                const float mk = k == 0 ? dg : fmaf(-vv2[r][q], inv[r][q], dg);
                                inv[r][q] = __frcp_rn(mk);
                            }
                    }
#pragma unroll
                    for (int r = 0; r < ROWS; ++r)
#pragma unroll
                        for (int q = 0; q < 4; ++q) iv[r][q] = inv[r][q];
                } else {
                    if (k >= k0 && k <= nz - 2) {
#pragma unroll
                        for (int r = 0; r < ROWS; ++r)
#pragma unroll
                            for (int q = 0; q < 4; ++q) iv[r][q] = ci[r][q];
                    } else {
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) lds4(iv[r], S0 + (IROW + r) * XW);
                    }
                }
            } else {
                const float t = __ldg(L.finv + k);
                wk = __ldg(L.fw + k);
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) iv[r][q] = t;
            }
            float rr[ROWS][4];
            if constexpr (SM) {
                if (k == 0) {
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) lds4(uc[r], S0 + (1 + r) * XW);
                }
                float up[ROWS][4] = {}, hs[4], hn[4], fv[ROWS][4];
                if (k + 1 < nz) {
                    const float* S1 = fmy + sb * FS;
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) lds4(up[r], S1 + (1 + r) * XW);
                }
                lds4(hs, S0);
                lds4(hn, S0 + (ROWS + 1) * XW);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) lds4(fv[r], S0 + (FROW + r) * XW);
                float le[ROWS], ri[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    le[r] = __shfl_up_sync(0xffffffffu, uc[r][3], 1);
                    ri[r] = __shfl_down_sync(0xffffffffu, uc[r][0], 1);
                }
                if (edge) {
                    const float* E = ring + sa * FS + eo;
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        if (lane == 0)
                            le[r] = E[r];
                        else
                            ri[r] = E[r];
                    }
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float w = q == 0 ? le[r] : uc[r][q - 1];
                        const float e = q == 3 ? ri[r] : uc[r][q + 1];
                        const float s = r == 0 ? hs[q] : uc[r > 0 ? r - 1 : 0][q];
                        const float n = r == ROWS - 1 ? hn[q] : uc[r + 1 < ROWS ? r + 1 : 0][q];
                        const float dg = nz == 1 ? dh : (end ? __fadd_rn(dh, v[r][q]) : dh2[r][q]);
                        rr[r][q] = sweep_residual<PolF32>(fv[r][q], dg, uc[r][q], w, e, s, n, um[r][q], up[r][q], cx,
                                                          cy, v[r][q], iso);
                    }
                if (want_norm) {
                    float a[ROWS];
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        a[r] = __fmul_rn(rr[r][0], rr[r][0]);
#pragma unroll
                        for (int q = 1; q < 4; ++q) a[r] = fmaf(rr[r][q], rr[r][q], a[r]);
                    }
                    psum = ROWS == 2 ? __fadd_rn(a[0], a[ROWS - 1]) : a[0];
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        um[r][q] = uc[r][q];
                        uc[r][q] = up[r][q];
                    }
            } else {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) lds4(rr[r], S0 + r * XW);
            }
            // forward elimination; the Smooth stacks g_k = u_k + rho d'_k - w_k u_{k+1}, so that the
            // backward recurrence y_k = g_k + w_k y_{k+1} yields u' = u + rho M^{-1} r directly
            float g[ROWS][4];
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    dp[r][q] = fmaf(v[r][q], dp[r][q], rr[r][q]) * iv[r][q];
                    if constexpr (SM) {
                        const float w = percol ? __fmul_rn(v[r][q], iv[r][q]) : wk;
                        g[r][q] = fmaf(-w, uc[r][q], fmaf(cf, dp[r][q], um[r][q]));
                    } else {
                        g[r][q] = dp[r][q];
                    }
                }
            float* gk = gsF + (size_t)k * TW + 4 * lane;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) st4_pol(gk + r * XW, g[r], pol_last);
        };

        // one plane of the backward sweep of the backward tile from ring slot sa
        auto back = [&](int k, int sa) {
            const float* S = bmy + sa * BS;
            float g[ROWS][4], w[ROWS][4];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) lds4(g[r], S + r * XW);
            if (!percol) {
                const float t = __ldg(L.fw + k);
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[r][q] = t;
            } else if (k >= k0 && k <= nz - 2) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[r][q] = cw[r][q];
            } else {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) lds4(w[r], S + (ROWS + r) * XW);
            }
            const size_t b = (size_t)k * pl;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                float o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    y[r][q] = fmaf(w[r][q], y[r][q], g[r][q]);
                    o[q] = SM ? y[r][q] : __fmul_rn(cf, y[r][q]);
                }
                st4_pol(out + b + bo0 + r * nx, o, pol_first);
            }
        };

        // the stage's planes in pairs through a ring of D slots; group j carries forward plane j and
        // backward plane nz-1-j
        auto run = [&](auto depth) {
            constexpr int D = decltype(depth)::value;
            for (int s = 0; s < D; ++s) {
                issue_f(s, s);
                issue_b(nz - 1 - s, s);
                commit();
            }
            int slot = 0;
            for (int k = 0; k < nz; k += 2) {
                const int s1 = slot + 1 == D ? 0 : slot + 1, s2 = s1 + 1 == D ? 0 : s1 + 1;
                wait_groups<D - 3>();  // this lane's groups k, k+1 and k+2 have landed
                if (FW) {
                    float p0 = 0.f, p1 = 0.f;
                    plane(k, slot, s1, p0);
                    if (k + 1 < nz) plane(k + 1, s1, s2, p1);
                    if (want_norm) {  // compensated running sum of the planes' sums
    #pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float yv = __fsub_rn(h == 0 ? p0 : p1, cmp);
                            const float t = __fadd_rn(acc, yv);
                            cmp = __fsub_rn(__fsub_rn(t, acc), yv);
                            acc = t;
                        }
                    }
                }
                if (BW) {  // backward planes kb and kb-1, from groups k and k+1
                    const int kb = nz - 1 - k;
                    __syncwarp();  // every lane's copies of both planes have landed: their stack lines are dead
                    const int kk = lane < LINES ? kb : kb - 1;
                    if (lane < 2 * LINES && kk >= 0) l2_discard(gsB + (size_t)kk * TW + 32 * (lane % LINES));
                    back(kb, slot);
                    if (kb >= 1) back(kb - 1, s1);
                }
                issue_f(k + D, slot);
                issue_b(nz - 1 - k - D, slot);
                commit();
                issue_f(k + D + 1, s1);
                issue_b(nz - 2 - k - D, s1);
                commit();
                slot = s2;
            }
            wait_groups<0>();
        };
        // a stage of the non-overlapping sweep has the whole ring (PD slots of the larger kind) to
        // itself: the smaller kind of slot gives it more planes in flight
        constexpr int MS = FS > BS ? FS : BS;
        constexpr int FPD = PIPE ? PD : (PD * MS) / FS, BPD = PIPE ? PD : (PD * MS) / BS;
        if (PIPE)
            run(std::integral_constant<int, PD>());
        else if (FW)
            run(std::integral_constant<int, FPD>());
        else
            run(std::integral_constant<int, BPD>());
        bo0 = o0;  // this stage's forward tile is the next stage's backward tile
    }
    if (want_norm) {
        double sm = PolF32::acc_get(acc, cmp);
        for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
        if (lane == 0) partials[blockIdx.x] = sm;
    }
}

namespace {

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Launches the sweep with at most per_sm one-warp blocks per SM and, where the level has enough
// tiles, at least min_tiles tiles per warp (so the stage pipeline keeps one tile of Thomas stack per
// warp in L2 instead of the whole level's); the grid is the smallest that covers the tiles in the
// same number of stages, so every warp gets the same number of tiles. -1 where the level or the
// fields do not take the tile (nx % 128, ny % ROWS, 16-byte alignment, no scratch or factors).
template <int MODE, int PD, bool RECOMP, int ROWS, bool PIPE>
int run_x4(const Lv<PolF32>& L, double coef, const float* u, const float* f, float* out, double* partials,
           const int* done, cudaStream_t s, int per_sm, int min_tiles) {
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    if (L.nx % XW || L.ny % ROWS || !L.gstack || !L.v || !L.finv || !L.fw) return -1;
    if (!al(L.v) || !al(u) || !al(out) || (MODE == MODE_SMOOTH && !al(f)) ||
        (L.fac_percol && (!al(L.fw) || !al(L.finv))))
        return -1;
    constexpr int FS = x4_fslot<MODE, RECOMP, ROWS>(), BS = x4_bslot<ROWS>();
    constexpr size_t smem = (size_t)PD * (PIPE ? FS + BS : (FS > BS ? FS : BS)) * sizeof(float);
    auto kern = k_sweep_x4<MODE, PD, RECOMP, ROWS, PIPE>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32, smem);
    if (occ < per_sm) per_sm = occ;
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (L.nx / XW) * (L.ny / ROWS);
    int nb = sm_count() * per_sm;
    const int slots = (int)(gstack_bytes(L.nz) / ((size_t)2 * L.nz * ROWS * XW * sizeof(float)));
    if (nb > slots) nb = slots;
    const int by_tiles = (ntiles + min_tiles - 1) / min_tiles;
    if (nb > by_tiles) nb = by_tiles;
    const int stages = (ntiles + nb - 1) / nb;
    if (!PIPE && stages > 1) return -1;  // one tile per warp: the level has more tiles than warps
    nb = (ntiles + stages - 1) / stages;
    kern<<<nb, 32, smem, s>>>(L, sweep_k<PolF32>(L.cx, L.cy, coef), u, f, out, partials, done);
    note_launch();
    return nb;
}

}  // namespace

// config 0: one-row tiles, one tile per warp (the untuned default; -1 where the level has more tiles
// than the SMs hold warps); 1: one-row tiles, two or more per warp as overlapping stages; 2: two-row
// tiles, one per warp; 3: one-row tiles, one per warp, a shallower ring and more warps per SM
int launch_smooth_x4(const Lv<PolF32>& L, double rho, const float* u, const float* f, float* uo, double* partials,
                     const int* done, cudaStream_t s, int config) {
    switch (config) {
        case 1: return run_x4<MODE_SMOOTH, 8, true, 1, true>(L, rho, u, f, uo, partials, done, s, 8, 2);
        case 2: return run_x4<MODE_SMOOTH, 8, true, 2, false>(L, rho, u, f, uo, partials, done, s, 8, 1);
        case 3: return run_x4<MODE_SMOOTH, 6, true, 1, false>(L, rho, u, f, uo, partials, done, s, 16, 1);
        default: return run_x4<MODE_SMOOTH, 7, true, 1, false>(L, rho, u, f, uo, partials, done, s, 14, 1);
    }
}

int launch_line_solve_x4(const Lv<PolF32>& L, const float* b, float* x, double scale, const int* done, cudaStream_t s) {
    int nb = run_x4<MODE_LINESOLVE, 8, true, 1, false>(L, scale, b, nullptr, x, nullptr, done, s, 16, 1);
    if (nb < 0) nb = run_x4<MODE_LINESOLVE, 8, true, 2, false>(L, scale, b, nullptr, x, nullptr, done, s, 8, 1);
    return nb;
}

}  // namespace tpmg
