// kernels.cuh -- internal declarations shared by the kernel translation units and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "arith.cuh"

namespace tpmg {

// Sum of x over a block whose size is a multiple of 32, valid in thread 0. Warp shuffles, then
// the warp sums in a fixed order: the result is deterministic.
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double wsum[32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((tid & 31) == 0) wsum[tid >> 5] = x;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < nw; ++w) s += wsum[w];
    return s;
}

// ---------------------------------------------------------------- L2 eviction priorities
// Policies for the L2::cache_hint forms of loads and stores (createpolicy); stores of a column pair
// or of one value and read-only loads carrying a policy; the drop of a dead 128-byte line from L2
// without write-back (discard.global.L2). Used to keep the Thomas scratch of the persistent sweeps
// in L2 while the fields stream past it.
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_pair_pol(float2* p, dw a, dw b, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(p), "f"(a.hi), "f"(a.lo),
                 "f"(b.hi), "f"(b.lo), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_pair_pol(float* p, float a, float b, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;\n" ::"l"(p), "f"(a), "f"(b), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_pair_pol(double* p, double a, double b, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;\n" ::"l"(p), "d"(a), "d"(b), "l"(pol) : "memory");
}
__device__ __forceinline__ void l2_discard(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(p) : "memory");
}
__device__ __forceinline__ void st_pol(float2* p, dw a, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;\n" ::"l"(p), "f"(a.hi), "f"(a.lo), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_pol(float* p, float a, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;\n" ::"l"(p), "f"(a), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_pol(double* p, double a, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;\n" ::"l"(p), "d"(a), "l"(pol) : "memory");
}
__device__ __forceinline__ dw ld_pol(const float2* p, unsigned long long pol) {
    dw a;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;\n" : "=f"(a.hi), "=f"(a.lo) : "l"(p), "l"(pol));
    return a;
}
__device__ __forceinline__ float ld_pol(const float* p, unsigned long long pol) {
    float a;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;\n" : "=f"(a) : "l"(p), "l"(pol));
    return a;
}
__device__ __forceinline__ double ld_pol(const double* p, unsigned long long pol) {
    double a;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;\n" : "=d"(a) : "l"(p), "l"(pol));
    return a;
}

// One multigrid level as the kernels see it: an nx x ny x nz box, x fastest, with horizontal
// couplings cx = omega^2/hx^2, cy = omega^2/hy^2 (scaled by 1/4 per coarsening) and one vertical
// coefficient v_ij = omega^2 lambda_ij^2 / hz^2 per column (stored in the policy's storage type).
//
// The Thomas factors of the level's column blocks, 1/m_k and w_k = v/m_k with
// m_0 = D_0, m_k = D_k - v^2/m_{k-1}, depend only on the operator, so they are computed once per
// level (k_factors) and read by the sweeps: fac_percol = 1 stores them per cell (index k*plane+c,
// lambda^2 varying over the level); 0 stores one shared table of nz entries (lambda^2 constant).
template <class P>
struct Lv {
    int nx, ny, nz;
    double cx, cy;
    const typename P::S* v;
    const typename P::S* finv;
    const typename P::S* fw;
    int fac_percol;
    // per-cell factors only: from plane fac_k0 to plane nz-2 every column's stored 1/m_k and v/m_k
    // equal (bit for bit) those of plane nz-2 -- the forward elimination has converged to its fixed
    // point -- so the sweeps may read plane nz-2's once per column instead (nz-1: no such range)
    int fac_k0 = 1 << 30;
    int variant;  // tile variant of the pipelined Smooth chosen by the autotuner (-1: default)
    // parallel-cyclic-reduction factors of the column blocks (small levels only, else null):
    // for each of pcr_steps strides 1, 2, 4, ... the two elimination multipliers per cell, then
    // 1/b of the decoupled rows; per cell when fac_percol, else one shared table of nz rows
    const typename P::S* pcr = nullptr;
    int pcr_steps = 0;
    // global scratch for the Thomas stacks of the persistent sweep variants (gstack_bytes(nz)
    // bytes, shared by the levels; null: those variants are not used)
    void* gstack = nullptr;
};

// A sweep's constants in the policy's arithmetic type: cx, cy, the horizontal part of the diagonal
// 1 + 2 cx + 2 cy and the sweep's coefficient (rho, or 1), converted from double on the host. On this
// part the FP64 pipe that a device-side conversion (and the double arithmetic of the diagonal) runs on
// issues about one warp-instruction per 19 cycles per SM, so doing it per tile in an FP32 or
// double-word kernel made every warp queue on that pipe at each tile start.
template <class P>
struct SweepK {
    typename P::R cx, cy, dh, coef;
    int iso;  // cx == cy: square cells, one product for the four horizontal neighbours
};
template <class P>
inline SweepK<P> sweep_k(double cx, double cy, double coef) {
    SweepK<P> k;
    k.cx = P::hcst(cx);
    k.cy = P::hcst(cy);
    k.dh = P::hcst(1.0 + 2.0 * cx + 2.0 * cy);
    k.coef = P::hcst(coef);
    k.iso = cx == cy;
    return k;
}

// persistent sweep variants: at most GS_BLOCKS_PER_SM blocks per SM, each covering at most GS_MAX_NT
// columns, own a stack slot of the scratch
static constexpr int GS_BLOCKS_PER_SM = 16;
static constexpr int GS_MAX_NT = 128;
size_t gstack_bytes(int nz);

// Levels with at most this many columns run the cell-parallel kernels (one thread per cell,
// the column solve by parallel cyclic reduction): a thread per column leaves the GPU idle there.
static constexpr int PCR_MAX_COLS = 4096;
inline int pcr_steps_for(int nz) {
    int s = 0;
    while ((1 << s) < nz) ++s;
    return s;
}

// r = f - (A u) at one cell of the plane-streaming sweeps, as a chain of fused multiply-adds:
// f - diag u_c + cx (u_w + u_e) + cy (u_s + u_n) + v (u_{k-1} + u_{k+1}); on square cells
// (cx == cy) one product covers the four horizontal neighbours.
template <class P>
__device__ __forceinline__ typename P::R sweep_residual(typename P::R fk, typename P::R diag, typename P::R uc,
                                                        typename P::R w, typename P::R e, typename P::R s,
                                                        typename P::R n, typename P::R um, typename P::R up,
                                                        typename P::R cx, typename P::R cy, typename P::R vv,
                                                        bool iso) {
    // one renormalisation at the end of the chain (the _u forms, see arith.cuh)
    typename P::R r = P::fma_u(P::neg(diag), uc, fk);
    if (iso)
        r = P::fma_u(cx, P::sum4_u(w, e, s, n), r);
    else
        r = P::fma_u(cy, P::add_u(s, n), P::fma_u(cx, P::add_u(w, e), r));
    return P::fma(vv, P::add_u(um, up), r);
}

// value of policy PA converted to policy PB's arithmetic (no-op when they coincide)
template <class PA, class PB>
struct Conv {
    __device__ __forceinline__ static typename PB::R f(typename PA::R x) { return PB::cst(PA::to_d(x)); }
};
template <class P>
struct Conv<P, P> {
    __device__ __forceinline__ static typename P::R f(typename P::R x) { return x; }
};

// Device-resident solver scalars (one struct per running solve). All solver control decisions
// are taken on the device by the finalize kernels so a whole iteration can be replayed from a
// CUDA graph without host round trips; kernels return immediately once `done` is set.
struct Scalars {
    double r0;      // norm of the initial residual
    double rel;     // latest relative residual
    double tol;
    double alpha, beta, kappa;  // CG: step, direction update, <r,z>
    double last_norm;
    int iters, max_iter, done, converged, nonfinite, pad;
};

// process-wide count of kernel launches issued by the library (k_util.cu)
unsigned long long& launch_counter();
inline void note_launch() { ++launch_counter(); }

// launch shape of the column-sweep kernels: 32 consecutive x columns per warp row
struct Shape {
    dim3 grid, block;
    size_t smem;
    int nblocks() const { return (int)(grid.x * grid.y); }
};

// Thomas stack: two values (forward-eliminated rhs and w_k = v/m_k) per level per thread.
Shape sweep_shape(int nx, int ny, int nz, int bytes_per_value, bool stack);
int max_partials(int nx, int ny);

// ---------------------------------------------------------------- launchers (k_sweep.cu)
// Thomas factors of level L into finv/fw (per cell when percol, else a table of nz entries).
template <class P>
void launch_factors(const Lv<P>& L, typename P::S* finv, typename P::S* fw, int percol, cudaStream_t s);
// first plane of the converged range of per-cell factors (see Lv::fac_k0), written to *k0 (device
// int, initialised by the caller to 0): the maximum over the columns
template <class P>
void launch_factor_k0(const Lv<P>& L, const typename P::S* finv, const typename P::S* fw, int* k0, cudaStream_t s);
// Plane-pipelined kernels for levels with nx % 32 == 0; each returns its number of thread blocks
// (= partial sums written), or -1 when the level does not fit and the caller must fall back.
template <class P>
int launch_smooth_pp(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                     typename P::S* uo, double* partials, const int* done, cudaStream_t s);
template <class P, class PO>
int launch_residual_pp(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r,
                       double* partials, const int* done, cudaStream_t s);
template <class P>
int launch_line_solve_pp(const Lv<P>& L, const typename P::S* b, typename P::S* x, double scale, const int* done,
                         cudaStream_t s);
// FP32 Smooth and line solve with one tile of 128 x 2 columns per warp (k_sweep4.cu): nx % 128 == 0,
// ny even, 16-byte aligned fields and the level's scratch and factors, else -1; config picks the
// ring depth and blocks per SM (0 the default)
int launch_smooth_x4(const Lv<PolF32>& L, double rho, const float* u, const float* f, float* uo, double* partials,
                     const int* done, cudaStream_t s, int config);
int launch_line_solve_x4(const Lv<PolF32>& L, const float* b, float* x, double scale, const int* done, cudaStream_t s);
// y = A x by the two-column sweep (nx % 64 == 0, 16-byte aligned fields), else -1
template <class P>
int launch_apply_A_x2(const Lv<P>& L, const typename P::S* x, typename P::S* y, cudaStream_t s);
template <class PF, class P>
int launch_restrict_smooth_pp(const Lv<P>& Lc, double rho, const typename PF::S* rf, typename P::S* fc,
                              typename P::S* uc, const int* done, cudaStream_t s);
// Residual of the fine level L and RestrictSmooth onto the coarse level Lc in one pass (the fine
// residual is not stored): f_c = R (f - A u), u_c = rho M_c^{-1} f_c, the same values as
// launch_residual followed by launch_restrict_smooth where those solve the coarse columns by the
// Thomas algorithm. -1 when the levels do not fit (nx % 64, ny % 2, alignment, small coarse level).
template <class P>
int launch_residual_restrict(const Lv<P>& L, const Lv<P>& Lc, double rho, const typename P::S* u,
                             const typename P::S* f, typename P::S* fc, typename P::S* uc, const int* done,
                             cudaStream_t s);
// number of blocks launch_residual_pp would launch for these fields (= partial sums it writes),
// -1 where it would return -1; nothing is launched
template <class P, class PO>
int residual_pp_blocks(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r);

// ---------------------------------------------------------------- launchers (k_coarse.cu)
// Cell-parallel kernels for levels of at most PCR_MAX_COLS columns; each returns its number of
// blocks (= partial sums written), or -1 when the level is too large (or has no PCR factors).
template <class P>
size_t pcr_factor_count(const Lv<P>& L, int percol);
template <class P>
void launch_pcr_factors(const Lv<P>& L, typename P::S* pcr, int percol, cudaStream_t s);
template <class P>
int pcr_blocks(const Lv<P>& L);
template <class P>
int launch_smooth_pcr(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f, typename P::S* uo,
                      double* partials, const int* done, cudaStream_t s);
template <class P>
int launch_line_solve_pcr(const Lv<P>& L, const typename P::S* b, typename P::S* x, double scale, const int* done,
                          cudaStream_t s);
template <class PF, class P>
int launch_restrict_smooth_pcr(const Lv<P>& Lc, double rho, const typename PF::S* rf, typename P::S* fc,
                               typename P::S* uc, const int* done, cudaStream_t s);
template <class P, class PO>
int launch_residual_cell(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r,
                         double* partials, const int* done, cudaStream_t s);
template <class P, class PF>
int launch_prolongate_cell(int nxc, int nyc, int nz, const typename P::S* uc, typename PF::S* uf, const int* done,
                           cudaStream_t s);
int cell_blocks(size_t n);
// u_f += P u_c with one thread per (coarse column, plane) and its 2 x 2 fine cells (any level)
template <class P, class PF>
int launch_prolongate_x4(int nxc, int nyc, int nz, const typename P::S* uc, typename PF::S* uf, const int* done,
                         cudaStream_t s);

// ---------------------------------------------------------------- launchers (k_mg.cu)
template <class P>
void launch_apply_A(const Lv<P>& L, const typename P::S* x, typename P::S* y, cudaStream_t s);
// x = scale * M^{-1} b (scale = 1: the line solve; scale = rho: a smoothing step from zero)
template <class P>
void launch_line_solve(const Lv<P>& L, const typename P::S* b, typename P::S* x, double scale, const int* done,
                       cudaStream_t s);
// returns the number of blocks (partial sums written when partials != NULL)
template <class P>
int launch_smooth(const Lv<P>& L, double rho, const typename P::S* u, const typename P::S* f,
                   typename P::S* uo, double* partials, const int* done, cudaStream_t s);
// residual with the output in policy PO's storage (PO = P, or PolF32 for the mixed hand-over)
template <class P, class PO>
int launch_residual(const Lv<P>& L, const typename P::S* u, const typename P::S* f,
                    typename PO::S* r, double* partials, const int* done, cudaStream_t s);
// number of blocks (= partial sums) launch_residual would launch for these fields, without launching
template <class P, class PO>
int residual_launch_blocks(const Lv<P>& L, const typename P::S* u, const typename P::S* f, typename PO::S* r);
// fine level in policy PF (its residual r_f), coarse level in P
template <class PF, class P>
void launch_restrict_smooth(const Lv<P>& Lc, double rho, const typename PF::S* rf,
                            typename P::S* fc, typename P::S* uc, const int* done, cudaStream_t s);
// coarse level in P, fine level in PF
template <class P, class PF>
void launch_prolongate(int nxc, int nyc, int nz, const typename P::S* uc, typename PF::S* uf,
                       const int* done, cudaStream_t s);
// u += e (e in FP32), the mixed-precision correction
template <class P>
void launch_correct(size_t n, typename P::S* u, const float* e, const int* done, cudaStream_t s);

// ---------------------------------------------------------------- launchers (k_cg.cu)
// each returns its number of blocks (partial sums per reduced quantity; *_blocks predicts it)
template <class P>
int cg_spmv_blocks(const Lv<P>& L);
template <class P>
int cg_tridiag_blocks(const Lv<P>& L);
template <class P>
int launch_cg_spmv(const Lv<P>& L, const Scalars* sc, typename P::S* u, typename P::S* p,
                   const typename P::S* z, typename P::S* q, double* partials, cudaStream_t s);
template <class P>
int launch_cg_tridiag(const Lv<P>& L, const Scalars* sc, typename P::S* r, const typename P::S* q,
                      typename P::S* z, double* partials, cudaStream_t s);
template <class P>
void launch_cg_finish(size_t n, const Scalars* sc, typename P::S* u, const typename P::S* p,
                      cudaStream_t s);

// ---------------------------------------------------------------- batched persistent solver (k_batched.cu)
// Many independent problems of different sizes advance through one mixed-precision iterative
// refinement together, inside one cooperative persistent launch: the work of each step of the
// cycle ("phase") is cut into tiles of 32 x BTY columns over all problems; a bounded grid barrier
// separates the phases. Per-problem state decides which problems are still active.
// BT_RRS: Residual of level `level` and RestrictSmooth onto level-1 in one two-column sweep
// (a = u, b = f of the fine level, out = f_c, out2 = u_c), where the fine level takes 64 x BTY tiles
enum { BT_OUTRES = 0, BT_FINAL = 1, BT_LS0 = 2, BT_SMOOTH = 3, BT_RESID = 4, BT_RS = 5, BT_PROL = 6, BT_CORR = 7,
       BT_RRS = 8 };
static constexpr int BTY = 4;  // rows of columns per tile (block = 32 x BTY threads)
static constexpr int BMAXL = 16;

struct BLevelDesc {  // FP32 view of one level of one problem
    int nx, ny, nz, percol;
    double cx, cy;
    const float* v;
    const float* finv;
    const float* fw;
    SweepK<PolF32> k1, krho;  // the level's sweep constants with coefficient 1 and rho
};
struct BProbDesc {
    int L, nz;
    BLevelDesc lev[BMAXL + 1];
    float2* uD;         // double-word finest iterate
    const float2* fD;   // double-word finest right-hand side
    const float2* vD;   // double-word finest v per column
    SweepK<PolDW> kD;   // double-word constants of the finest level (coefficient 1)
    float* r32;         // FP32 right-hand side of the inner cycle (finest level)
    int part_base;      // first partial-sum slot of this problem's outer residual norm
    int fine_tiles;     // tiles of the outer residual (= its partial sums)
    int fine_x2;        // 1: the outer residual runs on two-column tiles
    double* history;    // relative residual history (max_iter + 1 doubles)
};
struct BTask {
    int type, prob, level;
    const void* a;  // input field (iterate / residual / coarse correction)
    const void* b;  // right-hand side
    void* out;
    void* out2;
    int tiles_x, tiles_y, tile_base;
    int x2;  // 1: tiles of 64 x BTY columns run by the two-column sweep (Smooth, Residual, line solve, RRS)
};
struct BState {
    double r0, rel;
    int iters, active, converged, nonfinite;
};
struct BatchDesc {
    int nprob, ntasks, nphase;
    const BProbDesc* probs;
    BState* state;
    const BTask* tasks;
    const int* phase_begin;  // nphase + 1 task offsets
    const int* phase_tiles;  // tiles per phase
    double* partials;
    unsigned* bar_count;
    unsigned* bar_gen;
    int* error;     // 1: a barrier wait timed out
    int* n_active;  // problems still iterating
    double rho, tol;
    int max_iter;
    unsigned long long timeout_ns;
    int nz_max;
    float* scratch;  // Thomas stacks: nz_max x 64 BTY floats per block
};
// cooperative launch of the persistent kernel; returns the CUDA status of the launch
cudaError_t launch_batched(const BatchDesc& d, int grid, size_t smem, cudaStream_t s);
// blocks per SM of the persistent kernel and its dynamic shared memory (the two-column sweep's rings)
int batched_blocks_per_sm();
size_t batched_smem_bytes();
size_t batched_scratch_floats(int grid, int nz_max);
// whether a level of nx x ny columns and its fields suit the two-column sweep tiles
bool batched_x2_fits(int nx, int ny, const void* a, const void* b, const void* out);

// ---------------------------------------------------------------- scalar kernels (k_util.cu)
// modes of finalize_norm
enum { FIN_STORE = 0, FIN_MG_INIT = 1, FIN_MG_CYCLE = 2, FIN_SUM = 3 };
void launch_finalize_norm(const double* partials, int nparts, int mode, Scalars* sc,
                          double* history, double* out, cudaStream_t s);
void launch_cg_alpha(const double* partials, int nparts, Scalars* sc, cudaStream_t s);
void launch_cg_beta(const double* partials, int nparts, int init, Scalars* sc, double* history,
                    cudaStream_t s);
void launch_scalars_init(Scalars* sc, double tol, int max_iter, cudaStream_t s);
void launch_set_ab(Scalars* sc, double alpha, double beta, cudaStream_t s);
// dst = src (n elements of P's storage) unless *done is set
template <class P>
void launch_copy(size_t n, const typename P::S* src, typename P::S* dst, const int* done, cudaStream_t s);
void launch_f64_to_dw(size_t n, const double* x, float2* y, cudaStream_t s);
void launch_dw_to_f64(size_t n, const float2* x, double* y, cudaStream_t s);
// out = in transposed (in: rows x cols row-major, out: cols x rows row-major)
template <class T>
void launch_transpose(const T* in, T* out, size_t rows, size_t cols, cudaStream_t s);
void launch_f64_to_f32(size_t n, const double* x, float* y, cudaStream_t s);
void launch_f32_to_f64(size_t n, const float* x, double* y, cudaStream_t s);
void launch_coarsen_v_f64(int nxf, int nyf, const double* vf, double* vc, cudaStream_t s);

// 1 / diag(A) at plane k of a column with vertical coupling vc: 1 + 2cx + 2cy plus vc for each
// vertical neighbour inside the column (Eq. 6's flat-box diagonal with the Neumann ends). The
// learned stage measures the network's output in these units (a Jacobi step).
__device__ __forceinline__ float diag_inv_f32(float cx2cy2, float vc, int k, int nz) {
    const float d = 1.f + cx2cy2 + (k > 0 ? vc : 0.f) + (k < nz - 1 ? vc : 0.f);
    return 1.f / d;
}

}  // namespace tpmg
