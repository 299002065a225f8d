// api.cu -- the C ABI of include/tpmg.h: grid and operator objects, operator-owned workspace, the
// single-application entry points and the solvers (multigrid V-cycle, mixed-precision iterative
// refinement, fused line-preconditioned CG).
//
// Solver control lives on the device: the finalize kernels compute the norms, CG's alpha/beta and
// the convergence decision of Eq. (10) and raise a `done` flag that makes every later kernel of the
// iteration return at once. One iteration is captured into a CUDA graph and replayed; the host
// reads the flag once per iteration (one 64-byte device-to-host copy).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <cmath>
#include <cstdint>

#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"
#include "panel.cuh"
#include "tpmg.h"

using namespace tpmg;

static constexpr int MAXL = 16;
static constexpr int MAX_NZ = 256;
// the double-word solver runs a level in double-word arithmetic while 4 u kappa(M) <= 1e-10 with
// u = 2^-48 (the forward-error bound of its line solves stays at the FP64 parity tolerance)
static constexpr double DW_KAPPA_MAX = 7000.0;

static thread_local std::string g_err;

static tpmg_status set_err(tpmg_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return set_err(TPMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define TRY(expr)                                                                                 \
    do {                                                                                          \
        tpmg_status s_ = (expr);                                                                  \
        if (s_ != TPMG_OK) return s_;                                                             \
    } while (0)

struct tpmg_grid {
    int nx, ny, nz, L;
    int lnx[MAXL + 1], lny[MAXL + 1];
};

// the device buffers of one precision's multigrid hierarchy (level index 1..L)
struct Hier {
    bool ready = false;
    void* u[MAXL + 1] = {};
    void* ub[MAXL + 1] = {};
    void* f[MAXL + 1] = {};
    void* r[MAXL + 1] = {};
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;
    unsigned long long nkernels = 0;  // kernel nodes captured into the graph
};

struct tpmg_op {
    tpmg_grid g;
    int device = 0;
    double omega2 = 0, hx = 0, hy = 0, hz = 0;
    double cx[MAXL + 1], cy[MAXL + 1];
    std::vector<double> v_host[MAXL + 1];
    double* v64[MAXL + 1] = {};
    float* v32[MAXL + 1] = {};
    float2* vdw[MAXL + 1] = {};
    Hier hier[3];  // by policy id (F64, F32, DW)
    void* finv[3][MAXL + 1] = {};  // Thomas factors 1/m_k per policy and level
    void* pcr[3][MAXL + 1] = {};   // PCR factors of the small levels per policy and level
    void* gstack = nullptr;        // Thomas-stack scratch of the persistent sweep variants
    void* fw[3][MAXL + 1] = {};    // Thomas factors v/m_k
    int percol[MAXL + 1] = {};     // 1 if lambda^2 varies over the level (factors per cell)
    int fac_k0[3][MAXL + 1];       // first plane of the converged factor range (Lv::fac_k0)
    double kappa_M[MAXL + 1] = {}; // condition number of the level's column blocks
    int lsw_dw = 1;                // the double-word solver uses native FP64 below this level
    bool fac_ready[3] = {false, false, false};
    int variant[3][MAXL + 1];      // autotuned tile variant of the pipelined Smooth (-1: default)
    int fuse_restrict = 1;         // V-cycles fuse Residual and RestrictSmooth where the kernel applies
    void* cgbuf[3][4] = {};  // r, z, p, q per policy
    void* io[4] = {};        // DW conversion buffers for single applications (finest-level size)
    double* partials = nullptr;
    int max_parts = 0;
    Scalars* sc = nullptr;
    Scalars* sc_host = nullptr;  // pinned
    double* history = nullptr;
    int history_cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    GraphCache graphs[8];
    void* fcg_sc = nullptr;    // device scalars of flexible CG
    void* fcg_host = nullptr;  // pinned copy
    void* fcgbuf[3] = {};      // flexible CG scratch vectors (double-word)
    void* hio[3] = {};         // host-buffer solves: device f, u (finest level) and a transpose buffer
    cudaEvent_t hev[4] = {};   // host-buffer solves: start, solve start, solve end, end
    // the cubed-sphere panel operator (tpmg_create_panel_operator; native FP64 only)
    int panel = 0;
    double* pgeo[MAXL + 1][3] = {};  // per level: |T|, x-face and y-face coefficients
    double* prad[3] = {};            // radial E = a - b - c, B = -b, C = -c
    double* pfac[MAXL + 1][3] = {};  // per level: Thomas factors 1/m, forward and backward multipliers
    float* pgeo32[MAXL + 1][3] = {};  // FP32 copies for the mixed solve's inner V-cycles
    float* prad32[3] = {};
    float* pfac32[MAXL + 1][3] = {};
};

// ---------------------------------------------------------------- helpers
static size_t lvl_cells(const tpmg_op* op, int l) {
    return (size_t)op->g.lnx[l] * op->g.lny[l] * op->g.nz;
}
template <class P>
static const typename P::S* vptr(const tpmg_op* op, int l);
template <>
const double* vptr<PolF64>(const tpmg_op* op, int l) { return op->v64[l]; }
template <>
const float* vptr<PolF32>(const tpmg_op* op, int l) { return op->v32[l]; }
template <>
const float2* vptr<PolDW>(const tpmg_op* op, int l) { return op->vdw[l]; }
template <>
const float* vptr<PolF32B>(const tpmg_op* op, int l) { return op->v32[l]; }

template <class P>
static Lv<P> level_view(const tpmg_op* op, int l) {
    Lv<P> L;
    L.nx = op->g.lnx[l];
    L.ny = op->g.lny[l];
    L.nz = op->g.nz;
    L.cx = op->cx[l];
    L.cy = op->cy[l];
    L.v = vptr<P>(op, l);
    L.finv = (const typename P::S*)op->finv[P::id][l];
    L.fw = (const typename P::S*)op->fw[P::id][l];
    L.fac_percol = op->percol[l];
    L.fac_k0 = op->fac_k0[P::id][l];
    L.variant = op->variant[P::id][l];
    L.pcr = (const typename P::S*)op->pcr[P::id][l];
    L.gstack = op->gstack;
    L.pcr_steps = pcr_steps_for(op->g.nz);
    return L;
}

// Every device buffer of the library comes from dalloc: cudaMalloc, or the caller's allocator while
// one is installed (tpmg_set_allocator); dev_free returns a buffer to the allocator that made it.
struct AllocFns {
    tpmg_alloc_fn alloc = nullptr;
    tpmg_free_fn free = nullptr;
    void* ctx = nullptr;
};
static std::mutex g_alloc_mu;
static AllocFns g_alloc;
static std::unordered_map<void*, AllocFns>& caller_blocks() {
    static std::unordered_map<void*, AllocFns> m;
    return m;
}

static tpmg_status dalloc(void** p, size_t bytes) {
    if (*p) return TPMG_OK;
    const size_t sz = bytes < 256 ? 256 : bytes;
    AllocFns fns;
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        fns = g_alloc;
    }
    if (fns.alloc) {
        void* q = fns.alloc(sz, fns.ctx);
        if (!q) return set_err(TPMG_ERR_OOM, "the caller's allocator returned NULL");
        if (((uintptr_t)q & 255) != 0) {
            fns.free(q, fns.ctx);
            return set_err(TPMG_ERR_ARG, "the caller's allocator returned a block not aligned to 256 bytes");
        }
        std::lock_guard<std::mutex> g(g_alloc_mu);
        caller_blocks()[q] = fns;
        *p = q;
    } else {
        cudaError_t e = cudaMalloc(p, sz);
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            return set_err(TPMG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    cudaMemset(*p, 0, sz);  // defined contents for profiling runs
    return TPMG_OK;
}
static void dev_free(void* p) {
    if (!p) return;
    AllocFns fns;
    bool caller = false;
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        auto it = caller_blocks().find(p);
        if (it != caller_blocks().end()) {
            fns = it->second;
            caller_blocks().erase(it);
            caller = true;
        }
    }
    if (caller) {
        cudaDeviceSynchronize();  // no kernel of this library still uses the block
        fns.free(p, fns.ctx);
    } else {
        cudaFree(p);
    }
}
static void dfree(void*& p) {
    dev_free(p);
    p = nullptr;
}
static size_t elem_bytes(int pid) { return pid == 1 ? 4 : 8; }

static tpmg_status ensure_common(tpmg_op* op) {
    if (!op->partials) {
        // at least 152 x 8 per half: the grid-stride reductions of flexible CG use up to that many blocks
        op->max_parts = std::max(max_partials(op->g.nx, op->g.ny), 152 * 8);
        TRY(dalloc((void**)&op->partials, sizeof(double) * 2 * (size_t)op->max_parts));
    }
    if (!op->sc) TRY(dalloc((void**)&op->sc, sizeof(Scalars)));
    if (!op->sc_host) CK(cudaMallocHost((void**)&op->sc_host, sizeof(Scalars)));
    return TPMG_OK;
}

static void invalidate_graphs(tpmg_op* op) {
    for (auto& gc : op->graphs) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
        gc.key.clear();
    }
}

static tpmg_status ensure_history(tpmg_op* op, int n) {
    if (n <= op->history_cap) return TPMG_OK;
    if (op->history) {
        dev_free(op->history);
        op->history = nullptr;
        invalidate_graphs(op);
    }
    int cap = n < 1024 ? 1024 : n;
    TRY(dalloc((void**)&op->history, sizeof(double) * cap));
    op->history_cap = cap;
    return TPMG_OK;
}

// Thomas factors of every level in precision pid, computed once (they depend on the operator only)
static tpmg_status ensure_factors(tpmg_op* op, int pid) {
    if (op->fac_ready[pid]) return TPMG_OK;
    TRY(ensure_common(op));
    TRY(dalloc(&op->gstack, gstack_bytes(op->g.nz)));
    const size_t eb = elem_bytes(pid);
    for (int l = 1; l <= op->g.L; ++l) {
        size_t nvals = op->percol[l] ? lvl_cells(op, l) : (size_t)op->g.nz;
        TRY(dalloc(&op->finv[pid][l], nvals * eb));
        TRY(dalloc(&op->fw[pid][l], nvals * eb));
        switch (pid) {
            case 0: launch_factors<PolF64>(level_view<PolF64>(op, l), (double*)op->finv[0][l], (double*)op->fw[0][l], op->percol[l], 0); break;
            case 1: launch_factors<PolF32>(level_view<PolF32>(op, l), (float*)op->finv[1][l], (float*)op->fw[1][l], op->percol[l], 0); break;
            default: launch_factors<PolDW>(level_view<PolDW>(op, l), (float2*)op->finv[2][l], (float2*)op->fw[2][l], op->percol[l], 0); break;
        }
        if (op->percol[l] && op->g.nz >= 3) {
            // the converged range of the per-cell factors
            int* dk = (int*)op->partials;
            CK(cudaMemsetAsync(dk, 0, sizeof(int), 0));
            switch (pid) {
                case 0: launch_factor_k0<PolF64>(level_view<PolF64>(op, l), (const double*)op->finv[0][l], (const double*)op->fw[0][l], dk, 0); break;
                case 1: launch_factor_k0<PolF32>(level_view<PolF32>(op, l), (const float*)op->finv[1][l], (const float*)op->fw[1][l], dk, 0); break;
                default: launch_factor_k0<PolDW>(level_view<PolDW>(op, l), (const float2*)op->finv[2][l], (const float2*)op->fw[2][l], dk, 0); break;
            }
            int k0 = 0;
            CK(cudaMemcpy(&k0, dk, sizeof(int), cudaMemcpyDeviceToHost));
            op->fac_k0[pid][l] = k0;
        }
        // small levels: parallel-cyclic-reduction factors for the cell-parallel kernels
        if ((size_t)op->g.lnx[l] * op->g.lny[l] <= (size_t)PCR_MAX_COLS && op->g.nz <= 256) {
            switch (pid) {
                case 0: {
                    Lv<PolF64> L = level_view<PolF64>(op, l);
                    TRY(dalloc(&op->pcr[0][l], pcr_factor_count(L, op->percol[l]) * eb));
                    launch_pcr_factors<PolF64>(L, (double*)op->pcr[0][l], op->percol[l], 0);
                    break;
                }
                case 1: {
                    Lv<PolF32> L = level_view<PolF32>(op, l);
                    TRY(dalloc(&op->pcr[1][l], pcr_factor_count(L, op->percol[l]) * eb));
                    launch_pcr_factors<PolF32>(L, (float*)op->pcr[1][l], op->percol[l], 0);
                    break;
                }
                default: {
                    Lv<PolDW> L = level_view<PolDW>(op, l);
                    TRY(dalloc(&op->pcr[2][l], pcr_factor_count(L, op->percol[l]) * eb));
                    launch_pcr_factors<PolDW>(L, (float2*)op->pcr[2][l], op->percol[l], 0);
                    break;
                }
            }
        }
    }
    CK(cudaDeviceSynchronize());
    op->fac_ready[pid] = true;
    return TPMG_OK;
}

// hierarchy of precision pid; the finest level's u and f are allocated only when `own_fine`
// (DW: internal copies of the caller's FP64 fields; mixed inner FP32 cycle: e and r).
static tpmg_status ensure_hier(tpmg_op* op, int pid, bool own_fine) {
    TRY(ensure_factors(op, pid));
    Hier& h = op->hier[pid];
    const size_t eb = elem_bytes(pid);
    const int L = op->g.L;
    for (int l = 1; l <= L; ++l) {
        size_t bytes = lvl_cells(op, l) * eb;
        TRY(dalloc(&h.ub[l], bytes));
        TRY(dalloc(&h.r[l], bytes));
        if (l < L || own_fine) {
            TRY(dalloc(&h.u[l], bytes));
            TRY(dalloc(&h.f[l], bytes));
        }
    }
    h.ready = true;
    return ensure_common(op);
}

static tpmg_status ensure_io(tpmg_op* op) {
    size_t bytes = lvl_cells(op, op->g.L) * sizeof(float2);
    for (int t = 0; t < 4; ++t) TRY(dalloc(&op->io[t], bytes));
    return ensure_common(op);
}

static tpmg_status ensure_cg(tpmg_op* op, int pid) {
    TRY(ensure_factors(op, pid));  // the fused Tridiag reads the precomputed Thomas factors
    size_t bytes = lvl_cells(op, op->g.L) * elem_bytes(pid);
    for (int t = 0; t < 4; ++t) TRY(dalloc(&op->cgbuf[pid][t], bytes));
    if (pid == 2) TRY(ensure_hier(op, 2, true));  // DW fine u, f copies live in the DW hierarchy
    return ensure_common(op);
}

static tpmg_status check_level(const tpmg_op* op, int level) {
    if (!op) return set_err(TPMG_ERR_ARG, "NULL operator");
    if (level < 1 || level > op->g.L) return set_err(TPMG_ERR_ARG, "level out of range");
    return TPMG_OK;
}
// entry points written for the flat box refuse a cubed-sphere panel operator (its own entry points
// are tpmg_panel_*; tpmg_mg_solve, tpmg_cg_solve and tpmg_mg_solve_host serve both)
static tpmg_status flat_only(const tpmg_op* op) {
    if (op && op->panel)
        return set_err(TPMG_ERR_ARG, "a panel operator: use tpmg_panel_* or tpmg_mg_solve / tpmg_cg_solve");
    return TPMG_OK;
}

static int pid_of(tpmg_precision p) { return p == TPMG_F64 ? 0 : (p == TPMG_F32 ? 1 : 2); }

// ---------------------------------------------------------------- the V-cycle (Algorithm 1)
// Host-side orchestration of one cycle. Levels >= lsw run in policy PF, the coarser ones in PC
// (the double-word solver runs its coarsest, ill-conditioned levels in native FP64; every other
// solver uses one policy, lsw = 1). The finest level's first smoothing step is done by the caller
// (the solver fuses the convergence norm into it); `rest` continues from there.
template <class PF, class PC>
struct Cycle {
    typedef typename PF::S SF;
    typedef typename PC::S SC;
    tpmg_op* op;
    const tpmg_params* prm;
    cudaStream_t s;
    const int* done;
    int lsw;
    void* u[MAXL + 1];
    void* ub[MAXL + 1];
    void* f[MAXL + 1];
    void* r[MAXL + 1];

    Cycle(tpmg_op* o, const tpmg_params* p, cudaStream_t st, const int* d, int lsw_)
        : op(o), prm(p), s(st), done(d), lsw(lsw_) {
        for (int l = 0; l <= MAXL; ++l) {
            Hier& h = op->hier[l >= lsw ? PF::id : PC::id];
            u[l] = h.u[l];
            ub[l] = h.ub[l];
            f[l] = h.f[l];
            r[l] = h.r[l];
        }
    }
    bool hi(int l) const { return l >= lsw; }
    void smooth(int l, void*& cur, void*& oth, double* parts) {
        if (hi(l))
            launch_smooth<PF>(level_view<PF>(op, l), prm->rho, (const SF*)cur, (const SF*)f[l], (SF*)oth, parts, done, s);
        else
            launch_smooth<PC>(level_view<PC>(op, l), prm->rho, (const SC*)cur, (const SC*)f[l], (SC*)oth, parts, done, s);
        void* t = cur;
        cur = oth;
        oth = t;
    }
    void residual(int l, const void* cur) {
        if (hi(l))
            launch_residual<PF, PF>(level_view<PF>(op, l), (const SF*)cur, (const SF*)f[l], (SF*)r[l], nullptr, done, s);
        else
            launch_residual<PC, PC>(level_view<PC>(op, l), (const SC*)cur, (const SC*)f[l], (SC*)r[l], nullptr, done, s);
    }
    // coarse level l from the residual of level l+1
    void restrict_smooth(int l, void* cur) {
        if (hi(l))
            launch_restrict_smooth<PF, PF>(level_view<PF>(op, l), prm->rho, (const SF*)r[l + 1], (SF*)f[l], (SF*)cur, done, s);
        else if (hi(l + 1))
            launch_restrict_smooth<PF, PC>(level_view<PC>(op, l), prm->rho, (const SF*)r[l + 1], (SC*)f[l], (SC*)cur, done, s);
        else
            launch_restrict_smooth<PC, PC>(level_view<PC>(op, l), prm->rho, (const SC*)r[l + 1], (SC*)f[l], (SC*)cur, done, s);
    }
    // fine level l += P (level l-1)
    void prolongate(int l, const void* uc, void* cur) {
        const int nxc = op->g.lnx[l - 1], nyc = op->g.lny[l - 1], nz = op->g.nz;
        if (hi(l - 1))
            launch_prolongate<PF, PF>(nxc, nyc, nz, (const SF*)uc, (SF*)cur, done, s);
        else if (hi(l))
            launch_prolongate<PC, PF>(nxc, nyc, nz, (const SC*)uc, (SF*)cur, done, s);
        else
            launch_prolongate<PC, PC>(nxc, nyc, nz, (const SC*)uc, (SC*)cur, done, s);
    }
    // Residual of level l and RestrictSmooth onto level l-1 in one fused pass where both levels
    // run in the same policy and the shapes fit, else the two kernels; then the rest of the cycle
    // on level l-1. Returns level l-1's result.
    void* residual_coarse(int l, const void* cur) {
        if (hi(l) && hi(l - 1) && op->fuse_restrict &&
            launch_residual_restrict<PF>(level_view<PF>(op, l), level_view<PF>(op, l - 1), prm->rho, (const SF*)cur,
                                         (const SF*)f[l], (SF*)f[l - 1], (SF*)u[l - 1], done, s) >= 0)
            return coarse(l - 1, true);
        residual(l, cur);
        return coarse(l - 1, false);
    }
    // coarse level l: RestrictSmooth from level l+1's residual (already done when restricted), then
    // the rest of the cycle
    void* coarse(int l, bool restricted) {
        void* cur = u[l];
        void* oth = ub[l];
        if (!restricted) restrict_smooth(l, cur);
        if (l == 1) {
            for (int t = 1; t < prm->n_coarse; ++t) smooth(l, cur, oth, nullptr);
            return cur;
        }
        for (int t = 1; t < prm->nu_pre; ++t) smooth(l, cur, oth, nullptr);
        void* uc = residual_coarse(l, cur);
        prolongate(l, uc, cur);
        for (int t = 0; t < prm->nu_post; ++t) smooth(l, cur, oth, nullptr);
        return cur;
    }
    // finest level after its first smoothing step
    void rest(void*& cur, void*& oth) {
        const int L = op->g.L;
        if (L == 1) {
            for (int t = 1; t < prm->n_coarse; ++t) smooth(L, cur, oth, nullptr);
            return;
        }
        for (int t = 1; t < prm->nu_pre; ++t) smooth(L, cur, oth, nullptr);
        void* uc = residual_coarse(L, cur);
        prolongate(L, uc, cur);
        for (int t = 0; t < prm->nu_post; ++t) smooth(L, cur, oth, nullptr);
    }
};

// ---------------------------------------------------------------- graph replay of one iteration
template <class F>
static tpmg_status run_iteration(tpmg_op* op, int slot, const std::vector<const void*>& key, bool use_graph,
                                 cudaStream_t s, F&& body) {
    if (!use_graph) {
        body(s);
        CK(cudaGetLastError());
        return TPMG_OK;
    }
    GraphCache& gc = op->graphs[slot];
    if (!gc.exec || gc.key != key) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
        CK(cudaStreamBeginCapture(op->cap_stream, cudaStreamCaptureModeRelaxed));
        const unsigned long long c0 = launch_counter();
        body(op->cap_stream);
        gc.nkernels = launch_counter() - c0;
        launch_counter() = c0;  // captured launches run only when the graph is replayed
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(op->cap_stream, &graph);
        if (e != cudaSuccess) return set_err(TPMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gc.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            return set_err(TPMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        gc.key = key;
    }
    CK(cudaGraphLaunch(gc.exec, s));
    launch_counter() += gc.nkernels;
    return TPMG_OK;
}

static tpmg_status read_scalars(tpmg_op* op, cudaStream_t s) {
    CK(cudaMemcpyAsync(op->sc_host, op->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TPMG_OK;
}

static tpmg_status finish_info(tpmg_op* op, tpmg_info* info, cudaStream_t s) {
    const Scalars& h = *op->sc_host;
    if (info) {
        info->iters = h.iters;
        info->converged = h.converged;
        info->rel_res = h.rel;
        info->r0 = h.r0;
        if (info->history && info->history_len > 0) {
            int n = h.iters + 1 < info->history_len ? h.iters + 1 : info->history_len;
            CK(cudaMemcpyAsync(info->history, op->history, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        }
        CK(cudaEventSynchronize(op->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, op->ev0, op->ev1));
        info->ms = ms;
        CK(cudaStreamSynchronize(s));
    }
    if (h.nonfinite) return set_err(TPMG_ERR_NONFINITE, "non-finite norm or dot product");
    if (!h.converged) return set_err(TPMG_ERR_NOT_CONVERGED, "max_iter reached");
    return TPMG_OK;
}

static tpmg_status check_params(const tpmg_op* op, const tpmg_params* p) {
    if (!op || !p) return set_err(TPMG_ERR_ARG, "NULL operator or params");
    if (p->nu_pre < 1 || p->nu_post < 0 || p->n_coarse < 1 || p->max_iter < 0)
        return set_err(TPMG_ERR_ARG, "nu_pre >= 1, nu_post >= 0, n_coarse >= 1, max_iter >= 0 required");
    if (!(p->rho > 0.0) || !(p->tol >= 0.0)) return set_err(TPMG_ERR_ARG, "rho > 0 and tol >= 0 required");
    return TPMG_OK;
}

// multigrid solve on finest-level buffers A (iterate) and fL (rhs); levels >= lsw in PF, the
// coarser ones in PC
template <class PF, class PC>
static tpmg_status mg_loop(tpmg_op* op, const tpmg_params* prm, typename PF::S* A, typename PF::S* fL,
                           int lsw, cudaStream_t s) {
    typedef typename PF::S S;
    const int L = op->g.L;
    const int* done = &op->sc->done;
    S* B = (S*)op->hier[PF::id].ub[L];
    const size_t nfine = lvl_cells(op, L);
    Lv<PF> LL = level_view<PF>(op, L);
    launch_scalars_init(op->sc, prm->tol, prm->max_iter, s);
    const int nparts = launch_smooth<PF>(LL, prm->rho, A, fL, B, op->partials, done, s);
    launch_finalize_norm(op->partials, nparts, FIN_MG_INIT, op->sc, op->history, nullptr, s);
    CK(cudaGetLastError());
    TRY(read_scalars(op, s));
    auto body = [&](cudaStream_t st) {
        Cycle<PF, PC> c2(op, prm, st, done, lsw);
        c2.u[L] = A;
        c2.f[L] = fL;
        void* cur = B;
        void* oth = A;
        c2.rest(cur, oth);
        if (cur != (void*)A) launch_copy<PF>(nfine, (const S*)cur, A, done, st);
        const int np = launch_smooth<PF>(LL, prm->rho, A, fL, B, op->partials, done, st);
        launch_finalize_norm(op->partials, np, FIN_MG_CYCLE, op->sc, op->history, nullptr, st);
    };
    std::vector<const void*> key = {A, fL, B, op->history, (const void*)(size_t)prm->nu_pre,
                                    (const void*)(size_t)prm->nu_post, (const void*)(size_t)prm->n_coarse,
                                    (const void*)(size_t)(prm->rho * 1e12), (const void*)(size_t)lsw};
    int guard = 0;
    while (!op->sc_host->done && guard++ <= prm->max_iter + 1) {
        TRY(run_iteration(op, PF::id, key, prm->use_graph != 0, s, body));
        TRY(read_scalars(op, s));
    }
    return TPMG_OK;
}

// mixed precision: u, f in DW (finest level of the DW hierarchy), FP32 inner hierarchy
static tpmg_status mixed_loop(tpmg_op* op, const tpmg_params* prm, float2* uD, const float2* fD,
                              cudaStream_t s) {
    const int L = op->g.L;
    const int* done = &op->sc->done;
    Hier& h32 = op->hier[1];
    float* e = (float*)h32.u[L];
    float* eb = (float*)h32.ub[L];
    float* r32 = (float*)h32.f[L];
    const size_t nfine = lvl_cells(op, L);
    Lv<PolDW> LD = level_view<PolDW>(op, L);
    Lv<PolF32> L32 = level_view<PolF32>(op, L);
    launch_scalars_init(op->sc, prm->tol, prm->max_iter, s);
    const int nparts = launch_residual<PolDW, PolF32>(LD, uD, fD, r32, op->partials, done, s);
    launch_finalize_norm(op->partials, nparts, FIN_MG_INIT, op->sc, op->history, nullptr, s);
    CK(cudaGetLastError());
    TRY(read_scalars(op, s));
    auto body = [&](cudaStream_t st) {
        void* cur = e;
        void* oth = eb;
        // first smoothing step from e = 0: e = rho M^{-1} r
        launch_line_solve<PolF32>(L32, r32, e, prm->rho, done, st);
        if (prm->coarse_bf16) {
            Cycle<PolF32, PolF32B> c(op, prm, st, done, L);  // levels below the finest hold BF16 values
            c.rest(cur, oth);
        } else {
            Cycle<PolF32, PolF32> c(op, prm, st, done, 1);
            c.rest(cur, oth);
        }
        launch_correct<PolDW>(nfine, uD, (const float*)cur, done, st);
        const int np = launch_residual<PolDW, PolF32>(LD, uD, fD, r32, op->partials, done, st);
        launch_finalize_norm(op->partials, np, FIN_MG_CYCLE, op->sc, op->history, nullptr, st);
    };
    std::vector<const void*> key = {uD, fD, e, op->history, (const void*)(size_t)prm->nu_pre,
                                    (const void*)(size_t)prm->nu_post, (const void*)(size_t)prm->n_coarse,
                                    (const void*)(size_t)(prm->rho * 1e12), (const void*)(size_t)prm->coarse_bf16};
    int guard = 0;
    while (!op->sc_host->done && guard++ <= prm->max_iter + 1) {
        TRY(run_iteration(op, 3, key, prm->use_graph != 0, s, body));
        TRY(read_scalars(op, s));
    }
    return TPMG_OK;
}

template <class P>
static tpmg_status cg_loop(tpmg_op* op, const tpmg_params* prm, typename P::S* u, const typename P::S* f,
                           cudaStream_t s) {
    typedef typename P::S S;
    const int pid = P::id;
    S* r = (S*)op->cgbuf[pid][0];
    S* z = (S*)op->cgbuf[pid][1];
    S* p = (S*)op->cgbuf[pid][2];
    S* q = (S*)op->cgbuf[pid][3];
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    Lv<P> LL = level_view<P>(op, L);
    const int nb_spmv = cg_spmv_blocks(LL);
    const int nb_tri = cg_tridiag_blocks(LL);
    launch_scalars_init(op->sc, prm->tol, prm->max_iter, s);
    launch_residual<P, P>(LL, u, f, r, nullptr, nullptr, s);
    CK(cudaMemsetAsync(p, 0, n * sizeof(S), s));
    CK(cudaMemsetAsync(q, 0, n * sizeof(S), s));
    launch_cg_tridiag<P>(LL, op->sc, r, q, z, op->partials, s);
    launch_cg_beta(op->partials, nb_tri, 1, op->sc, op->history, s);
    CK(cudaGetLastError());
    TRY(read_scalars(op, s));
    auto body = [&](cudaStream_t st) {
        launch_cg_spmv<P>(LL, op->sc, u, p, z, q, op->partials, st);
        launch_cg_alpha(op->partials, nb_spmv, op->sc, st);
        launch_cg_tridiag<P>(LL, op->sc, r, q, z, op->partials, st);
        launch_cg_beta(op->partials, nb_tri, 0, op->sc, op->history, st);
    };
    std::vector<const void*> key = {u, f, r, op->history};
    int guard = 0;
    while (!op->sc_host->done && guard++ <= prm->max_iter + 1) {
        TRY(run_iteration(op, 4 + pid, key, prm->use_graph != 0, s, body));
        TRY(read_scalars(op, s));
    }
    launch_cg_finish<P>(n, op->sc, u, p, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

// ================================================================ C ABI
extern "C" {

const char* tpmg_status_string(tpmg_status s) {
    switch (s) {
        case TPMG_OK: return "ok";
        case TPMG_ERR_ARG: return "invalid argument";
        case TPMG_ERR_CUDA: return "CUDA error";
        case TPMG_ERR_OOM: return "out of device memory";
        case TPMG_ERR_NOT_CONVERGED: return "not converged";
        case TPMG_ERR_NONFINITE: return "non-finite value";
        case TPMG_ERR_TIMEOUT: return "device wait timed out";
        case TPMG_ERR_NN_REJECTED: return "learned stage rejected";
    }
    return "unknown status";
}

const char* tpmg_last_error(void) { return g_err.c_str(); }

tpmg_status tpmg_create_grid(int nx, int ny, int nz, int nlevels, tpmg_grid** out) {
    if (!out) return set_err(TPMG_ERR_ARG, "NULL output pointer");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nz > MAX_NZ) return set_err(TPMG_ERR_ARG, "need nx, ny >= 1 and 1 <= nz <= 256");
    if (nlevels < 0 || nlevels > MAXL) return set_err(TPMG_ERR_ARG, "nlevels must be in [0, 16]");
    int L = nlevels;
    if (L == 0) {
        L = 1;
        int a = nx, b = ny;
        while (a % 2 == 0 && b % 2 == 0 && (a > b ? a : b) > 8 && L < MAXL) {
            a /= 2;
            b /= 2;
            ++L;
        }
    }
    const int div = 1 << (L - 1);
    if (nx % div != 0 || ny % div != 0) return set_err(TPMG_ERR_ARG, "nx and ny must be divisible by 2^(nlevels-1)");
    tpmg_grid* g = new tpmg_grid();
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->L = L;
    for (int l = 0; l <= MAXL; ++l) g->lnx[l] = g->lny[l] = 0;
    for (int l = L; l >= 1; --l) {
        g->lnx[l] = nx >> (L - l);
        g->lny[l] = ny >> (L - l);
    }
    *out = g;
    return TPMG_OK;
}

tpmg_status tpmg_destroy_grid(tpmg_grid* g) {
    delete g;
    return TPMG_OK;
}

int tpmg_grid_nlevels(const tpmg_grid* g) { return g ? g->L : 0; }

tpmg_status tpmg_grid_level_size(const tpmg_grid* g, int level, int* nx, int* ny) {
    if (!g || level < 1 || level > g->L) return set_err(TPMG_ERR_ARG, "bad grid or level");
    if (nx) *nx = g->lnx[level];
    if (ny) *ny = g->lny[level];
    return TPMG_OK;
}

tpmg_status tpmg_create_operator(const tpmg_grid* g, double omega2, double hx, double hy, double hz,
                                 double lambda2, const double* lambda2_col, tpmg_op** out) {
    if (!g || !out) return set_err(TPMG_ERR_ARG, "NULL grid or output pointer");
    *out = nullptr;
    if (!(omega2 >= 0.0) || !(hx > 0.0) || !(hy > 0.0) || !(hz > 0.0))
        return set_err(TPMG_ERR_ARG, "omega2 >= 0 and positive mesh widths required");
    tpmg_op* op = new tpmg_op();
    for (int p = 0; p < 3; ++p)
        for (int l = 0; l <= MAXL; ++l) {
            op->variant[p][l] = -1;  // untuned: the launcher's default
            op->fac_k0[p][l] = 1 << 30;
        }
    op->g = *g;
    op->omega2 = omega2;
    op->hx = hx;
    op->hy = hy;
    op->hz = hz;
    cudaGetDevice(&op->device);
    const int L = g->L;
    // finest-level coefficients (Sec. 2.1.1): cx = omega^2/hx^2, cy = omega^2/hy^2,
    // v_ij = omega^2 lambda_ij^2 / hz^2; coarse levels: h doubles (cx, cy / 4), v averaged
    op->cx[L] = omega2 / (hx * hx);
    op->cy[L] = omega2 / (hy * hy);
    for (int l = L - 1; l >= 1; --l) {
        op->cx[l] = op->cx[l + 1] / 4.0;
        op->cy[l] = op->cy[l + 1] / 4.0;
    }
    const size_t ncol = (size_t)g->nx * g->ny;
    std::vector<double> vf(ncol);
    for (size_t c = 0; c < ncol; ++c) {
        double lam = lambda2_col ? lambda2_col[c] : lambda2;
        if (!(lam >= 0.0)) {
            delete op;
            return set_err(TPMG_ERR_ARG, "lambda^2 must be non-negative and finite");
        }
        vf[c] = omega2 * lam / (hz * hz);
    }
    tpmg_status st = TPMG_OK;
    auto fail = [&](tpmg_status s2) {
        tpmg_destroy_operator(op);
        return s2;
    };
    for (int l = L; l >= 1; --l) {
        size_t nc = (size_t)g->lnx[l] * g->lny[l];
        if ((st = dalloc((void**)&op->v64[l], nc * sizeof(double))) != TPMG_OK) return fail(st);
        if ((st = dalloc((void**)&op->v32[l], nc * sizeof(float))) != TPMG_OK) return fail(st);
        if ((st = dalloc((void**)&op->vdw[l], nc * sizeof(float2))) != TPMG_OK) return fail(st);
        if (l == L) {
            if (cudaMemcpy(op->v64[l], vf.data(), nc * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(set_err(TPMG_ERR_CUDA, "copy of lambda^2 failed"));
        } else {
            launch_coarsen_v_f64(g->lnx[l + 1], g->lny[l + 1], op->v64[l + 1], op->v64[l], 0);
        }
        launch_f64_to_f32(nc, op->v64[l], op->v32[l], 0);
        launch_f64_to_dw(nc, op->v64[l], op->vdw[l], 0);
        op->v_host[l].resize(nc);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(set_err(TPMG_ERR_CUDA, "operator setup kernels failed"));
    for (int l = 1; l <= L; ++l) {
        cudaMemcpy(op->v_host[l].data(), op->v64[l], op->v_host[l].size() * sizeof(double), cudaMemcpyDeviceToHost);
        const std::vector<double>& vh = op->v_host[l];
        op->percol[l] = 0;
        double vmax = 0.0;
        for (size_t c = 0; c < vh.size(); ++c) {
            if (vh[c] != vh[0]) op->percol[l] = 1;
            vmax = vh[c] > vmax ? vh[c] : vmax;
        }
        // kappa(M) = (largest/smallest eigenvalue) of the column block: D - v L_N with L_N the
        // Neumann 1-D Laplacian, whose spectrum lies in [0, 4): kappa < 1 + 4 v / (1 + 2cx + 2cy)
        op->kappa_M[l] = 1.0 + 4.0 * vmax / (1.0 + 2.0 * op->cx[l] + 2.0 * op->cy[l]);
    }
    // Double-word arithmetic (unit roundoff ~2^-48) loses log2(kappa(M)) bits in the line solves;
    // levels with kappa(M) > DW_KAPPA_MAX (all coarse and small) run in native FP64 instead, which
    // keeps every smoother application within 1e-10 of an FP64 computation (4 u kappa <= 1e-10).
    op->lsw_dw = L + 1;
    for (int l = L; l >= 1 && op->kappa_M[l] <= DW_KAPPA_MAX; --l) op->lsw_dw = l;
    if (cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&op->ev0) != cudaSuccess || cudaEventCreate(&op->ev1) != cudaSuccess)
        return fail(set_err(TPMG_ERR_CUDA, "stream/event creation failed"));
    *out = op;
    return TPMG_OK;
}

static void drop_batches_of(const tpmg_op* op);

tpmg_status tpmg_destroy_operator(tpmg_op* op) {
    if (!op) return TPMG_OK;
    cudaDeviceSynchronize();
    drop_batches_of(op);
    invalidate_graphs(op);
    for (int l = 0; l <= MAXL; ++l) {
        dfree((void*&)op->v64[l]);
        dfree((void*&)op->v32[l]);
        dfree((void*&)op->vdw[l]);
        for (int p = 0; p < 3; ++p) {
            dfree(op->finv[p][l]);
            dfree(op->pcr[p][l]);
            dfree(op->fw[p][l]);
            dfree(op->hier[p].u[l]);
            dfree(op->hier[p].ub[l]);
            dfree(op->hier[p].f[l]);
            dfree(op->hier[p].r[l]);
        }
    }
    for (int p = 0; p < 3; ++p)
        for (int t = 0; t < 4; ++t) dfree(op->cgbuf[p][t]);
    for (int t = 0; t < 4; ++t) dfree(op->io[t]);
    for (int t = 0; t < 3; ++t) dfree(op->fcgbuf[t]);
    dfree(op->fcg_sc);
    if (op->fcg_host) cudaFreeHost(op->fcg_host);
    dfree((void*&)op->partials);
    dfree(op->gstack);
    dfree((void*&)op->sc);
    dfree((void*&)op->history);
    if (op->sc_host) cudaFreeHost(op->sc_host);
    if (op->cap_stream) cudaStreamDestroy(op->cap_stream);
    if (op->ev0) cudaEventDestroy(op->ev0);
    if (op->ev1) cudaEventDestroy(op->ev1);
    for (int t = 0; t < 3; ++t) dfree(op->hio[t]);
    for (int t = 0; t < 4; ++t)
        if (op->hev[t]) cudaEventDestroy(op->hev[t]);
    for (int t = 0; t < 3; ++t) {
        dfree((void*&)op->prad[t]);
        dfree((void*&)op->prad32[t]);
        for (int l = 0; l <= MAXL; ++l) {
            dfree((void*&)op->pgeo[l][t]);
            dfree((void*&)op->pfac[l][t]);
            dfree((void*&)op->pgeo32[l][t]);
            dfree((void*&)op->pfac32[l][t]);
        }
    }
    delete op;
    return TPMG_OK;
}

tpmg_status tpmg_op_reserve(tpmg_op* op, tpmg_precision prec) {
    TRY(flat_only(op));
    if (!op) return set_err(TPMG_ERR_ARG, "NULL operator");
    switch (prec) {
        case TPMG_F64: TRY(ensure_hier(op, 0, false)); TRY(ensure_cg(op, 0)); break;
        case TPMG_F32: TRY(ensure_hier(op, 1, false)); TRY(ensure_cg(op, 1)); break;
        case TPMG_DW: TRY(ensure_hier(op, 2, true)); TRY(ensure_cg(op, 2)); TRY(ensure_io(op)); break;
        case TPMG_MIXED: TRY(ensure_hier(op, 2, true)); TRY(ensure_hier(op, 1, true)); break;
        default: return set_err(TPMG_ERR_ARG, "unknown precision");
    }
    TRY(ensure_history(op, 1024));
    CK(cudaDeviceSynchronize());
    return TPMG_OK;
}

tpmg_status tpmg_op_level_coefficients(const tpmg_op* op, int level, double* cx, double* cy, double* v_host) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (cx) *cx = op->cx[level];
    if (cy) *cy = op->cy[level];
    if (v_host) memcpy(v_host, op->v_host[level].data(), op->v_host[level].size() * sizeof(double));
    return TPMG_OK;
}

// ---------------------------------------------------------------- single applications
#define DISPATCH_PREC(prec, ...)                                                                 \
    switch (prec) {                                                                              \
        case TPMG_F64: { typedef PolF64 P; __VA_ARGS__; } break;                                 \
        case TPMG_F32: { typedef PolF32 P; __VA_ARGS__; } break;                                 \
        case TPMG_DW:  { typedef PolDW P; __VA_ARGS__; } break;                                  \
        default: return set_err(TPMG_ERR_ARG, "precision must be TPMG_F64, TPMG_F32 or TPMG_DW"); \
    }

}  // extern "C"

// For TPMG_DW the caller's double fields are converted into the io buffers around the kernel.
struct DWIO {
    tpmg_op* op;
    cudaStream_t s;
    float2* in(int slot, const void* x, size_t n) {
        launch_f64_to_dw(n, (const double*)x, (float2*)op->io[slot], s);
        return (float2*)op->io[slot];
    }
    float2* buf(int slot) { return (float2*)op->io[slot]; }
    void out(int slot, void* y, size_t n) { launch_dw_to_f64(n, (const float2*)op->io[slot], (double*)y, s); }
};

template <class P>
static typename P::S* in_ptr(tpmg_op* op, cudaStream_t s, int slot, const void* x, size_t n) {
    if (P::id == 2) return (typename P::S*)DWIO{op, s}.in(slot, x, n);
    return (typename P::S*)x;
}
template <class P>
static typename P::S* out_ptr(tpmg_op* op, int slot, void* y) {
    if (P::id == 2) return (typename P::S*)op->io[slot];
    return (typename P::S*)y;
}
template <class P>
static void out_back(tpmg_op* op, cudaStream_t s, int slot, void* y, size_t n) {
    if (P::id == 2) DWIO{op, s}.out(slot, y, n);
}

static tpmg_status prep_unit(tpmg_op* op, tpmg_precision prec) {
    if (prec == TPMG_DW) TRY(ensure_io(op));
    if (prec == TPMG_F64 || prec == TPMG_F32 || prec == TPMG_DW) TRY(ensure_factors(op, pid_of(prec)));
    return ensure_common(op);
}

extern "C" {

tpmg_status tpmg_apply_A(tpmg_op* op, int level, tpmg_precision prec, const void* x, void* y, void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec == TPMG_DW && level < op->lsw_dw) prec = TPMG_F64;  // see DW_KAPPA_MAX
    if (!x || !y) return set_err(TPMG_ERR_ARG, "NULL field");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = lvl_cells(op, level);
    DISPATCH_PREC(prec, {
        auto* xi = in_ptr<P>(op, s, 0, x, n);
        auto* yo = out_ptr<P>(op, 1, y);
        launch_apply_A<P>(level_view<P>(op, level), xi, yo, s);
        out_back<P>(op, s, 1, y, n);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_line_solve(tpmg_op* op, int level, tpmg_precision prec, const void* b, void* x, void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec == TPMG_DW && level < op->lsw_dw) prec = TPMG_F64;  // see DW_KAPPA_MAX
    if (!x || !b) return set_err(TPMG_ERR_ARG, "NULL field");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = lvl_cells(op, level);
    DISPATCH_PREC(prec, {
        auto* bi = in_ptr<P>(op, s, 0, b, n);
        auto* xo = out_ptr<P>(op, 1, x);
        launch_line_solve<P>(level_view<P>(op, level), bi, xo, 1.0, nullptr, s);
        out_back<P>(op, s, 1, x, n);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_smooth(tpmg_op* op, int level, tpmg_precision prec, double rho, const void* u,
                        const void* f, void* u_out, double* norm_out, void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec == TPMG_DW && level < op->lsw_dw) prec = TPMG_F64;  // see DW_KAPPA_MAX
    if (!u || !f || !u_out) return set_err(TPMG_ERR_ARG, "NULL field");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = lvl_cells(op, level);
    DISPATCH_PREC(prec, {
        Lv<P> LL = level_view<P>(op, level);
        auto* ui = in_ptr<P>(op, s, 0, u, n);
        auto* fi = in_ptr<P>(op, s, 1, f, n);
        auto* uo = out_ptr<P>(op, 2, u_out);
        const int np = launch_smooth<P>(LL, rho, ui, fi, uo, norm_out ? op->partials : nullptr, nullptr, s);
        if (norm_out) launch_finalize_norm(op->partials, np, FIN_STORE, op->sc, nullptr, norm_out, s);
        out_back<P>(op, s, 2, u_out, n);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_residual(tpmg_op* op, int level, tpmg_precision prec, const void* u, const void* f,
                          void* r, double* norm_out, void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec == TPMG_DW && level < op->lsw_dw) prec = TPMG_F64;  // see DW_KAPPA_MAX
    if (!u || !f || !r) return set_err(TPMG_ERR_ARG, "NULL field");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = lvl_cells(op, level);
    DISPATCH_PREC(prec, {
        Lv<P> LL = level_view<P>(op, level);
        auto* ui = in_ptr<P>(op, s, 0, u, n);
        auto* fi = in_ptr<P>(op, s, 1, f, n);
        auto* ro = out_ptr<P>(op, 2, r);
        const int np = launch_residual<P, P>(LL, ui, fi, ro, norm_out ? op->partials : nullptr, nullptr, s);
        if (norm_out) launch_finalize_norm(op->partials, np, FIN_STORE, op->sc, nullptr, norm_out, s);
        out_back<P>(op, s, 2, r, n);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_restrict_smooth(tpmg_op* op, int level, tpmg_precision prec, double rho, const void* r_fine,
                                 void* f_c, void* u_c, void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec == TPMG_DW && level < op->lsw_dw) prec = TPMG_F64;  // see DW_KAPPA_MAX
    if (level >= op->g.L) return set_err(TPMG_ERR_ARG, "restrict_smooth needs a coarse level < L");
    if (!r_fine || !f_c || !u_c) return set_err(TPMG_ERR_ARG, "NULL field");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nc = lvl_cells(op, level), nf = lvl_cells(op, level + 1);
    DISPATCH_PREC(prec, {
        auto* ri = in_ptr<P>(op, s, 0, r_fine, nf);
        auto* fo = out_ptr<P>(op, 1, f_c);
        auto* uo = out_ptr<P>(op, 2, u_c);
        launch_restrict_smooth<P, P>(level_view<P>(op, level), rho, ri, fo, uo, nullptr, s);
        out_back<P>(op, s, 1, f_c, nc);
        out_back<P>(op, s, 2, u_c, nc);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_residual_restrict_smooth(tpmg_op* op, int level, tpmg_precision prec, double rho,
                                          const void* u_fine, const void* f_fine, void* f_c, void* u_c,
                                          void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (level >= op->g.L) return set_err(TPMG_ERR_ARG, "residual_restrict_smooth needs a coarse level < L");
    if (!u_fine || !f_fine || !f_c || !u_c) return set_err(TPMG_ERR_ARG, "NULL field");
    if (prec == TPMG_DW && level + 1 < op->lsw_dw) prec = TPMG_F64;  // see DW_KAPPA_MAX
    if (prec == TPMG_DW && level < op->lsw_dw) {
        // double-word fine level over a native-FP64 coarse level: the two kernels, the residual
        // handed over in FP64 through a staging buffer
        TRY(prep_unit(op, prec));
        TRY(tpmg_residual(op, level + 1, prec, u_fine, f_fine, op->io[3], nullptr, stream));
        return tpmg_restrict_smooth(op, level, prec, rho, op->io[3], f_c, u_c, stream);
    }
    TRY(prep_unit(op, prec));
    TRY(ensure_hier(op, pid_of(prec), true));  // the fine residual buffer of the unfused fallback
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nc = lvl_cells(op, level), nf = lvl_cells(op, level + 1);
    DISPATCH_PREC(prec, {
        typedef typename P::S S;
        auto* ui = in_ptr<P>(op, s, 0, u_fine, nf);
        auto* fi = in_ptr<P>(op, s, 1, f_fine, nf);
        auto* fo = out_ptr<P>(op, 2, f_c);
        auto* uo = out_ptr<P>(op, 3, u_c);
        Lv<P> LF = level_view<P>(op, level + 1), LC = level_view<P>(op, level);
        if (launch_residual_restrict<P>(LF, LC, rho, ui, fi, fo, uo, nullptr, s) < 0) {
            S* r = (S*)op->hier[P::id].r[level + 1];
            launch_residual<P, P>(LF, ui, fi, r, nullptr, nullptr, s);
            launch_restrict_smooth<P, P>(LC, rho, r, fo, uo, nullptr, s);
        }
        out_back<P>(op, s, 2, f_c, nc);
        out_back<P>(op, s, 3, u_c, nc);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_set_allocator(tpmg_alloc_fn alloc_fn, tpmg_free_fn free_fn, void* ctx) {
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return set_err(TPMG_ERR_ARG, "tpmg_set_allocator needs both functions or neither");
    std::lock_guard<std::mutex> g(g_alloc_mu);
    g_alloc.alloc = alloc_fn;
    g_alloc.free = free_fn;
    g_alloc.ctx = alloc_fn ? ctx : nullptr;
    return TPMG_OK;
}

tpmg_status tpmg_set_fusion(tpmg_op* op, int enable) {
    TRY(flat_only(op));
    if (!op) return set_err(TPMG_ERR_ARG, "NULL operator");
    const int on = enable != 0;
    if (op->fuse_restrict != on) {
        op->fuse_restrict = on;
        invalidate_graphs(op);
        drop_batches_of(op);  // their task lists follow the switch
    }
    return TPMG_OK;
}

tpmg_status tpmg_prolongate(tpmg_op* op, int level, tpmg_precision prec, const void* u_c, void* u_f, void* stream) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec == TPMG_DW && level - 1 < op->lsw_dw) prec = TPMG_F64;
    if (level <= 1) return set_err(TPMG_ERR_ARG, "prolongate needs a fine level > 1");
    if (!u_c || !u_f) return set_err(TPMG_ERR_ARG, "NULL field");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nc = lvl_cells(op, level - 1), nf = lvl_cells(op, level);
    DISPATCH_PREC(prec, {
        auto* ci = in_ptr<P>(op, s, 0, u_c, nc);
        auto* fio = in_ptr<P>(op, s, 1, u_f, nf);
        launch_prolongate<P, P>(op->g.lnx[level - 1], op->g.lny[level - 1], op->g.nz, ci, fio, nullptr, s);
        out_back<P>(op, s, 1, u_f, nf);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_cg_fused_spmv(tpmg_op* op, tpmg_precision prec, double alpha, double beta, void* u, void* p,
                               const void* z, void* q, double* sigma_out, void* stream) {
    TRY(flat_only(op));
    if (!op) return set_err(TPMG_ERR_ARG, "NULL operator");
    if (prec == TPMG_DW && op->lsw_dw > op->g.L) prec = TPMG_F64;
    if (!u || !p || !z || !q || !sigma_out) return set_err(TPMG_ERR_ARG, "NULL argument");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    launch_set_ab(op->sc, alpha, beta, s);
    DISPATCH_PREC(prec, {
        Lv<P> LL = level_view<P>(op, L);
        auto* ui = in_ptr<P>(op, s, 0, u, n);
        auto* pi = in_ptr<P>(op, s, 1, p, n);
        auto* zi = in_ptr<P>(op, s, 2, z, n);
        auto* qi = in_ptr<P>(op, s, 3, q, n);
        const int nb = launch_cg_spmv<P>(LL, op->sc, ui, pi, zi, qi, op->partials, s);
        launch_finalize_norm(op->partials, nb, FIN_SUM, op->sc, nullptr, sigma_out, s);
        out_back<P>(op, s, 0, u, n);
        out_back<P>(op, s, 1, p, n);
        out_back<P>(op, s, 3, q, n);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_cg_fused_tridiag(tpmg_op* op, tpmg_precision prec, double alpha, void* r, const void* q, void* z,
                                  double* rr_out, double* rz_out, void* stream) {
    TRY(flat_only(op));
    if (!op) return set_err(TPMG_ERR_ARG, "NULL operator");
    if (prec == TPMG_DW && op->lsw_dw > op->g.L) prec = TPMG_F64;
    if (!r || !q || !z || !rr_out || !rz_out) return set_err(TPMG_ERR_ARG, "NULL argument");
    TRY(prep_unit(op, prec));
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    launch_set_ab(op->sc, alpha, 0.0, s);
    DISPATCH_PREC(prec, {
        Lv<P> LL = level_view<P>(op, L);
        auto* ri = in_ptr<P>(op, s, 0, r, n);
        auto* qi = in_ptr<P>(op, s, 1, q, n);
        auto* zo = out_ptr<P>(op, 2, z);
        const int nb = launch_cg_tridiag<P>(LL, op->sc, ri, qi, zo, op->partials, s);
        launch_finalize_norm(op->partials, nb, FIN_SUM, op->sc, nullptr, rr_out, s);
        launch_finalize_norm(op->partials + nb, nb, FIN_SUM, op->sc, nullptr, rz_out, s);
        out_back<P>(op, s, 0, r, n);
        out_back<P>(op, s, 2, z, n);
    });
    CK(cudaGetLastError());
    return TPMG_OK;
}

// ---------------------------------------------------------------- solvers
void tpmg_default_params(tpmg_params* p) {
    if (!p) return;
    p->nu_pre = 2;
    p->nu_post = 2;
    p->n_coarse = 2;
    p->max_iter = 100;
    p->rho = 0.8;
    p->tol = 1e-6;
    p->prec = TPMG_DW;
    p->use_graph = 1;
    p->timeout_s = 1.0;
    p->zero_guess = 0;
    p->coarse_bf16 = 0;
}

static tpmg_status panel_mg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, tpmg_info* info,
                                  void* stream);
static tpmg_status panel_cg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, tpmg_info* info,
                                  void* stream);

// The initial iterate: the caller's u, converted to the solve's storage, or zero without reading u.
static tpmg_status init_u_dw(size_t n, const tpmg_params* prm, const void* u, float2* uD, cudaStream_t s) {
    if (prm->zero_guess) CK(cudaMemsetAsync(uD, 0, n * sizeof(float2), s));
    else launch_f64_to_dw(n, (const double*)u, uD, s);
    return TPMG_OK;
}

static tpmg_status init_u(size_t n, size_t bytes, const tpmg_params* prm, void* u, cudaStream_t s) {
    if (prm->zero_guess) CK(cudaMemsetAsync(u, 0, n * bytes, s));
    return TPMG_OK;
}

tpmg_status tpmg_mg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, tpmg_info* info,
                          void* stream) {
    TRY(check_params(op, prm));
    if (!f || !u) return set_err(TPMG_ERR_ARG, "NULL field");
    if (op->panel) return panel_mg_solve(op, prm, f, u, info, stream);
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    TRY(ensure_history(op, prm->max_iter + 2));
    tpmg_precision prec = prm->prec;
    if (prec == TPMG_DW && op->lsw_dw > L) prec = TPMG_F64;  // no level where double-word suffices
    switch (prec) {
        case TPMG_F64:
            TRY(ensure_hier(op, 0, false));
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u(n, sizeof(double), prm, u, s));
            TRY((mg_loop<PolF64, PolF64>(op, prm, (double*)u, (double*)f, 1, s)));
            break;
        case TPMG_F32:
            TRY(ensure_hier(op, 1, false));
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u(n, sizeof(float), prm, u, s));
            TRY((mg_loop<PolF32, PolF32>(op, prm, (float*)u, (float*)f, 1, s)));
            break;
        case TPMG_DW: {
            TRY(ensure_hier(op, 2, true));
            TRY(ensure_hier(op, 0, false));
            float2* uD = (float2*)op->hier[2].u[L];
            float2* fD = (float2*)op->hier[2].f[L];
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u_dw(n, prm, u, uD, s));
            launch_f64_to_dw(n, (const double*)f, fD, s);
            TRY((mg_loop<PolDW, PolF64>(op, prm, uD, fD, op->lsw_dw, s)));
            launch_dw_to_f64(n, uD, (double*)u, s);
            break;
        }
        case TPMG_MIXED: {
            TRY(ensure_hier(op, 2, true));
            TRY(ensure_hier(op, 1, true));
            float2* uD = (float2*)op->hier[2].u[L];
            float2* fD = (float2*)op->hier[2].f[L];
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u_dw(n, prm, u, uD, s));
            launch_f64_to_dw(n, (const double*)f, fD, s);
            TRY(mixed_loop(op, prm, uD, fD, s));
            launch_dw_to_f64(n, uD, (double*)u, s);
            break;
        }
        default: return set_err(TPMG_ERR_ARG, "unknown precision");
    }
    CK(cudaEventRecord(op->ev1, s));
    CK(cudaGetLastError());
    return finish_info(op, info, s);
}

// Host fields (Sec. 5.1, "total solution time"): f is copied to the device -- transposed there
// from the vertically contiguous layout when asked --, the device solve runs, and u goes back the
// same way. Every step is ordered on `stream`.
tpmg_status tpmg_mg_solve_host(tpmg_op* op, const tpmg_params* prm, int layout, const void* f_host, void* u_host,
                               tpmg_info* info, double* ms_io, void* stream) {
    TRY(check_params(op, prm));
    if (!f_host || !u_host) return set_err(TPMG_ERR_ARG, "NULL field");
    if (layout != TPMG_LAYOUT_X && layout != TPMG_LAYOUT_Z) return set_err(TPMG_ERR_ARG, "unknown layout");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L), ncol = (size_t)op->g.nx * op->g.ny, nz = (size_t)op->g.nz;
    const bool f32 = prm->prec == TPMG_F32;
    const size_t eb = f32 ? sizeof(float) : sizeof(double), bytes = n * eb;
    // sized for 8-byte values whatever the precision, so a later call of another precision fits
    for (int t = 0; t < (layout == TPMG_LAYOUT_Z ? 3 : 2); ++t) TRY(dalloc(&op->hio[t], n * sizeof(double)));
    for (int t = 0; t < 4; ++t)
        if (!op->hev[t]) CK(cudaEventCreate(&op->hev[t]));
    void* fd = op->hio[0];
    void* ud = op->hio[1];
    // one field in: host -> device, then (z-contiguous host layout) columns-by-planes -> planes-by-columns
    auto field_in = [&](const void* h, void* d) -> tpmg_status {
        if (layout == TPMG_LAYOUT_X) {
            CK(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s));
        } else {
            CK(cudaMemcpyAsync(op->hio[2], h, bytes, cudaMemcpyHostToDevice, s));
            if (f32) launch_transpose<float>((const float*)op->hio[2], (float*)d, ncol, nz, s);
            else launch_transpose<double>((const double*)op->hio[2], (double*)d, ncol, nz, s);
        }
        return TPMG_OK;
    };
    CK(cudaEventRecord(op->hev[0], s));
    TRY(field_in(f_host, fd));
    if (!prm->zero_guess) TRY(field_in(u_host, ud));
    CK(cudaEventRecord(op->hev[1], s));
    tpmg_info inner{};
    if (info) {
        inner.history = info->history;
        inner.history_len = info->history_len;
    }
    const tpmg_status st = tpmg_mg_solve(op, prm, fd, ud, &inner, stream);
    if (st != TPMG_OK && st != TPMG_ERR_NOT_CONVERGED && st != TPMG_ERR_NONFINITE) return st;
    const std::string solve_err = g_err;
    CK(cudaEventRecord(op->hev[2], s));
    // u back (also on NOT_CONVERGED / NONFINITE: the last iterate, as tpmg_mg_solve leaves it)
    if (layout == TPMG_LAYOUT_X) {
        CK(cudaMemcpyAsync(u_host, ud, bytes, cudaMemcpyDeviceToHost, s));
    } else {
        if (f32) launch_transpose<float>((const float*)ud, (float*)op->hio[2], nz, ncol, s);
        else launch_transpose<double>((const double*)ud, (double*)op->hio[2], nz, ncol, s);
        CK(cudaMemcpyAsync(u_host, op->hio[2], bytes, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(op->hev[3], s));
    CK(cudaEventSynchronize(op->hev[3]));
    CK(cudaGetLastError());
    float t_all = 0, t_in = 0, t_out = 0;
    CK(cudaEventElapsedTime(&t_all, op->hev[0], op->hev[3]));
    CK(cudaEventElapsedTime(&t_in, op->hev[0], op->hev[1]));
    CK(cudaEventElapsedTime(&t_out, op->hev[2], op->hev[3]));
    if (info) {
        *info = inner;
        info->ms = t_all;
    }
    if (ms_io) *ms_io = (double)t_in + (double)t_out;
    if (st != TPMG_OK) return set_err(st, solve_err);
    return TPMG_OK;
}

tpmg_status tpmg_vcycle(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, void* stream) {
    TRY(flat_only(op));
    TRY(check_params(op, prm));
    if (!f || !u) return set_err(TPMG_ERR_ARG, "NULL field");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    auto one = [&](auto tagF, auto tagC, auto* A, auto* fL, int lsw) -> tpmg_status {
        typedef decltype(tagF) PF;
        typedef decltype(tagC) PC;
        typedef typename PF::S S;
        Cycle<PF, PC> c(op, prm, s, nullptr, lsw);
        c.u[L] = A;
        c.f[L] = fL;
        S* B = (S*)op->hier[PF::id].ub[L];
        launch_smooth<PF>(level_view<PF>(op, L), prm->rho, A, fL, B, nullptr, nullptr, s);
        void* cur = B;
        void* oth = A;
        c.rest(cur, oth);
        if (cur != (void*)A) launch_copy<PF>(n, (const S*)cur, A, nullptr, s);
        return TPMG_OK;
    };
    tpmg_precision prec = prm->prec;
    if (prec == TPMG_DW && op->lsw_dw > L) prec = TPMG_F64;
    switch (prec) {
        case TPMG_F64:
            TRY(ensure_hier(op, 0, false));
            TRY(one(PolF64(), PolF64(), (double*)u, (double*)f, 1));
            break;
        case TPMG_F32:
            TRY(ensure_hier(op, 1, false));
            TRY(one(PolF32(), PolF32(), (float*)u, (float*)f, 1));
            break;
        case TPMG_DW: {
            TRY(ensure_hier(op, 2, true));
            TRY(ensure_hier(op, 0, false));
            float2* uD = (float2*)op->hier[2].u[L];
            float2* fD = (float2*)op->hier[2].f[L];
            launch_f64_to_dw(n, (const double*)u, uD, s);
            launch_f64_to_dw(n, (const double*)f, fD, s);
            TRY(one(PolDW(), PolF64(), uD, fD, op->lsw_dw));
            launch_dw_to_f64(n, uD, (double*)u, s);
            break;
        }
        default: return set_err(TPMG_ERR_ARG, "tpmg_vcycle: precision must be TPMG_F64, TPMG_F32 or TPMG_DW");
    }
    CK(cudaGetLastError());
    return TPMG_OK;
}

unsigned long long tpmg_kernel_launches(void) { return launch_counter(); }

tpmg_status tpmg_set_variant(tpmg_op* op, tpmg_precision prec, int level, int variant) {
    TRY(flat_only(op));
    TRY(check_level(op, level));
    if (prec != TPMG_F64 && prec != TPMG_F32 && prec != TPMG_DW) return set_err(TPMG_ERR_ARG, "bad precision");
    if (variant < 0 || variant >= TPMG_NUM_VARIANTS) return set_err(TPMG_ERR_ARG, "bad variant");
    if (op->variant[pid_of(prec)][level] != variant) {
        op->variant[pid_of(prec)][level] = variant;
        invalidate_graphs(op);
    }
    return TPMG_OK;
}

tpmg_status tpmg_autotune(tpmg_op* op, tpmg_precision prec, int reps, int* variants_out, void* stream) {
    TRY(flat_only(op));
    if (!op || reps < 1) return set_err(TPMG_ERR_ARG, "NULL operator or reps < 1");
    if (prec != TPMG_F64 && prec != TPMG_F32 && prec != TPMG_DW) return set_err(TPMG_ERR_ARG, "bad precision");
    const int pid = pid_of(prec);
    TRY(ensure_hier(op, pid, true));
    cudaStream_t s = (cudaStream_t)stream;
    for (int l = 1; l <= op->g.L; ++l) {
        double best = 1e300;
        int best_v = 0;
        for (int v = 0; v < TPMG_NUM_VARIANTS; ++v) {
            if (v >= 8 && pid != 1) continue;  // the four-column tiles are FP32 only
            op->variant[pid][l] = v;
            auto run = [&](auto tag) {
                typedef decltype(tag) P;
                typedef typename P::S S;
                Hier& h = op->hier[pid];
                launch_smooth<P>(level_view<P>(op, l), 0.8, (const S*)h.u[l], (const S*)h.f[l], (S*)h.ub[l],
                                 op->partials, nullptr, s);
            };
            auto once = [&]() {
                if (pid == 0) run(PolF64());
                else if (pid == 1) run(PolF32());
                else run(PolDW());
            };
            once();
            CK(cudaEventRecord(op->ev0, s));
            for (int t = 0; t < reps; ++t) once();
            CK(cudaEventRecord(op->ev1, s));
            CK(cudaEventSynchronize(op->ev1));
            CK(cudaGetLastError());
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, op->ev0, op->ev1));
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        op->variant[pid][l] = best_v;
        if (variants_out) variants_out[l] = best_v;
    }
    invalidate_graphs(op);
    return TPMG_OK;
}

tpmg_status tpmg_time_kernel(tpmg_op* op, tpmg_precision prec, tpmg_kernel k, int reps, double* ms,
                             void* stream) {
    TRY(flat_only(op));
    if (!op || !ms || reps < 1) return set_err(TPMG_ERR_ARG, "NULL operator/output or reps < 1");
    if (prec != TPMG_F64 && prec != TPMG_F32 && prec != TPMG_DW)
        return set_err(TPMG_ERR_ARG, "precision must be TPMG_F64, TPMG_F32 or TPMG_DW");
    const int pid = pid_of(prec), L = op->g.L;
    if ((k == TPMG_K_RESTRICT_SMOOTH || k == TPMG_K_PROLONGATE || k == TPMG_K_RESIDUAL_RESTRICT) && L < 2)
        return set_err(TPMG_ERR_ARG, "transfer kernels need two levels");
    TRY(ensure_hier(op, pid, true));
    TRY(ensure_cg(op, pid));
    TRY(ensure_history(op, 16));
    cudaStream_t s = (cudaStream_t)stream;
    launch_scalars_init(op->sc, 0.0, 1, s);
    const size_t n = lvl_cells(op, L);
    bool bad = false;  // the kernel does not apply to this operator's levels
    auto run = [&](auto tag) {
        typedef decltype(tag) P;
        typedef typename P::S S;
        Hier& h = op->hier[pid];
        S* a = (S*)h.u[L];
        S* f = (S*)h.f[L];
        S* b = (S*)h.ub[L];
        S* r = (S*)h.r[L];
        S** cg = (S**)op->cgbuf[pid];
        Lv<P> LL = level_view<P>(op, L);
        switch (k) {
            case TPMG_K_SMOOTH: launch_smooth<P>(LL, 0.8, a, f, b, op->partials, nullptr, s); break;
            case TPMG_K_RESIDUAL: launch_residual<P, P>(LL, a, f, r, op->partials, nullptr, s); break;
            case TPMG_K_APPLY_A: launch_apply_A<P>(LL, a, b, s); break;
            case TPMG_K_LINE_SOLVE: launch_line_solve<P>(LL, f, b, 1.0, nullptr, s); break;
            case TPMG_K_RESTRICT_SMOOTH:
                launch_restrict_smooth<P, P>(level_view<P>(op, L - 1), 0.8, r, (S*)h.f[L - 1], (S*)h.u[L - 1], nullptr, s);
                break;
            case TPMG_K_PROLONGATE:
                launch_prolongate<P, P>(op->g.lnx[L - 1], op->g.lny[L - 1], op->g.nz, (S*)h.u[L - 1], a, nullptr, s);
                break;
            case TPMG_K_CG_SPMV: launch_cg_spmv<P>(LL, op->sc, cg[0], cg[2], cg[1], cg[3], op->partials, s); break;
            case TPMG_K_CG_TRIDIAG: launch_cg_tridiag<P>(LL, op->sc, cg[0], cg[3], cg[1], op->partials, s); break;
            case TPMG_K_RESIDUAL_RESTRICT:
                if (launch_residual_restrict<P>(LL, level_view<P>(op, L - 1), 0.8, a, f, (S*)h.f[L - 1],
                                                (S*)h.u[L - 1], nullptr, s) < 0)
                    bad = true;
                break;
            default: break;
        }
        (void)n;
    };
    if (k < 0 || k >= TPMG_K_COUNT) return set_err(TPMG_ERR_ARG, "unknown kernel id");
    auto once = [&]() {
        if (pid == 0) run(PolF64());
        else if (pid == 1) run(PolF32());
        else run(PolDW());
    };
    once();  // warm-up
    if (bad) return set_err(TPMG_ERR_ARG, "the fused kernel does not apply to this operator's finest levels");
    CK(cudaEventRecord(op->ev0, s));
    for (int t = 0; t < reps; ++t) once();
    CK(cudaEventRecord(op->ev1, s));
    CK(cudaEventSynchronize(op->ev1));
    CK(cudaGetLastError());
    float t_ms = 0;
    CK(cudaEventElapsedTime(&t_ms, op->ev0, op->ev1));
    *ms = t_ms / reps;
    return TPMG_OK;
}

tpmg_status tpmg_cg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, tpmg_info* info,
                          void* stream) {
    TRY(check_params(op, prm));
    if (!f || !u) return set_err(TPMG_ERR_ARG, "NULL field");
    if (op->panel) return panel_cg_solve(op, prm, f, u, info, stream);
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    TRY(ensure_history(op, prm->max_iter + 2));
    tpmg_precision prec = prm->prec;
    if (prec == TPMG_DW && op->lsw_dw > L) prec = TPMG_F64;
    switch (prec) {
        case TPMG_F64:
            TRY(ensure_cg(op, 0));
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u(n, sizeof(double), prm, u, s));
            TRY(cg_loop<PolF64>(op, prm, (double*)u, (const double*)f, s));
            break;
        case TPMG_F32:
            TRY(ensure_cg(op, 1));
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u(n, sizeof(float), prm, u, s));
            TRY(cg_loop<PolF32>(op, prm, (float*)u, (const float*)f, s));
            break;
        case TPMG_DW: {
            TRY(ensure_cg(op, 2));
            float2* uD = (float2*)op->hier[2].u[L];
            float2* fD = (float2*)op->hier[2].f[L];
            CK(cudaEventRecord(op->ev0, s));
            TRY(init_u_dw(n, prm, u, uD, s));
            launch_f64_to_dw(n, (const double*)f, fD, s);
            TRY(cg_loop<PolDW>(op, prm, uD, fD, s));
            launch_dw_to_f64(n, uD, (double*)u, s);
            break;
        }
        default: return set_err(TPMG_ERR_ARG, "tpmg_cg_solve: precision must be TPMG_F64, TPMG_F32 or TPMG_DW");
    }
    CK(cudaEventRecord(op->ev1, s));
    CK(cudaGetLastError());
    return finish_info(op, info, s);
}

}  // extern "C"

// ================================================================ batched persistent solver
// Tables for k_batched (see kernels.cuh): per problem its level descriptors and buffers, per phase
// the tasks of all problems; built once per set of operators and parameters and kept with a CUDA
// graph of the whole batched solve (conversions in, one persistent launch, conversions out).
struct BatchCache {
    std::vector<tpmg_op*> ops;
    int nu_pre = 0, nu_post = 0, n_coarse = 0, max_iter = 0;
    double rho = 0, tol = 0, timeout_s = 0;
    std::vector<const void*> io_key;
    int nprob = 0, nphase = 0, ntasks = 0, total_parts = 0, nz_max = 0, grid = 0;
    size_t smem = 0;
    BProbDesc* d_probs = nullptr;
    BState* d_state = nullptr;
    BState* h_state = nullptr;  // pinned: initial state (copied in each solve) and results
    BTask* d_tasks = nullptr;
    int* d_phase_begin = nullptr;
    int* d_phase_tiles = nullptr;
    double* d_partials = nullptr;
    unsigned* d_bar = nullptr;  // count, generation
    int* d_flags = nullptr;     // error, n_active
    int* h_flags = nullptr;     // pinned: initial flags and results
    double* d_hist = nullptr;
    float* d_scratch = nullptr;  // the persistent blocks' Thomas stacks
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_kernels = 0;
    std::vector<BTask> h_tasks;
    std::vector<int> h_phase_begin, h_phase_tiles;
    ~BatchCache() {
        if (graph) cudaGraphExecDestroy(graph);
        void* ptrs[] = {d_probs,    d_state, d_tasks, d_phase_begin, d_phase_tiles, d_partials,
                        d_bar,      d_flags, d_hist,  d_scratch};
        for (void* p : ptrs) dev_free(p);
        if (h_state) cudaFreeHost(h_state);
        if (h_flags) cudaFreeHost(h_flags);
    }
};
static std::vector<BatchCache*> g_batches;

static void drop_batches_of(const tpmg_op* op) {
    for (size_t i = 0; i < g_batches.size();) {
        bool uses = false;
        for (tpmg_op* o : g_batches[i]->ops) uses |= (o == op);
        if (uses) {
            delete g_batches[i];
            g_batches.erase(g_batches.begin() + i);
        } else {
            ++i;
        }
    }
}

// the FP32 inner V-cycle of problem b as a list of tasks (same steps and buffers as Cycle)
static void cycle_tasks(tpmg_op* op, int b, const tpmg_params* prm, std::vector<BTask>& out) {
    Hier& h = op->hier[1];
    const int L = op->g.L;
    auto task = [&](int type, int level, const void* a, const void* rhs, void* o, void* o2) {
        BTask t;
        t.type = type;
        t.prob = b;
        t.level = level;
        t.a = a;
        t.b = rhs;
        t.out = o;
        t.out2 = o2;
        const int nxl = op->g.lnx[level];
        const int nyl = op->g.lny[level];
        t.x2 = (type == BT_SMOOTH || type == BT_RESID || type == BT_LS0 || type == BT_RRS) &&
               batched_x2_fits(nxl, nyl, a ? a : rhs, rhs, type == BT_RRS ? a : o);
        t.tiles_x = t.x2 ? nxl / 64 : (nxl + 31) / 32;
        t.tiles_y = (nyl + BTY - 1) / BTY;
        t.tile_base = 0;
        out.push_back(t);
    };
    void* cur = h.u[L];
    void* oth = h.ub[L];
    auto smooth = [&](int l, void*& c, void*& o, const void* rhs) {
        task(BT_SMOOTH, l, c, rhs, o, nullptr);
        std::swap(c, o);
    };
    task(BT_LS0, L, nullptr, h.f[L], cur, nullptr);
    if (L == 1) {
        for (int s = 1; s < prm->n_coarse; ++s) smooth(L, cur, oth, h.f[L]);
    } else {
        for (int s = 1; s < prm->nu_pre; ++s) smooth(L, cur, oth, h.f[L]);
        std::vector<void*> lcur(L + 1), loth(L + 1);
        for (int l = 1; l < L; ++l) {
            lcur[l] = h.u[l];
            loth[l] = h.ub[l];
        }
        // Residual of level l, then RestrictSmooth onto l-1: one fused task where level l takes
        // two-column tiles (the same arithmetic), else the two tasks; returns whether it fused
        auto residual_restrict = [&](int l, const void* u_l) {
            if (op->fuse_restrict && batched_x2_fits(op->g.lnx[l], op->g.lny[l], u_l, h.f[l], u_l)) {
                task(BT_RRS, l, u_l, h.f[l], h.f[l - 1], lcur[l - 1]);
                return true;
            }
            task(BT_RESID, l, u_l, h.f[l], h.r[l], nullptr);
            return false;
        };
        bool restricted = residual_restrict(L, cur);
        // descend
        for (int l = L - 1; l >= 1; --l) {
            if (!restricted) task(BT_RS, l, h.r[l + 1], nullptr, h.f[l], lcur[l]);
            if (l == 1) {
                for (int s = 1; s < prm->n_coarse; ++s) smooth(l, lcur[l], loth[l], h.f[l]);
            } else {
                for (int s = 1; s < prm->nu_pre; ++s) smooth(l, lcur[l], loth[l], h.f[l]);
                restricted = residual_restrict(l, lcur[l]);
            }
        }
        // ascend
        for (int l = 2; l < L; ++l) {
            task(BT_PROL, l, lcur[l - 1], nullptr, lcur[l], nullptr);
            for (int s = 0; s < prm->nu_post; ++s) smooth(l, lcur[l], loth[l], h.f[l]);
        }
        task(BT_PROL, L, lcur[L - 1], nullptr, cur, nullptr);
        for (int s = 0; s < prm->nu_post; ++s) smooth(L, cur, oth, h.f[L]);
    }
    task(BT_CORR, L, cur, nullptr, nullptr, nullptr);
}

static tpmg_status build_batch(BatchCache* bc, const tpmg_params* prm) {
    const int np = (int)bc->ops.size();
    bc->nprob = np;
    std::vector<BProbDesc> probs(np);
    std::vector<std::vector<BTask>> lists(np);
    int parts = 0, maxlen = 0, nz_max = 1;
    for (int b = 0; b < np; ++b) {
        tpmg_op* op = bc->ops[b];
        const int L = op->g.L;
        BProbDesc& pd = probs[b];
        memset(&pd, 0, sizeof(pd));
        pd.L = L;
        pd.nz = op->g.nz;
        nz_max = op->g.nz > nz_max ? op->g.nz : nz_max;
        for (int l = 1; l <= L; ++l) {
            BLevelDesc& ld = pd.lev[l];
            ld.nx = op->g.lnx[l];
            ld.ny = op->g.lny[l];
            ld.nz = op->g.nz;
            ld.percol = op->percol[l];
            ld.cx = op->cx[l];
            ld.cy = op->cy[l];
            ld.v = op->v32[l];
            ld.finv = (const float*)op->finv[1][l];
            ld.fw = (const float*)op->fw[1][l];
            ld.k1 = sweep_k<PolF32>(op->cx[l], op->cy[l], 1.0);
            ld.krho = sweep_k<PolF32>(op->cx[l], op->cy[l], prm->rho);
        }
        pd.kD = sweep_k<PolDW>(op->cx[L], op->cy[L], 1.0);
        pd.uD = (float2*)op->hier[2].u[L];
        pd.fD = (const float2*)op->hier[2].f[L];
        pd.vD = op->vdw[L];
        pd.r32 = (float*)op->hier[1].f[L];
        pd.fine_x2 = batched_x2_fits(op->g.lnx[L], op->g.lny[L], pd.uD, pd.fD, pd.r32) ? 1 : 0;
        pd.fine_tiles = (pd.fine_x2 ? op->g.lnx[L] / 64 : (op->g.lnx[L] + 31) / 32) * ((op->g.lny[L] + BTY - 1) / BTY);
        pd.part_base = parts;
        parts += pd.fine_tiles;
        cycle_tasks(op, b, prm, lists[b]);
        maxlen = (int)lists[b].size() > maxlen ? (int)lists[b].size() : maxlen;
    }
    bc->nz_max = nz_max;
    bc->total_parts = parts;
    // phases: outer residual, convergence decision, then the p-th step of every problem's cycle
    std::vector<BTask>& tasks = bc->h_tasks;
    tasks.clear();
    bc->h_phase_begin.clear();
    bc->h_phase_tiles.clear();
    auto close_phase = [&](size_t first) {
        int tiles = 0;
        for (size_t t = first; t < tasks.size(); ++t) {
            tasks[t].tile_base = tiles;
            tiles += tasks[t].tiles_x * tasks[t].tiles_y;
        }
        bc->h_phase_tiles.push_back(tiles);
    };
    for (int ph = 0; ph < 2 + maxlen; ++ph) {
        const size_t first = tasks.size();
        bc->h_phase_begin.push_back((int)first);
        for (int b = 0; b < np; ++b) {
            tpmg_op* op = bc->ops[b];
            BTask t;
            memset(&t, 0, sizeof(t));
            t.prob = b;
            t.level = op->g.L;
            if (ph < 2) {
                t.type = ph == 0 ? BT_OUTRES : BT_FINAL;
                t.x2 = ph == 0 ? probs[b].fine_x2 : 0;
                t.tiles_x = ph == 0 ? (t.x2 ? op->g.lnx[op->g.L] / 64 : (op->g.lnx[op->g.L] + 31) / 32) : 1;
                t.tiles_y = ph == 0 ? (op->g.lny[op->g.L] + BTY - 1) / BTY : 1;
                tasks.push_back(t);
            } else if (ph - 2 < (int)lists[b].size()) {
                tasks.push_back(lists[b][ph - 2]);
            }
        }
        close_phase(first);
    }
    bc->h_phase_begin.push_back((int)tasks.size());
    bc->nphase = (int)bc->h_phase_tiles.size();
    bc->ntasks = (int)tasks.size();
    // device tables
    const int hist_len = prm->max_iter + 1;
    for (int b = 0; b < np; ++b) probs[b].history = nullptr;  // set below once d_hist exists
    TRY(dalloc((void**)&bc->d_hist, sizeof(double) * (size_t)np * hist_len));
    for (int b = 0; b < np; ++b) probs[b].history = bc->d_hist + (size_t)b * hist_len;
    TRY(dalloc((void**)&bc->d_probs, sizeof(BProbDesc) * np));
    TRY(dalloc((void**)&bc->d_state, sizeof(BState) * np));
    TRY(dalloc((void**)&bc->d_tasks, sizeof(BTask) * tasks.size()));
    TRY(dalloc((void**)&bc->d_phase_begin, sizeof(int) * bc->h_phase_begin.size()));
    TRY(dalloc((void**)&bc->d_phase_tiles, sizeof(int) * bc->h_phase_tiles.size()));
    TRY(dalloc((void**)&bc->d_partials, sizeof(double) * (parts > 0 ? parts : 1)));
    TRY(dalloc((void**)&bc->d_bar, sizeof(unsigned) * 2));
    TRY(dalloc((void**)&bc->d_flags, sizeof(int) * 2));
    CK(cudaMallocHost((void**)&bc->h_state, sizeof(BState) * np));
    CK(cudaMallocHost((void**)&bc->h_flags, sizeof(int) * 2));
    CK(cudaMemcpy(bc->d_probs, probs.data(), sizeof(BProbDesc) * np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(bc->d_tasks, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(bc->d_phase_begin, bc->h_phase_begin.data(), sizeof(int) * bc->h_phase_begin.size(),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(bc->d_phase_tiles, bc->h_phase_tiles.data(), sizeof(int) * bc->h_phase_tiles.size(),
                  cudaMemcpyHostToDevice));
    bc->smem = batched_smem_bytes();
    int per_sm = batched_blocks_per_sm();
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, bc->ops[0]->device));
    if (per_sm < 1) return set_err(TPMG_ERR_ARG, "batched kernel does not fit on an SM");
    bc->grid = per_sm * nsm;
    TRY(dalloc((void**)&bc->d_scratch, sizeof(float) * batched_scratch_floats(bc->grid, nz_max)));
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_mg_solve_batched(int nprob, tpmg_op* const* ops, const tpmg_params* prm,
                                             const double* const* f, double* const* u, tpmg_info* infos,
                                             void* stream) {
    if (nprob < 1 || !ops || !prm || !f || !u) return set_err(TPMG_ERR_ARG, "bad batched arguments");
    if (prm->prec != TPMG_MIXED) return set_err(TPMG_ERR_ARG, "the batched solver runs TPMG_MIXED");
    if (prm->nu_pre < 1 || prm->nu_post < 0 || prm->n_coarse < 1 || prm->max_iter < 0 || !(prm->rho > 0.0))
        return set_err(TPMG_ERR_ARG, "bad multigrid parameters");
    const int dev = ops[0]->device;
    for (int b = 0; b < nprob; ++b) {
        if (!ops[b] || !f[b] || !u[b]) return set_err(TPMG_ERR_ARG, "NULL operator or field");
        TRY(flat_only(ops[b]));
        if (ops[b]->device != dev) return set_err(TPMG_ERR_ARG, "all operators must live on one device");
        for (int c = 0; c < b; ++c)
            if (ops[c] == ops[b]) return set_err(TPMG_ERR_ARG, "an operator appears twice in the batch");
        TRY(ensure_hier(ops[b], 2, true));
        TRY(ensure_hier(ops[b], 1, true));
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double timeout_s = prm->timeout_s >= 0.0 ? prm->timeout_s : 1.0;
    // find or build the tables
    BatchCache* bc = nullptr;
    for (BatchCache* c : g_batches) {
        if ((int)c->ops.size() != nprob || c->nu_pre != prm->nu_pre || c->nu_post != prm->nu_post ||
            c->n_coarse != prm->n_coarse || c->max_iter != prm->max_iter || c->rho != prm->rho || c->tol != prm->tol ||
            c->timeout_s != timeout_s)
            continue;
        bool same = true;
        for (int b = 0; b < nprob && same; ++b) same = c->ops[b] == ops[b];
        if (same) bc = c;
    }
    if (!bc) {
        bc = new BatchCache();
        bc->ops.assign(ops, ops + nprob);
        bc->nu_pre = prm->nu_pre;
        bc->nu_post = prm->nu_post;
        bc->n_coarse = prm->n_coarse;
        bc->max_iter = prm->max_iter;
        bc->rho = prm->rho;
        bc->tol = prm->tol;
        bc->timeout_s = timeout_s;
        tpmg_status st = build_batch(bc, prm);
        if (st != TPMG_OK) {
            delete bc;
            return st;
        }
        g_batches.push_back(bc);
    }
    for (int b = 0; b < nprob; ++b) {
        memset(&bc->h_state[b], 0, sizeof(BState));
        bc->h_state[b].active = 1;
    }
    bc->h_flags[0] = 0;
    bc->h_flags[1] = nprob;
    BatchDesc d;
    d.nprob = nprob;
    d.ntasks = bc->ntasks;
    d.nphase = bc->nphase;
    d.probs = bc->d_probs;
    d.state = bc->d_state;
    d.tasks = bc->d_tasks;
    d.phase_begin = bc->d_phase_begin;
    d.phase_tiles = bc->d_phase_tiles;
    d.partials = bc->d_partials;
    d.bar_count = bc->d_bar;
    d.bar_gen = bc->d_bar + 1;
    d.error = bc->d_flags;
    d.n_active = bc->d_flags + 1;
    d.rho = prm->rho;
    d.tol = prm->tol;
    d.max_iter = prm->max_iter;
    d.timeout_ns = (unsigned long long)(timeout_s * 1e9);
    d.nz_max = bc->nz_max;
    d.scratch = bc->d_scratch;
    std::vector<const void*> io_key;
    for (int b = 0; b < nprob; ++b) {
        io_key.push_back(f[b]);
        io_key.push_back(u[b]);
    }
    io_key.push_back(prm->zero_guess ? (const void*)1 : nullptr);  // the graph holds a memset instead of u's conversion
    cudaError_t launch_err = cudaSuccess;
    auto body = [&](cudaStream_t st) {
        CK(cudaMemcpyAsync(bc->d_state, bc->h_state, sizeof(BState) * nprob, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(bc->d_flags, bc->h_flags, sizeof(int) * 2, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(bc->d_bar, 0, sizeof(unsigned) * 2, st));
        for (int b = 0; b < nprob; ++b) {
            const size_t n = lvl_cells(ops[b], ops[b]->g.L);
            launch_f64_to_dw(n, f[b], (float2*)ops[b]->hier[2].f[ops[b]->g.L], st);
            if (prm->zero_guess)
                CK(cudaMemsetAsync(ops[b]->hier[2].u[ops[b]->g.L], 0, n * sizeof(float2), st));
            else
                launch_f64_to_dw(n, u[b], (float2*)ops[b]->hier[2].u[ops[b]->g.L], st);
        }
        launch_err = launch_batched(d, bc->grid, bc->smem, st);
        for (int b = 0; b < nprob; ++b) {
            const size_t n = lvl_cells(ops[b], ops[b]->g.L);
            launch_dw_to_f64(n, (const float2*)ops[b]->hier[2].u[ops[b]->g.L], u[b], st);
        }
        return TPMG_OK;
    };
    tpmg_op* op0 = ops[0];
    CK(cudaEventRecord(op0->ev0, s));
    bool ran = false;
    if (prm->use_graph) {
        if (!bc->graph || bc->io_key != io_key) {
            if (bc->graph) cudaGraphExecDestroy(bc->graph);
            bc->graph = nullptr;
            if (cudaStreamBeginCapture(op0->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                const unsigned long long c0 = launch_counter();
                body(op0->cap_stream);
                bc->graph_kernels = launch_counter() - c0;
                launch_counter() = c0;
                cudaGraph_t g = nullptr;
                if (cudaStreamEndCapture(op0->cap_stream, &g) == cudaSuccess && launch_err == cudaSuccess &&
                    cudaGraphInstantiate(&bc->graph, g, 0) == cudaSuccess) {
                    bc->io_key = io_key;
                } else {
                    bc->graph = nullptr;
                }
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();  // a failed capture falls back to direct launches
        }
        if (bc->graph) {
            CK(cudaGraphLaunch(bc->graph, s));
            launch_counter() += bc->graph_kernels;
            ran = true;
        }
    }
    if (!ran) {
        launch_err = cudaSuccess;
        TRY(body(s));
        if (launch_err != cudaSuccess)
            return set_err(TPMG_ERR_CUDA, std::string("cooperative launch: ") + cudaGetErrorString(launch_err));
    }
    CK(cudaEventRecord(op0->ev1, s));
    CK(cudaMemcpyAsync(bc->h_state, bc->d_state, sizeof(BState) * nprob, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(bc->h_flags, bc->d_flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, op0->ev0, op0->ev1));
    bool any_nonfinite = false, all_conv = true;
    for (int b = 0; b < nprob; ++b) {
        const BState& stt = bc->h_state[b];
        any_nonfinite |= stt.nonfinite != 0;
        all_conv &= stt.converged != 0;
        if (infos) {
            tpmg_info& in = infos[b];
            in.iters = stt.iters;
            in.converged = stt.converged;
            in.rel_res = stt.rel;
            in.r0 = stt.r0;
            in.ms = ms;
            if (in.history && in.history_len > 0) {
                int nh = stt.iters + 1 < in.history_len ? stt.iters + 1 : in.history_len;
                CK(cudaMemcpy(in.history, bc->d_hist + (size_t)b * (prm->max_iter + 1), sizeof(double) * nh,
                              cudaMemcpyDeviceToHost));
            }
        }
    }
    if (bc->h_flags[0]) return set_err(TPMG_ERR_TIMEOUT, "a grid barrier wait of the batched solver timed out");
    if (any_nonfinite) return set_err(TPMG_ERR_NONFINITE, "non-finite residual in a batched problem");
    if (!all_conv) return set_err(TPMG_ERR_NOT_CONVERGED, "max_iter reached for a batched problem");
    return TPMG_OK;
}

// ================================================================ learned stage and flexible CG
#include "fcg.cuh"
#include "nn.cuh"

struct tpmg_nn {
    NNBufs b;
    int adam_t = 0;
    bool weights_ready = false;
};

static tpmg_status nn_ensure_cap(tpmg_nn* nn, size_t n) {
    NNBufs& b = nn->b;
    if (n <= b.ncap) return TPMG_OK;
    void* ptrs[] = {b.a1, b.a2, b.a3, b.d1, b.d2, b.x, b.out, b.d4, b.tmp};
    for (void* p : ptrs) dev_free(p);
    b.a1 = b.a2 = b.a3 = b.d1 = b.d2 = b.x = nullptr;
    b.out = b.d4 = b.tmp = nullptr;
    b.ncap = 0;
    TRY(dalloc((void**)&b.a1, n * 32));
    TRY(dalloc((void**)&b.a2, n * 32));
    TRY(dalloc((void**)&b.a3, n * 32));
    TRY(dalloc((void**)&b.d1, n * 32));
    TRY(dalloc((void**)&b.d2, n * 32));
    TRY(dalloc((void**)&b.x, n * 2 * (size_t)b.cin));
    TRY(dalloc((void**)&b.out, n * 4));
    TRY(dalloc((void**)&b.d4, n * 4));
    TRY(dalloc((void**)&b.tmp, n * 4));
    b.ncap = n;
    return TPMG_OK;
}

static tpmg_status nn_check_shape(int nx, int ny, int nz) {
    if (nx < 64 || nx % 64 != 0 || ny < 2 || ny % 2 != 0 || nz < 1)
        return set_err(TPMG_ERR_ARG, "the network kernels need nx a multiple of 64 and ny even");
    return TPMG_OK;
}

static void nn_refresh(tpmg_nn* nn, cudaStream_t s) {
    nn_prepare_weights(nn->b, s);
    nn->weights_ready = true;
}

extern "C" {

int tpmg_nn_nparams(int cin) { return 16 * cin * 27 + 16 + 2 * (16 * 16 * 27 + 16) + 16 * 27 + 1; }

tpmg_status tpmg_nn_create(int cin, const float* params_host, tpmg_nn** out) {
    if (!out || (cin != 1 && cin != 2)) return set_err(TPMG_ERR_ARG, "cin must be 1 or 2");
    tpmg_nn* nn = new tpmg_nn();
    memset(&nn->b, 0, sizeof(NNBufs));
    NNBufs& b = nn->b;
    b.cin = cin;
    b.nparams = tpmg_nn_nparams(cin);
    const size_t np = (size_t)b.nparams;
    tpmg_status st = TPMG_OK;
    void** bufs[] = {(void**)&b.params, (void**)&b.grad, (void**)&b.adam_m, (void**)&b.adam_v};
    for (void** q : bufs)
        if ((st = dalloc(q, np * sizeof(float))) != TPMG_OK) break;
    void** wb[] = {(void**)&b.w1, (void**)&b.w2f, (void**)&b.w2b, (void**)&b.w3f, (void**)&b.w3b, (void**)&b.w4};
    for (void** q : wb)
        if (st == TPMG_OK) st = dalloc(q, 16 * 16 * 27 * 2);
    if (st == TPMG_OK) st = dalloc((void**)&b.part, sizeof(float) * 1024 * 16 * 16 * 27);
    if (st == TPMG_OK) st = dalloc((void**)&b.dpart, sizeof(double) * 4096);
    if (st == TPMG_OK) st = dalloc((void**)&b.err, sizeof(int));
    if (st == TPMG_OK && cudaMemset(b.err, 0, sizeof(int)) != cudaSuccess) st = set_err(TPMG_ERR_CUDA, "memset failed");
    if (st == TPMG_OK && params_host)
        if (cudaMemcpy(b.params, params_host, np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            st = set_err(TPMG_ERR_CUDA, "parameter upload failed");
    if (st != TPMG_OK) {
        tpmg_nn_destroy(nn);
        return st;
    }
    *out = nn;
    return TPMG_OK;
}

tpmg_status tpmg_nn_destroy(tpmg_nn* nn) {
    if (!nn) return TPMG_OK;
    cudaDeviceSynchronize();
    NNBufs& b = nn->b;
    void* ptrs[] = {b.params, b.grad, b.adam_m, b.adam_v, b.w1, b.w2f, b.w2b, b.w3f, b.w3b, b.w4,
                    b.a1,     b.a2,   b.a3,     b.d1,     b.d2, b.x,   b.out, b.d4,  b.part, b.dpart, b.tmp, b.err};
    for (void* p : ptrs) dev_free(p);
    delete nn;
    return TPMG_OK;
}

// TPMG_ERR_TIMEOUT if a tensor-core convolution of this network gave up a wait (synchronises)
static tpmg_status nn_check(const tpmg_nn* nn) {
    int e = 0;
    CK(cudaMemcpy(&e, nn->b.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return set_err(TPMG_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
    return TPMG_OK;
}

tpmg_status tpmg_nn_get_params(const tpmg_nn* nn, float* host) {
    if (!nn || !host) return set_err(TPMG_ERR_ARG, "NULL network or buffer");
    CK(cudaMemcpy(host, nn->b.params, sizeof(float) * nn->b.nparams, cudaMemcpyDeviceToHost));
    return nn_check(nn);
}

tpmg_status tpmg_nn_set_params(tpmg_nn* nn, const float* host) {
    if (!nn || !host) return set_err(TPMG_ERR_ARG, "NULL network or buffer");
    CK(cudaMemcpy(nn->b.params, host, sizeof(float) * nn->b.nparams, cudaMemcpyHostToDevice));
    CK(cudaMemset(nn->b.adam_m, 0, sizeof(float) * nn->b.nparams));
    CK(cudaMemset(nn->b.adam_v, 0, sizeof(float) * nn->b.nparams));
    nn->adam_t = 0;
    nn->weights_ready = false;
    return TPMG_OK;
}

// x: DEVICE fp32, channels-last (cin values per cell)
static tpmg_status nn_load_input(tpmg_nn* nn, size_t n, const float* x, cudaStream_t s);

tpmg_status tpmg_nn_forward(tpmg_nn* nn, int nx, int ny, int nz, const float* x, float* out, void* stream) {
    if (!nn || !x || !out) return set_err(TPMG_ERR_ARG, "NULL argument");
    TRY(nn_check_shape(nx, ny, nz));
    const size_t n = (size_t)nx * ny * nz;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(nn_ensure_cap(nn, n));
    if (!nn->weights_ready) nn_refresh(nn, s);
    TRY(nn_load_input(nn, n, x, s));
    nn_forward(nn->b, nx, ny, nz, nn->b.x, out, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_nn_loss_grad(tpmg_nn* nn, int nx, int ny, int nz, const float* x, const float* target,
                              double* loss_out, float* grad_out, void* stream) {
    if (!nn || !x || !target || !loss_out) return set_err(TPMG_ERR_ARG, "NULL argument");
    TRY(nn_check_shape(nx, ny, nz));
    const size_t n = (size_t)nx * ny * nz;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(nn_ensure_cap(nn, n));
    if (!nn->weights_ready) nn_refresh(nn, s);
    TRY(nn_load_input(nn, n, x, s));
    NNBufs& b = nn->b;
    nn_forward(b, nx, ny, nz, b.x, b.out, s);
    const int nbl = 2048;
    nn_mse(b.out, target, b.d4, b.dpart, n, nbl, s);
    launch_finalize_norm(b.dpart, nbl, FIN_SUM, nullptr, nullptr, loss_out, s);
    nn_backward(b, nx, ny, nz, b.x, b.d4, grad_out ? grad_out : b.grad, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_nn_train_step(tpmg_nn* nn, int nx, int ny, int nz, const float* x, const float* target, double lr,
                               double* loss_out, void* stream) {
    TRY(tpmg_nn_loss_grad(nn, nx, ny, nz, x, target, loss_out, nullptr, stream));
    cudaStream_t s = (cudaStream_t)stream;
    NNBufs& b = nn->b;
    nn_adam(b.nparams, b.params, b.grad, b.adam_m, b.adam_v, (float)lr, ++nn->adam_t, s);
    nn_refresh(nn, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

// Residual loss mean((r - A D^{-1} NN(x))^2) on the finest level of op (FP32 operator, D = diag(A)),
// r = channel 0 of x; its gradient w.r.t. the output is -2 D^{-1} A (r - A D^{-1} NN(x)) / n.
tpmg_status tpmg_nn_loss_grad_residual(tpmg_nn* nn, tpmg_op* op, const float* x, double* loss_out, float* grad_out,
                                       void* stream) {
    TRY(flat_only(op));
    if (!nn || !op || !x || !loss_out) return set_err(TPMG_ERR_ARG, "NULL argument");
    const int L = op->g.L, nx = op->g.nx, ny = op->g.ny, nz = op->g.nz;
    TRY(nn_check_shape(nx, ny, nz));
    TRY(prep_unit(op, TPMG_F32));
    const size_t n = (size_t)nx * ny * nz;
    cudaStream_t s = (cudaStream_t)stream;
    TRY(nn_ensure_cap(nn, n));
    if (!nn->weights_ready) nn_refresh(nn, s);
    TRY(nn_load_input(nn, n, x, s));
    NNBufs& b = nn->b;
    const Lv<PolF32> LF = level_view<PolF32>(op, L);
    const size_t ncol = (size_t)nx * ny;
    nn_forward(b, nx, ny, nz, b.x, b.out, s);
    nn_scale_dinv(n, ncol, nz, LF.cx, LF.cy, LF.v, b.out, b.tmp, s);  // D^{-1} y
    launch_apply_A<PolF32>(LF, b.tmp, b.d4, s);                      // q = A D^{-1} y
    const int nbl = 2048;
    nn_res_loss(b.x, b.cin, b.d4, b.tmp, b.dpart, n, nbl, s);  // tmp = -2 (r - q) / n
    launch_finalize_norm(b.dpart, nbl, FIN_SUM, nullptr, nullptr, loss_out, s);
    launch_apply_A<PolF32>(LF, b.tmp, b.out, s);                   // A tmp
    nn_scale_dinv(n, ncol, nz, LF.cx, LF.cy, LF.v, b.out, b.d4, s);  // dLoss/dy = D^{-1} A tmp
    nn_backward(b, nx, ny, nz, b.x, b.d4, grad_out ? grad_out : b.grad, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

tpmg_status tpmg_nn_train_step_residual(tpmg_nn* nn, tpmg_op* op, const float* x, double lr, double* loss_out,
                                        void* stream) {
    TRY(tpmg_nn_loss_grad_residual(nn, op, x, loss_out, nullptr, stream));
    cudaStream_t s = (cudaStream_t)stream;
    NNBufs& b = nn->b;
    nn_adam(b.nparams, b.params, b.grad, b.adam_m, b.adam_v, (float)lr, ++nn->adam_t, s);
    nn_refresh(nn, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

}  // extern "C"

// the FP32 input rounded to BF16 (round to nearest even), four values per thread and step where the
// buffer allows 16-byte loads, one at a time otherwise
__global__ void k_nn_input_f32(size_t m, const float* __restrict__ x, __nv_bfloat16* __restrict__ xb) {
    const size_t stride = (size_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if ((m & 3) == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)xb & 7) == 0) {
        for (size_t t = t0; t < m / 4; t += stride) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(x) + t);
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 o;
            o.x = *reinterpret_cast<uint32_t*>(&lo);
            o.y = *reinterpret_cast<uint32_t*>(&hi);
            reinterpret_cast<uint2*>(xb)[t] = o;
        }
    } else {
        for (size_t t = t0; t < m; t += stride) xb[t] = __float2bfloat16_rn(x[t]);
    }
}
static tpmg_status nn_load_input(tpmg_nn* nn, size_t n, const float* x, cudaStream_t s) {
    const size_t m = n * nn->b.cin;
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    size_t blocks = (m / 4 + 255) / 256;
    if (blocks > (size_t)nsm * 8) blocks = (size_t)nsm * 8;  // eight 256-thread blocks per SM, grid-stride
    if (blocks < 1) blocks = 1;
    k_nn_input_f32<<<(unsigned)blocks, 256, 0, s>>>(m, x, nn->b.x);
    note_launch();
    return TPMG_OK;
}

__global__ void k_sumsq_f64(size_t n, const double* __restrict__ r, double* partials) {
    double s = 0.0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        s = fma(r[t], r[t], s);
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
__global__ void k_bf16_to_f32(size_t n, const __nv_bfloat16* __restrict__ a, float* __restrict__ b) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        b[t] = __bfloat162float(a[t]);
}

extern "C" tpmg_status tpmg_nn_make_pair(tpmg_op* op, int cin, const double* r, const double* u_star,
                                         const double* u_k, const float* aux, float* x_out, float* target_out,
                                         void* stream) {
    TRY(flat_only(op));
    if (!op || (cin != 1 && cin != 2) || !r || !x_out || (cin == 2 && !aux) || (target_out && (!u_star || !u_k)))
        return set_err(TPMG_ERR_ARG, "bad arguments");
    const int L = op->g.L, nx = op->g.nx, ny = op->g.ny, nz = op->g.nz;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny * nz, ncol = (size_t)nx * ny;
    const Lv<PolF32> LF = level_view<PolF32>(op, L);
    // scratch: partial sums, their total and the bf16 input (allocated per call: a training tool)
    double* part = nullptr;
    __nv_bfloat16* xb = nullptr;
    TRY(dalloc((void**)&part, sizeof(double) * 1025));
    if (dalloc((void**)&xb, n * 2 * cin) != TPMG_OK) {
        dev_free(part);
        return TPMG_ERR_OOM;
    }
    k_sumsq_f64<<<1024, 256, 0, s>>>(n, r, part);
    launch_finalize_norm(part, 1024, FIN_SUM, nullptr, nullptr, part + 1024, s);
    nn_make_input_f64(n, ncol, nz, cin, r, aux, part + 1024, xb, u_star, u_k, LF.cx, LF.cy, LF.v, target_out, s);
    k_bf16_to_f32<<<1024, 256, 0, s>>>(n * cin, xb, x_out);
    note_launch();
    note_launch();
    cudaError_t err = cudaStreamSynchronize(s);
    dev_free(part);
    dev_free(xb);
    if (err != cudaSuccess) return set_err(TPMG_ERR_CUDA, cudaGetErrorString(err));
    return TPMG_OK;
}

static tpmg_status read_fcg(tpmg_op* op, cudaStream_t s) {
    CK(cudaMemcpyAsync(op->fcg_host, op->fcg_sc, sizeof(FcgScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return TPMG_OK;
}

// Flexible CG(1) on double-word vectors (the iteration of the oracle's orc_fcg_solve); the
// preconditioner is one FP32 V-cycle of the mixed solver and, when a network is given, the learned
// correction, kept only when it lowers the residual.
extern "C" tpmg_status tpmg_fcg_solve(tpmg_op* op, tpmg_nn* nn, const float* aux, const tpmg_params* prm,
                                      const double* f, double* u, tpmg_info* info, int* nn_accepted, void* stream) {
    TRY(flat_only(op));
    TRY(check_params(op, prm));
    if (!f || !u) return set_err(TPMG_ERR_ARG, "NULL field");
    const int L = op->g.L;
    const int nx = op->g.nx, ny = op->g.ny, nz = op->g.nz;
    if (nn) {
        TRY(nn_check_shape(nx, ny, nz));
        if (nn->b.cin == 2 && !aux) return set_err(TPMG_ERR_ARG, "a 2-channel network needs the aux field");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = lvl_cells(op, L), ncol = (size_t)nx * ny;
    TRY(ensure_hier(op, 2, true));
    TRY(ensure_hier(op, 1, true));
    TRY(ensure_cg(op, 2));
    TRY(ensure_history(op, prm->max_iter + 2));
    if (!op->fcg_sc) TRY(dalloc((void**)&op->fcg_sc, sizeof(FcgScalars)));
    if (!op->fcg_host) CK(cudaMallocHost((void**)&op->fcg_host, sizeof(FcgScalars)));
    for (int t = 0; t < 3; ++t) TRY(dalloc(&op->fcgbuf[t], n * sizeof(float2)));
    if (nn) {
        TRY(nn_ensure_cap(nn, n));
        if (!nn->weights_ready) nn_refresh(nn, s);
    }
    FcgScalars* sc = (FcgScalars*)op->fcg_sc;
    const FcgScalars* hs = (const FcgScalars*)op->fcg_host;
    float2* uD = (float2*)op->hier[2].u[L];
    float2* fD = (float2*)op->hier[2].f[L];
    float2* r = (float2*)op->cgbuf[2][0];
    float2* z = (float2*)op->cgbuf[2][1];
    float2* p = (float2*)op->cgbuf[2][2];
    float2* q = (float2*)op->cgbuf[2][3];
    float2* z1 = (float2*)op->fcgbuf[0];
    float2* c = (float2*)op->fcgbuf[1];
    float2* w = (float2*)op->fcgbuf[2];
    Hier& h32 = op->hier[1];
    float* r32 = (float*)h32.f[L];
    Lv<PolDW> LD = level_view<PolDW>(op, L);
    Lv<PolF32> L32 = level_view<PolF32>(op, L);
    double* part = op->partials;
    auto precondition = [&]() {
        // z1 = V-cycle_FP32(r): the mixed solver's inner cycle from a zero guess
        fcg_f32_from_dw(n, r, r32, s);
        Cycle<PolF32, PolF32> cyc(op, prm, s, nullptr, 1);
        void* cur = h32.u[L];
        void* oth = h32.ub[L];
        launch_line_solve<PolF32>(L32, r32, (float*)cur, prm->rho, nullptr, s);
        cyc.rest(cur, oth);
        fcg_dw_from_f32(n, (const float*)cur, nn ? z1 : z, s);
        if (!nn) return;
        // learned stage: r1 = r - A z1; c = z1 + rms(r1) NN(r1 / rms(r1)); keep c if ||r - A c|| < ||r1||
        const int nr = launch_residual<PolDW, PolDW>(LD, z1, r, c, part, nullptr, s);
        fcg_scalar(FCG_R1, part, nr, sc, nullptr, s);
        nn_make_input_dw(n, ncol, nz, nn->b.cin, c, aux, &sc->r1sq, nn->b.x, s);
        nn_forward(nn->b, nx, ny, nz, nn->b.x, nn->b.out, s);
        fcg_learned(n, ncol, nz, op->cx[L], op->cy[L], op->v32[L], sc, z1, nn->b.out, c, s);
        const int nr2 = launch_residual<PolDW, PolDW>(LD, c, r, w, part, nullptr, s);
        fcg_scalar(FCG_DECIDE, part, nr2, sc, nullptr, s);
        fcg_select(n, sc, c, z1, z, s);
    };
    CK(cudaEventRecord(op->ev0, s));
    TRY(init_u_dw(n, prm, u, uD, s));
    launch_f64_to_dw(n, f, fD, s);
    fcg_init(sc, prm->tol, prm->max_iter, s);
    const int nb = launch_residual<PolDW, PolDW>(LD, uD, fD, r, part, nullptr, s);  // r = f - A u
    fcg_scalar(FCG_INIT_NORM, part, nb, sc, op->history, s);
    TRY(read_fcg(op, s));
    if (!hs->done) {
        precondition();
        CK(cudaMemcpyAsync(p, z, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
        for (int guard = 0; guard <= prm->max_iter + 1; ++guard) {
            const int na = fcg_apply(LD, p, r, q, part, s);  // q = A p, <p, q>, <p, r>
            fcg_scalar(FCG_ALPHA, part, na, sc, nullptr, s);
            const int nu = fcg_update(n, sc, uD, p, r, q, part, s);  // u += alpha p, r -= alpha q
            fcg_scalar(FCG_CHECK, part, nu, sc, op->history, s);
            TRY(read_fcg(op, s));
            if (hs->done) break;
            precondition();
            const int nd = fcg_dot(n, z, q, part, s);  // beta = <z, q> / <p, q>
            fcg_scalar(FCG_BETA, part, nd, sc, nullptr, s);
            fcg_direction(n, sc, z, p, s);  // p = z - beta p
        }
    }
    launch_dw_to_f64(n, uD, u, s);
    CK(cudaEventRecord(op->ev1, s));
    TRY(read_fcg(op, s));
    CK(cudaGetLastError());
    if (nn_accepted) *nn_accepted = hs->accepted;
    if (info) {
        info->iters = hs->iters;
        info->converged = hs->converged;
        info->rel_res = hs->rel;
        info->r0 = hs->r0;
        if (info->history && info->history_len > 0) {
            const int nh = hs->iters + 1 < info->history_len ? hs->iters + 1 : info->history_len;
            CK(cudaMemcpy(info->history, op->history, sizeof(double) * nh, cudaMemcpyDeviceToHost));
        }
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, op->ev0, op->ev1));
        info->ms = ms;
    }
    if (nn) TRY(nn_check(nn));
    if (hs->nonfinite) return set_err(TPMG_ERR_NONFINITE, "non-finite value in flexible CG");
    if (!hs->converged) return set_err(TPMG_ERR_NOT_CONVERGED, "max_iter reached");
    return TPMG_OK;
}

// ================================================================ the cubed-sphere panel operator
// Eq. (1) on one gnomonic cubed-sphere panel (Sec. 2.1.1: cell-centred finite volumes, homogeneous
// Dirichlet on the panel boundary, Neumann at the bottom and top) in the factorised form of Eq. (14).
// The host computes the geometry of every level (the rediscretised panel, Sec. 3.1) and the radial
// vectors once; k_panel.cu holds the kernels.

namespace {

struct V3 {
    double x, y, z;
};
// the cube-face point (X, Y, 1) projected onto the unit sphere
V3 gnomonic_point(double X, double Y) {
    const double r = std::sqrt(1.0 + X * X + Y * Y);
    return V3{X / r, Y / r, 1.0 / r};
}
// great-circle distance of two unit vectors (the atan2 form keeps short arcs accurate)
double great_arc(const V3& p, const V3& q) {
    const double cx = p.y * q.z - p.z * q.y, cy = p.z * q.x - p.x * q.z, cz = p.x * q.y - p.y * q.x;
    return std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), p.x * q.x + p.y * q.y + p.z * q.z);
}
// antiderivative of the spherical area element (1 + X^2 + Y^2)^(-3/2) dX dY of the gnomonic map
double gnomonic_area_prim(double X, double Y) { return std::atan(X * Y / std::sqrt(1.0 + X * X + Y * Y)); }

// |T| (ny x nx), x-face coefficients (ny x (nx+1)) and y-face coefficients ((ny+1) x nx) of an
// nx x ny grid on the panel [-ext, ext]^2: alpha = -omega^2 |e| / d, |e| the edge's great-circle
// length, d the great-circle distance of the two cell centres (the images of the coordinate
// midpoints; beyond the boundary the centre of the ghost cell of the extended grid).
void panel_level_geometry(int nx, int ny, double omega2, double ext, std::vector<double>& area,
                          std::vector<double>& ax, std::vector<double>& ay) {
    auto xs = [&](int i) { return -ext + 2.0 * ext * i / nx; };  // corner coordinates
    auto ys = [&](int j) { return -ext + 2.0 * ext * j / ny; };
    auto xc = [&](int i) { return -ext + 2.0 * ext * (i + 0.5) / nx; };  // centres, i = -1 .. nx
    auto yc = [&](int j) { return -ext + 2.0 * ext * (j + 0.5) / ny; };
    area.assign((size_t)nx * ny, 0.0);
    ax.assign((size_t)ny * (nx + 1), 0.0);
    ay.assign((size_t)(ny + 1) * nx, 0.0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            area[(size_t)j * nx + i] = gnomonic_area_prim(xs(i + 1), ys(j + 1)) - gnomonic_area_prim(xs(i), ys(j + 1)) -
                                       gnomonic_area_prim(xs(i + 1), ys(j)) + gnomonic_area_prim(xs(i), ys(j));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            const double e = great_arc(gnomonic_point(xs(i), ys(j)), gnomonic_point(xs(i), ys(j + 1)));
            const double d = great_arc(gnomonic_point(xc(i - 1), yc(j)), gnomonic_point(xc(i), yc(j)));
            ax[(size_t)j * (nx + 1) + i] = -omega2 * e / d;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double e = great_arc(gnomonic_point(xs(i), ys(j)), gnomonic_point(xs(i + 1), ys(j)));
            const double d = great_arc(gnomonic_point(xc(i), yc(j - 1)), gnomonic_point(xc(i), yc(j)));
            ay[(size_t)j * nx + i] = -omega2 * e / d;
        }
}

}  // namespace

static PanelLv panel_view(const tpmg_op* op, int l) {
    PanelLv L;
    L.nx = op->g.lnx[l];
    L.ny = op->g.lny[l];
    L.nz = op->g.nz;
    L.area = op->pgeo[l][0];
    L.ax = op->pgeo[l][1];
    L.ay = op->pgeo[l][2];
    L.E = op->prad[0];
    L.B = op->prad[1];
    L.C = op->prad[2];
    L.inv = op->pfac[l][0];
    L.fl = op->pfac[l][1];
    L.fw = op->pfac[l][2];
    return L;
}

// the FP64 hierarchy of a panel operator (u, u', f, r per level; the finest u, f are the caller's)
static tpmg_status panel_ensure_hier(tpmg_op* op) {
    Hier& h = op->hier[0];
    if (h.ready) return ensure_common(op);
    const int L = op->g.L;
    for (int l = 1; l <= L; ++l) {
        const size_t bytes = lvl_cells(op, l) * sizeof(double);
        TRY(dalloc(&h.ub[l], bytes));
        TRY(dalloc(&h.r[l], bytes));
        if (l < L) {
            TRY(dalloc(&h.u[l], bytes));
            TRY(dalloc(&h.f[l], bytes));
        }
    }
    h.ready = true;
    return ensure_common(op);
}

extern "C" tpmg_status tpmg_create_panel_operator(const tpmg_grid* g, double omega2, double lambda2, double H,
                                                  double extent, tpmg_op** out) {
    if (!g || !out) return set_err(TPMG_ERR_ARG, "NULL grid or output pointer");
    *out = nullptr;
    if (!(omega2 > 0.0) || !(lambda2 >= 0.0) || !(H > 0.0) || !(extent > 0.0 && extent <= 1.0))
        return set_err(TPMG_ERR_ARG, "omega2 > 0, lambda2 >= 0, H > 0 and 0 < extent <= 1 required");
    tpmg_op* op = new tpmg_op();
    for (int p = 0; p < 3; ++p)
        for (int l = 0; l <= MAXL; ++l) {
            op->variant[p][l] = -1;
            op->fac_k0[p][l] = 1 << 30;
        }
    op->g = *g;
    op->panel = 1;
    op->omega2 = omega2;
    cudaGetDevice(&op->device);
    const int L = g->L, nz = g->nz;
    tpmg_status st = TPMG_OK;
    auto fail = [&](tpmg_status s2) {
        tpmg_destroy_operator(op);
        return s2;
    };
    // radial vectors of r in [1, 1 + H] with nz cells: a_k = (r_{k+1/2}^3 - r_{k-1/2}^3) / (3 h_z),
    // B_k = omega^2 lambda^2 r_{k-1/2}^2 / h_z^2 (0 at k = 0), C_k = B_{k+1} (0 at the top)
    const double hz = H / nz;
    std::vector<double> E(nz), B(nz), C(nz);
    auto rface = [&](int k) { return 1.0 + H * k / nz; };
    for (int k = 0; k < nz; ++k) B[k] = k == 0 ? 0.0 : omega2 * lambda2 * rface(k) * rface(k) / (hz * hz);
    for (int k = 0; k < nz; ++k) {
        C[k] = k + 1 < nz ? B[k + 1] : 0.0;
        const double a = (std::pow(rface(k + 1), 3) - std::pow(rface(k), 3)) / (3.0 * hz);
        E[k] = a + B[k] + C[k];
    }
    const std::vector<double>* rad[3] = {&E, &B, &C};
    for (int t = 0; t < 3; ++t) {
        if ((st = dalloc((void**)&op->prad[t], nz * sizeof(double))) != TPMG_OK) return fail(st);
        if (cudaMemcpy(op->prad[t], rad[t]->data(), nz * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(set_err(TPMG_ERR_CUDA, "copy of the radial vectors failed"));
    }
    for (int l = L; l >= 1; --l) {
        const int nx = g->lnx[l], ny = g->lny[l];
        std::vector<double> geo[3];
        panel_level_geometry(nx, ny, omega2, extent, geo[0], geo[1], geo[2]);
        for (int t = 0; t < 3; ++t) {
            if ((st = dalloc((void**)&op->pgeo[l][t], geo[t].size() * sizeof(double))) != TPMG_OK) return fail(st);
            if (cudaMemcpy(op->pgeo[l][t], geo[t].data(), geo[t].size() * sizeof(double), cudaMemcpyHostToDevice) !=
                cudaSuccess)
                return fail(set_err(TPMG_ERR_CUDA, "copy of the panel geometry failed"));
        }
        for (int t = 0; t < 3; ++t)
            if ((st = dalloc((void**)&op->pfac[l][t], lvl_cells(op, l) * sizeof(double))) != TPMG_OK) return fail(st);
        launch_panel_factors(panel_view(op, l), op->pfac[l][0], op->pfac[l][1], op->pfac[l][2], 0);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(set_err(TPMG_ERR_CUDA, "panel setup kernels failed"));
    if (cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&op->ev0) != cudaSuccess || cudaEventCreate(&op->ev1) != cudaSuccess)
        return fail(set_err(TPMG_ERR_CUDA, "stream/event creation failed"));
    *out = op;
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_panel_level_geometry(const tpmg_op* op, int level, double* area, double* ax, double* ay) {
    TRY(check_level(op, level));
    if (!op->panel) return set_err(TPMG_ERR_ARG, "not a panel operator");
    const size_t nx = op->g.lnx[level], ny = op->g.lny[level];
    const size_t sz[3] = {nx * ny, ny * (nx + 1), (ny + 1) * nx};
    double* dst[3] = {area, ax, ay};
    for (int t = 0; t < 3; ++t)
        if (dst[t]) CK(cudaMemcpy(dst[t], op->pgeo[level][t], sz[t] * sizeof(double), cudaMemcpyDeviceToHost));
    return TPMG_OK;
}

static tpmg_status panel_unit_check(tpmg_op* op, int level) {
    TRY(check_level(op, level));
    if (!op->panel) return set_err(TPMG_ERR_ARG, "not a panel operator (tpmg_create_panel_operator)");
    return panel_ensure_hier(op);
}

extern "C" tpmg_status tpmg_panel_apply_A(tpmg_op* op, int level, const double* x, double* y, void* stream) {
    TRY(panel_unit_check(op, level));
    if (!x || !y) return set_err(TPMG_ERR_ARG, "NULL field");
    launch_panel_sweep<double>(PANEL_APPLY, panel_view(op, level), 1.0, x, nullptr, y, nullptr, nullptr, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_panel_line_solve(tpmg_op* op, int level, const double* b, double* x, void* stream) {
    TRY(panel_unit_check(op, level));
    if (!b || !x) return set_err(TPMG_ERR_ARG, "NULL field");
    launch_panel_sweep<double>(PANEL_LINESOLVE, panel_view(op, level), 1.0, b, nullptr, x, nullptr, nullptr,
                       (cudaStream_t)stream);
    CK(cudaGetLastError());
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_panel_smooth(tpmg_op* op, int level, double rho, const double* u, const double* f,
                                         double* u_out, double* norm_out, void* stream) {
    TRY(panel_unit_check(op, level));
    if (!u || !f || !u_out) return set_err(TPMG_ERR_ARG, "NULL field");
    cudaStream_t s = (cudaStream_t)stream;
    const int np = launch_panel_sweep<double>(PANEL_SMOOTH, panel_view(op, level), rho, u, f, u_out,
                                      norm_out ? op->partials : nullptr, nullptr, s);
    if (norm_out) launch_finalize_norm(op->partials, np, FIN_STORE, op->sc, nullptr, norm_out, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_panel_residual(tpmg_op* op, int level, const double* u, const double* f, double* r,
                                           double* norm_out, void* stream) {
    TRY(panel_unit_check(op, level));
    if (!u || !f || !r) return set_err(TPMG_ERR_ARG, "NULL field");
    cudaStream_t s = (cudaStream_t)stream;
    const int np = launch_panel_sweep<double>(PANEL_RESIDUAL, panel_view(op, level), 1.0, u, f, r,
                                      norm_out ? op->partials : nullptr, nullptr, s);
    if (norm_out) launch_finalize_norm(op->partials, np, FIN_STORE, op->sc, nullptr, norm_out, s);
    CK(cudaGetLastError());
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_panel_restrict_smooth(tpmg_op* op, int level, double rho, const double* r_fine,
                                                  double* f_c, double* u_c, void* stream) {
    TRY(panel_unit_check(op, level));
    if (level >= op->g.L) return set_err(TPMG_ERR_ARG, "the coarse level must be below the finest");
    if (!r_fine || !f_c || !u_c) return set_err(TPMG_ERR_ARG, "NULL field");
    launch_panel_restrict_smooth(panel_view(op, level), rho, r_fine, f_c, u_c, nullptr, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return TPMG_OK;
}

extern "C" tpmg_status tpmg_panel_prolongate(tpmg_op* op, int level, const double* u_c, double* u_f, void* stream) {
    TRY(panel_unit_check(op, level));
    if (level < 2) return set_err(TPMG_ERR_ARG, "the fine level must be above the coarsest");
    if (!u_c || !u_f) return set_err(TPMG_ERR_ARG, "NULL field");
    launch_panel_prolongate(op->g.lnx[level - 1], op->g.lny[level - 1], op->g.nz, u_c, u_f, nullptr,
                            (cudaStream_t)stream);
    CK(cudaGetLastError());
    return TPMG_OK;
}

static PanelLvT<float> panel_view32(const tpmg_op* op, int l) {
    PanelLvT<float> L;
    L.nx = op->g.lnx[l];
    L.ny = op->g.lny[l];
    L.nz = op->g.nz;
    L.area = op->pgeo32[l][0];
    L.ax = op->pgeo32[l][1];
    L.ay = op->pgeo32[l][2];
    L.E = op->prad32[0];
    L.B = op->prad32[1];
    L.C = op->prad32[2];
    L.inv = op->pfac32[l][0];
    L.fl = op->pfac32[l][1];
    L.fw = op->pfac32[l][2];
    return L;
}
template <class T>
static PanelLvT<T> panel_view_t(const tpmg_op* op, int l);
template <>
PanelLvT<double> panel_view_t<double>(const tpmg_op* op, int l) {
    return panel_view(op, l);
}
template <>
PanelLvT<float> panel_view_t<float>(const tpmg_op* op, int l) {
    return panel_view32(op, l);
}

// FP32 copies of the geometry, radial vectors and Thomas factors (rounded from the FP64 ones) and the
// FP32 hierarchy, for the mixed-precision solve's inner V-cycles
static tpmg_status panel_ensure_f32(tpmg_op* op, cudaStream_t s) {
    Hier& h = op->hier[1];
    if (h.ready) return TPMG_OK;
    const int L = op->g.L, nz = op->g.nz;
    for (int t = 0; t < 3; ++t) {
        TRY(dalloc((void**)&op->prad32[t], nz * sizeof(float)));
        launch_f64_to_f32(nz, op->prad[t], op->prad32[t], s);
    }
    for (int l = 1; l <= L; ++l) {
        const size_t nx = op->g.lnx[l], ny = op->g.lny[l], n = lvl_cells(op, l);
        const size_t gsz[3] = {nx * ny, ny * (nx + 1), (ny + 1) * nx};
        for (int t = 0; t < 3; ++t) {
            TRY(dalloc((void**)&op->pgeo32[l][t], gsz[t] * sizeof(float)));
            launch_f64_to_f32(gsz[t], op->pgeo[l][t], op->pgeo32[l][t], s);
            TRY(dalloc((void**)&op->pfac32[l][t], n * sizeof(float)));
            launch_f64_to_f32(n, op->pfac[l][t], op->pfac32[l][t], s);
        }
        const size_t bytes = n * sizeof(float);
        TRY(dalloc(&h.u[l], bytes));
        TRY(dalloc(&h.ub[l], bytes));
        TRY(dalloc(&h.f[l], bytes));
        TRY(dalloc(&h.r[l], bytes));
    }
    CK(cudaGetLastError());
    h.ready = true;
    return TPMG_OK;
}

// One V-cycle of Algorithm 1 on the panel hierarchy of value type T (FP64: op->hier[0]; FP32, the
// mixed solve's inner cycle: op->hier[1]) after the finest level's first smoothing step, as Cycle
// does for the flat box (RestrictSmooth opening every coarse level, nu_pre - 1 further pre-smoothing
// steps, the residual, the recursion, the prolongation, nu_post post-smoothing steps; n_coarse steps
// in all on the coarsest level).
template <class T>
struct PanelCycle {
    tpmg_op* op;
    const tpmg_params* prm;
    cudaStream_t s;
    const int* done;
    const T* fL;
    Hier& hier() { return op->hier[sizeof(T) == 8 ? 0 : 1]; }
    void smooth(int l, T*& cur, T*& oth, const T* f) {
        launch_panel_sweep<T>(PANEL_SMOOTH, panel_view_t<T>(op, l), prm->rho, cur, f, oth, nullptr, done, s);
        T* t = cur;
        cur = oth;
        oth = t;
    }
    T* coarse(int l) {
        Hier& h = hier();
        T* cur = (T*)h.u[l];
        T* oth = (T*)h.ub[l];
        const T* f = (const T*)h.f[l];
        launch_panel_restrict_smooth<T>(panel_view_t<T>(op, l), prm->rho, (const T*)h.r[l + 1], (T*)h.f[l], cur, done,
                                        s);
        if (l == 1) {
            for (int t = 1; t < prm->n_coarse; ++t) smooth(l, cur, oth, f);
            return cur;
        }
        for (int t = 1; t < prm->nu_pre; ++t) smooth(l, cur, oth, f);
        return below(l, cur, oth, f);
    }
    // residual of level l, the coarser levels, prolongation and post-smoothing on level l
    T* below(int l, T* cur, T* oth, const T* f) {
        Hier& h = hier();
        launch_panel_sweep<T>(PANEL_RESIDUAL, panel_view_t<T>(op, l), 1.0, cur, f, (T*)h.r[l], nullptr, done, s);
        const T* uc = coarse(l - 1);
        launch_panel_prolongate<T>(op->g.lnx[l - 1], op->g.lny[l - 1], op->g.nz, uc, cur, done, s);
        for (int t = 0; t < prm->nu_post; ++t) smooth(l, cur, oth, f);
        return cur;
    }
    T* rest(T* cur, T* oth) {
        const int L = op->g.L;
        if (L == 1) {
            for (int t = 1; t < prm->n_coarse; ++t) smooth(L, cur, oth, fL);
            return cur;
        }
        for (int t = 1; t < prm->nu_pre; ++t) smooth(L, cur, oth, fL);
        return below(L, cur, oth, fL);
    }
};

static tpmg_status panel_mg_loop(tpmg_op* op, const tpmg_params* prm, double* A, const double* fL, cudaStream_t s) {
    const int L = op->g.L;
    const int* done = &op->sc->done;
    double* B = (double*)op->hier[0].ub[L];
    const size_t nfine = lvl_cells(op, L);
    const PanelLv LL = panel_view(op, L);
    launch_scalars_init(op->sc, prm->tol, prm->max_iter, s);
    const int nparts = launch_panel_sweep<double>(PANEL_SMOOTH, LL, prm->rho, A, fL, B, op->partials, done, s);
    launch_finalize_norm(op->partials, nparts, FIN_MG_INIT, op->sc, op->history, nullptr, s);
    CK(cudaGetLastError());
    TRY(read_scalars(op, s));
    auto body = [&](cudaStream_t st) {
        PanelCycle<double> c{op, prm, st, done, fL};
        double* cur = c.rest(B, A);
        if (cur != A) launch_copy<PolF64>(nfine, cur, A, done, st);
        const int np = launch_panel_sweep<double>(PANEL_SMOOTH, LL, prm->rho, A, fL, B, op->partials, done, st);
        launch_finalize_norm(op->partials, np, FIN_MG_CYCLE, op->sc, op->history, nullptr, st);
    };
    std::vector<const void*> key = {A, fL, B, op->history, (const void*)(size_t)prm->nu_pre,
                                    (const void*)(size_t)prm->nu_post, (const void*)(size_t)prm->n_coarse,
                                    (const void*)(size_t)(prm->rho * 1e12)};
    int guard = 0;
    while (!op->sc_host->done && guard++ <= prm->max_iter + 1) {
        TRY(run_iteration(op, 7, key, prm->use_graph != 0, s, body));
        TRY(read_scalars(op, s));
    }
    return TPMG_OK;
}

// Mixed precision on the panel: iterative refinement with the outer residual r = f - A u in native
// FP64 (stored FP32), one FP32 V-cycle for A e = r from e = 0, u += e in FP64, until Eq. (10) holds.
static tpmg_status panel_mixed_loop(tpmg_op* op, const tpmg_params* prm, double* u, const double* f, cudaStream_t s) {
    const int L = op->g.L;
    const int* done = &op->sc->done;
    Hier& h32 = op->hier[1];
    float* e = (float*)h32.u[L];
    float* eb = (float*)h32.ub[L];
    float* r32 = (float*)h32.f[L];
    const size_t nfine = lvl_cells(op, L);
    const PanelLv LD = panel_view(op, L);
    const PanelLvT<float> L32 = panel_view32(op, L);
    launch_scalars_init(op->sc, prm->tol, prm->max_iter, s);
    const int nparts = launch_panel_residual_to_f32(LD, u, f, r32, op->partials, done, s);
    launch_finalize_norm(op->partials, nparts, FIN_MG_INIT, op->sc, op->history, nullptr, s);
    CK(cudaGetLastError());
    TRY(read_scalars(op, s));
    auto body = [&](cudaStream_t st) {
        // first smoothing step from e = 0: e = rho M^{-1} r
        launch_panel_sweep<float>(PANEL_LINESOLVE, L32, prm->rho, r32, nullptr, e, nullptr, done, st);
        PanelCycle<float> c{op, prm, st, done, r32};
        const float* cur = c.rest(e, eb);
        launch_correct<PolF64>(nfine, u, cur, done, st);
        const int np = launch_panel_residual_to_f32(LD, u, f, r32, op->partials, done, st);
        launch_finalize_norm(op->partials, np, FIN_MG_CYCLE, op->sc, op->history, nullptr, st);
    };
    std::vector<const void*> key = {u, f, e, op->history, (const void*)(size_t)prm->nu_pre,
                                    (const void*)(size_t)prm->nu_post, (const void*)(size_t)prm->n_coarse,
                                    (const void*)(size_t)(prm->rho * 1e12)};
    int guard = 0;
    while (!op->sc_host->done && guard++ <= prm->max_iter + 1) {
        TRY(run_iteration(op, 3, key, prm->use_graph != 0, s, body));  // a panel operator runs no flat mixed solve
        TRY(read_scalars(op, s));
    }
    return TPMG_OK;
}

static tpmg_status panel_mg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, tpmg_info* info,
                                  void* stream) {
    if (prm->prec != TPMG_F64 && prm->prec != TPMG_MIXED)
        return set_err(TPMG_ERR_ARG, "the panel operator runs in native FP64 (TPMG_F64) or mixed (TPMG_MIXED)");
    if (prm->coarse_bf16) return set_err(TPMG_ERR_ARG, "coarse_bf16 is a flat-box measurement");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = lvl_cells(op, op->g.L);
    TRY(panel_ensure_hier(op));
    if (prm->prec == TPMG_MIXED) TRY(panel_ensure_f32(op, s));
    TRY(ensure_history(op, prm->max_iter + 2));
    CK(cudaEventRecord(op->ev0, s));
    TRY(init_u(n, sizeof(double), prm, u, s));
    if (prm->prec == TPMG_MIXED)
        TRY(panel_mixed_loop(op, prm, (double*)u, (const double*)f, s));
    else
        TRY(panel_mg_loop(op, prm, (double*)u, (const double*)f, s));
    CK(cudaEventRecord(op->ev1, s));
    CK(cudaGetLastError());
    return finish_info(op, info, s);
}

// Line-preconditioned CG on the panel (Sec. 2.2) with the fused SpMV and Tridiag kernels of Sec. 3.1,
// the same iteration and device-side scalars as the flat-box CG.
static tpmg_status panel_cg_solve(tpmg_op* op, const tpmg_params* prm, const void* fv, void* uv, tpmg_info* info,
                                  void* stream) {
    if (prm->prec != TPMG_F64) return set_err(TPMG_ERR_ARG, "the panel operator runs in native FP64 (TPMG_F64)");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = op->g.L;
    const size_t n = lvl_cells(op, L);
    TRY(panel_ensure_hier(op));
    TRY(ensure_history(op, prm->max_iter + 2));
    for (int t = 0; t < 4; ++t) TRY(dalloc(&op->cgbuf[0][t], n * sizeof(double)));
    double* u = (double*)uv;
    const double* f = (const double*)fv;
    double* r = (double*)op->cgbuf[0][0];
    double* z = (double*)op->cgbuf[0][1];
    double* p = (double*)op->cgbuf[0][2];
    double* q = (double*)op->cgbuf[0][3];
    const PanelLv LL = panel_view(op, L);
    const int nb = panel_blocks(LL.nx, LL.ny);
    CK(cudaEventRecord(op->ev0, s));
    TRY(init_u(n, sizeof(double), prm, u, s));
    launch_scalars_init(op->sc, prm->tol, prm->max_iter, s);
    launch_panel_sweep<double>(PANEL_RESIDUAL, LL, 1.0, u, f, r, nullptr, nullptr, s);
    CK(cudaMemsetAsync(p, 0, n * sizeof(double), s));
    CK(cudaMemsetAsync(q, 0, n * sizeof(double), s));
    launch_panel_cg_tridiag(LL, op->sc, r, q, z, op->partials, s);  // alpha = 0: z = M^{-1} r
    launch_cg_beta(op->partials, nb, 1, op->sc, op->history, s);
    CK(cudaGetLastError());
    TRY(read_scalars(op, s));
    auto body = [&](cudaStream_t st) {
        launch_panel_cg_spmv(LL, op->sc, u, p, z, q, op->partials, st);
        launch_cg_alpha(op->partials, nb, op->sc, st);
        launch_panel_cg_tridiag(LL, op->sc, r, q, z, op->partials, st);
        launch_cg_beta(op->partials, nb, 0, op->sc, op->history, st);
    };
    std::vector<const void*> key = {u, f, r, op->history};
    int guard = 0;
    while (!op->sc_host->done && guard++ <= prm->max_iter + 1) {
        TRY(run_iteration(op, 4, key, prm->use_graph != 0, s, body));  // a panel operator runs no flat CG
        TRY(read_scalars(op, s));
    }
    launch_cg_finish<PolF64>(n, op->sc, u, p, s);
    CK(cudaEventRecord(op->ev1, s));
    CK(cudaGetLastError());
    return finish_info(op, info, s);
}
