/*
 * tpmg.h -- C ABI of the GB300 tensor-product multigrid / line-preconditioned CG library for the
 * strongly vertically anisotropic elliptic problem of Mueller, Scheichl & Vainikko, "Petascale
 * elliptic solvers for anisotropic PDEs on GPU clusters" (arXiv:1402.3545).
 *
 * Problem (Sec. 2.1.1, flat-box form of Eq. (6) "TridiagonalPDE"):
 *   -omega^2 (d_xx u + d_yy u + lambda^2(x,y) d_zz u) + u = f
 * on an nx x ny x nz cell-centred grid, periodic in x and y, homogeneous Neumann at the bottom and
 * top (Sec. 2.1). The discrete operator is the 7-point stencil
 *   (A u)_ijk = (1 + 2cx + 2cy + v_ij n_k) u_ijk - cx (u_{i-1,j,k} + u_{i+1,j,k})
 *               - cy (u_{i,j-1,k} + u_{i,j+1,k}) - v_ij (u_{i,j,k-1} + u_{i,j,k+1})
 * with cx = omega^2/hx^2, cy = omega^2/hy^2, v_ij = omega^2 lambda_ij^2/hz^2, n_k the number of
 * vertical neighbours of cell k (2 inside, 1 at a Neumann end) and the missing neighbours dropped.
 *
 * Conventions shared by every entry point:
 *  - Fields are device arrays of nz*ny*nx values, x fastest: element (i,j,k) at (k*ny + j)*nx + i
 *    (x-contiguous like Eq. (13) "MemoryMapSingleGPU"; k outermost so horizontal planes are
 *    contiguous). The caller owns them; they must not overlap unless an entry point says so.
 *  - Multigrid levels are numbered as in Sec. 2.2: 1 = coarsest ... L = finest. Level l has
 *    nx/2^(L-l) x ny/2^(L-l) x nz cells, cx and cy divided by 4^(L-l), and v averaged over the
 *    2x2 children of each coarse column.
 *  - Element type of a field argument by precision: TPMG_F64 and TPMG_DW: double; TPMG_F32:
 *    float; TPMG_MIXED (solvers only): double. TPMG_DW computes in double-word ("float-float")
 *    arithmetic on the FP32 units (about 2^-47 relative accuracy per operation) and converts at the
 *    boundary through library-owned workspace; TPMG_F64 computes in native FP64.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Every entry point is stream
 *    ordered; only the solvers and tpmg_op_reserve synchronise (solvers: once per iteration, to
 *    read the convergence flag).
 *  - Errors are returned as a tpmg_status, never thrown; nothing aborts the process. A failed
 *    CUDA call yields TPMG_ERR_CUDA and tpmg_last_error() describes it.
 *  - Workspace (coarse levels, ping-pong buffers, precision-conversion buffers, partial sums) is
 *    owned by the operator, allocated with cudaMalloc on the first call that needs it (or by
 *    tpmg_op_reserve) and freed by tpmg_destroy_operator. Call tpmg_op_reserve before capturing
 *    library calls into a CUDA graph.
 *  - One operator must not be used by two host threads or two streams at the same time.
 */
#ifndef TPMG_H
#define TPMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TPMG_OK = 0,
    TPMG_ERR_ARG = 1,           /* invalid argument (sizes, level, precision, NULL pointer) */
    TPMG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    TPMG_ERR_OOM = 3,           /* workspace allocation failed */
    TPMG_ERR_NOT_CONVERGED = 4, /* max_iter reached; u holds the last iterate */
    TPMG_ERR_NONFINITE = 5,     /* NaN or Inf met in a norm or dot product; u holds the last iterate */
    TPMG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    TPMG_ERR_NN_REJECTED = 7    /* the learned preconditioner stage was rejected (fallback used) */
} tpmg_status;

typedef enum {
    TPMG_F64 = 0,  /* FP64 storage, native FP64 arithmetic */
    TPMG_F32 = 1,  /* FP32 storage and arithmetic */
    TPMG_DW = 2,   /* FP64 storage at the interface, double-word (float-float) arithmetic inside */
    TPMG_MIXED = 3 /* solvers: FP64-accurate outer residual and correction (double-word), FP32
                      inner V-cycles (iterative refinement) */
} tpmg_precision;

typedef struct tpmg_grid tpmg_grid; /* opaque, library owned */
typedef struct tpmg_op tpmg_op;     /* opaque, library owned */

/* Device memory. The library allocates its own buffers (hierarchy, workspace, scratch, tables)
 * with cudaMalloc when an operator, solve or network first needs them, and frees them in the
 * matching destroy call. tpmg_set_allocator installs a caller's allocator instead (for instance a
 * framework's caching allocator, so that one pool serves everything): alloc_fn(bytes, ctx) returns
 * device memory of at least `bytes` bytes, aligned to 256 bytes, usable on the streams the caller
 * passes to this library, or NULL (the call that needed it fails with TPMG_ERR_OOM); free_fn(ptr,
 * ctx) takes a block back; the library synchronises the device before it returns a block. Both
 * functions NULL restores cudaMalloc / cudaFree; one NULL is TPMG_ERR_ARG. Process-wide: the
 * functions installed when a buffer is allocated are the ones it is returned to, whatever is
 * installed later; each call into the library that allocates must not overlap a
 * tpmg_set_allocator call. */
typedef void* (*tpmg_alloc_fn)(size_t bytes, void* ctx);
typedef void (*tpmg_free_fn)(void* ptr, void* ctx);
tpmg_status tpmg_set_allocator(tpmg_alloc_fn alloc_fn, tpmg_free_fn free_fn, void* ctx);

/* Grid of nx x ny x nz cells with `nlevels` multigrid levels (0 = halve nx and ny while both stay
 * even and the larger one exceeds 8: 8 x 8 for square grids; on elongated grids the short side may
 * reach 1, which keeps the coarsest level well conditioned). nx and ny must be divisible by
 * 2^(nlevels-1);
 * 1 <= nz <= 256; nlevels <= 16. Sec. 2.2 (horizontal-only semicoarsening, nz fixed). */
tpmg_status tpmg_create_grid(int nx, int ny, int nz, int nlevels, tpmg_grid** out);
tpmg_status tpmg_destroy_grid(tpmg_grid* g);
/* Number of levels, and the horizontal size of `level` (1 = coarsest). */
int tpmg_grid_nlevels(const tpmg_grid* g);
tpmg_status tpmg_grid_level_size(const tpmg_grid* g, int level, int* nx, int* ny);

/* Operator -omega2 (Lap_h + lambda^2 d_zz) + I on grid g with mesh widths hx, hy, hz
 * (Sec. 2.1.1). lambda2_col is a HOST array of ny*nx values lambda^2 per column (index j*nx + i),
 * copied at creation; when NULL the constant `lambda2` is used. Builds the per-level coefficients
 * on the current CUDA device (the operator is bound to that device). The grid may be destroyed
 * afterwards. */
tpmg_status tpmg_create_operator(const tpmg_grid* g, double omega2, double hx, double hy, double hz,
                                 double lambda2, const double* lambda2_col, tpmg_op** out);
tpmg_status tpmg_destroy_operator(tpmg_op* op);
/* Allocates now the workspace a solver in precision `prec` needs (see the conventions above). */
tpmg_status tpmg_op_reserve(tpmg_op* op, tpmg_precision prec);
/* Discrete coefficients of `level`: cx, cy and the HOST copy of v (ny_l*nx_l values), any NULL. */
tpmg_status tpmg_op_level_coefficients(const tpmg_op* op, int level, double* cx, double* cy,
                                       double* v_host);

/* ---------------------------------------------------------------- single applications
 * Each applies one kernel of the method on `level` (1..L). x, y, b, u, f, r, u_out are device
 * fields of that level in the element type of `prec` (TPMG_F64, TPMG_F32 or TPMG_DW). */

/* y = A x, Eq. (9) "SpMVPrec" (SpMV). x and y must not overlap. */
tpmg_status tpmg_apply_A(tpmg_op* op, int level, tpmg_precision prec, const void* x, void* y,
                         void* stream);
/* x = M^{-1} b with M the vertical line relaxation (block diagonal of the column blocks A_T of
 * Eq. (6)), one Thomas solve per column: Eq. (9) (Preconditioner), Sec. 2.2. */
tpmg_status tpmg_line_solve(tpmg_op* op, int level, tpmg_precision prec, const void* b, void* x,
                            void* stream);
/* u_out = u + rho M^{-1}(f - A u): one block-Jacobi smoothing step, Eq. (11)
 * "MultigridSmoother". If norm_out (a DEVICE double) is not NULL it receives ||f - A u||_2. */
tpmg_status tpmg_smooth(tpmg_op* op, int level, tpmg_precision prec, double rho, const void* u,
                        const void* f, void* u_out, double* norm_out, void* stream);
/* r = f - A u (kernel "Residual", Sec. 3.1); optional ||r||_2 into the DEVICE double norm_out. */
tpmg_status tpmg_residual(tpmg_op* op, int level, tpmg_precision prec, const void* u,
                          const void* f, void* r, double* norm_out, void* stream);
/* Fused restriction and first smoothing step on coarse level `level` (< L) (kernel
 * "RestrictSmooth", Algorithm 1): f_c = R r_f (cell average of the 2x2 children of the residual
 * r_f of level+1), u_c = rho M_c^{-1} f_c. */
tpmg_status tpmg_restrict_smooth(tpmg_op* op, int level, tpmg_precision prec, double rho,
                                 const void* r_fine, void* f_c, void* u_c, void* stream);
/* Residual of fine level level+1 and RestrictSmooth onto coarse level `level` (< L) in one pass
 * (Algorithm 1: the kernels "Residual" and "RestrictSmooth" of Sec. 3.1 fused; the fine residual is
 * not stored): f_c = R (f_fine - A u_fine), u_c = rho M_c^{-1} f_c. u_fine, f_fine are fields of
 * level+1, f_c, u_c of `level` (caller-owned device memory, layout and element type as above). The
 * fused kernel performs the two kernels' arithmetic operation for operation: in TPMG_F64 and
 * TPMG_F32 the result equals tpmg_residual followed by tpmg_restrict_smooth bit for bit (in TPMG_DW
 * those separate calls round the residual to double in between, the fused pass does not). Where the
 * fused kernel does not apply (fine nx % 64 != 0 or odd ny, a coarse level of at most 4096 columns,
 * 16-byte misaligned fine fields, a double-word fine level over a native-FP64 coarse one) the two
 * kernels run instead. The multigrid cycles use the fusion unless tpmg_set_fusion turned it off. */
tpmg_status tpmg_residual_restrict_smooth(tpmg_op* op, int level, tpmg_precision prec, double rho,
                                          const void* u_fine, const void* f_fine, void* f_c, void* u_c,
                                          void* stream);
/* enable != 0 (the default): V-cycles of this operator fuse Residual and RestrictSmooth wherever
 * tpmg_residual_restrict_smooth's fused kernel applies (in tpmg_mg_solve_batched: wherever the
 * fine level takes its two-column tiles); 0: separate kernels. Same results bit for bit either way.
 * Invalidates the operator's cached CUDA graphs and batched-solve tables. */
tpmg_status tpmg_set_fusion(tpmg_op* op, int enable);
/* u_f += P u_c on fine level `level` (> 1), P the cell-centred bilinear interpolation from level-1
 * (kernel "Prolongate", Sec. 2.2). */
tpmg_status tpmg_prolongate(tpmg_op* op, int level, tpmg_precision prec, const void* u_c, void* u_f,
                            void* stream);
/* Fused CG kernels on the finest level (Sec. 3.1, "Conjugate Gradient"):
 * spmv:    u += alpha p; p = z + beta p; q = A z + beta q; *sigma_out = <p, q>
 * tridiag: r -= alpha q; z = M^{-1} r; *rr_out = <r, r>; *rz_out = <r, z>
 * The scalar outputs are DEVICE doubles. u, p, z, q, r are fields of the finest level; in TPMG_DW
 * the fields are double and converted in and out around the fused kernel. */
tpmg_status tpmg_cg_fused_spmv(tpmg_op* op, tpmg_precision prec, double alpha, double beta, void* u,
                               void* p, const void* z, void* q, double* sigma_out, void* stream);
tpmg_status tpmg_cg_fused_tridiag(tpmg_op* op, tpmg_precision prec, double alpha, void* r,
                                  const void* q, void* z, double* rr_out, double* rz_out,
                                  void* stream);

/* ---------------------------------------------------------------- solvers */
typedef struct {
    int nu_pre;      /* pre-smoothing steps per level (>= 1); the first one on coarse levels is the
                        fused RestrictSmooth */
    int nu_post;     /* post-smoothing steps per level (>= 0) */
    int n_coarse;    /* smoothing steps on the coarsest level (>= 1), Sec. 2.2 last paragraph */
    int max_iter;    /* V-cycles or CG iterations */
    double rho;      /* relaxation of the block-Jacobi smoother, Eq. (11) */
    double tol;      /* stop when ||f - A u|| / ||f - A u_0|| < tol, Eq. (10) */
    tpmg_precision prec;
    int use_graph;   /* 1: replay each iteration from a CUDA graph (default), 0: plain launches */
    double timeout_s; /* time limit of every device-side wait (the batched solver's grid barrier);
                         default 1.0 s; when it runs out the solve ends with TPMG_ERR_TIMEOUT */
    int zero_guess;  /* 1: start from u = 0 without reading u (u is then output only), 0: start from
                        the u passed in (default) */
    int coarse_bf16; /* TPMG_MIXED multigrid only: 1 rounds every value the inner FP32 V-cycle stores
                        on the levels below the finest to BF16 (kept in FP32 words), to measure how
                        BF16 storage of the coarse levels affects convergence; 0 (default): FP32 */
} tpmg_params;

typedef struct {
    int iters;          /* V-cycles (or CG iterations) done */
    int converged;      /* 1 if the tolerance was met */
    double rel_res;     /* final ||r||/||r0|| as the solver measured it */
    double r0;          /* ||f - A u_0|| */
    double* history;    /* caller's HOST array of history_len doubles, or NULL: relative residual
                           before the first and after each iteration */
    int history_len;
    double ms;          /* device time of the solve in milliseconds (CUDA events on `stream`) */
} tpmg_info;

/* V(2,2), 2 coarse steps, rho 0.8, tol 1e-6, max_iter 100, TPMG_DW, graphs on, 1 s wait limit. */
void tpmg_default_params(tpmg_params* p);

/* Multigrid solve (Sec. 2.2, Algorithm 1 with nu_pre/nu_post smoothing steps): V-cycles from the
 * initial guess in u until Eq. (10) holds. f and u are finest-level device fields (double for
 * TPMG_F64, TPMG_DW and TPMG_MIXED, float for TPMG_F32). With TPMG_DW and TPMG_MIXED, f and u may
 * instead be host memory the device addresses (page-locked allocations such as cudaHostAlloc's):
 * the solve then reads f and the initial u from the host and writes the final u there inside its
 * first and last kernels (one pass each way, no separate copy). TPMG_MIXED runs iterative refinement:
 * r = f - A u in double-word arithmetic (stored FP32), one FP32 V-cycle for A e = r from e = 0,
 * u += e in double-word arithmetic. Returns TPMG_OK, TPMG_ERR_NOT_CONVERGED or
 * TPMG_ERR_NONFINITE (u then holds the last iterate), or an argument/CUDA error. */
tpmg_status tpmg_mg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u,
                          tpmg_info* info, void* stream);
/* Host-buffer solve, the paper's "total solution time" path (Sec. 5.1, Table SingleGPUTiming: the
 * right-hand side copied to the device and transposed from the vertically contiguous layout of the
 * CPU code to the horizontally contiguous one of Eq. (13), the solve, the solution transposed and
 * copied back). f_host, u_host: HOST arrays of the finest level's nx*ny*nz values (double; float for
 * TPMG_F32), in layout TPMG_LAYOUT_X (x fastest, index (k*ny + j)*nx + i, as on the device) or
 * TPMG_LAYOUT_Z (z fastest: column c = j*nx + i holds its nz values at c*nz .. c*nz + nz-1).
 * Page-locked memory (cudaHostAlloc) lets the copies run at the link's rate; pageable memory works
 * too, with the driver's staging. u_host is read as the initial guess unless prm->zero_guess, and
 * receives the final iterate (also on TPMG_ERR_NOT_CONVERGED / TPMG_ERR_NONFINITE). The copies,
 * the transposes (one tiled kernel each way) and the solve (tpmg_mg_solve on library-owned device
 * fields, allocated on the first call) are ordered on `stream`; returns after u_host is written.
 * info->ms (if info) is the device time of the whole call; *ms_io (if ms_io) the part spent in the
 * copies and transposes. Same return values as tpmg_mg_solve. */
typedef enum { TPMG_LAYOUT_X = 0, TPMG_LAYOUT_Z = 1 } tpmg_layout;
tpmg_status tpmg_mg_solve_host(tpmg_op* op, const tpmg_params* prm, int layout, const void* f_host,
                               void* u_host, tpmg_info* info, double* ms_io, void* stream);
/* One V-cycle from u (in place), for testing a cycle against a reference. */
tpmg_status tpmg_vcycle(tpmg_op* op, const tpmg_params* prm, const void* f, void* u, void* stream);
/* Line-preconditioned CG (Sec. 2.2) with the fused kernels of Sec. 3.1. prec: TPMG_F64, TPMG_F32
 * or TPMG_DW (TPMG_MIXED is rejected). Same return values as tpmg_mg_solve. */
tpmg_status tpmg_cg_solve(tpmg_op* op, const tpmg_params* prm, const void* f, void* u,
                          tpmg_info* info, void* stream);

/* ---------------------------------------------------------------- profiling */
typedef enum {
    TPMG_K_SMOOTH = 0,          /* finest level Smooth */
    TPMG_K_RESIDUAL = 1,        /* finest level Residual */
    TPMG_K_APPLY_A = 2,         /* finest level y = A x */
    TPMG_K_LINE_SOLVE = 3,      /* finest level x = M^{-1} b */
    TPMG_K_RESTRICT_SMOOTH = 4, /* level L-1 RestrictSmooth from level L */
    TPMG_K_PROLONGATE = 5,      /* level L-1 -> L Prolongate */
    TPMG_K_CG_SPMV = 6,         /* fused CG SpMV on the finest level */
    TPMG_K_CG_TRIDIAG = 7,      /* fused CG Tridiag on the finest level */
    TPMG_K_RESIDUAL_RESTRICT = 8, /* level L Residual + level L-1 RestrictSmooth, fused */
    TPMG_K_COUNT = 9
} tpmg_kernel;
/* Launches kernel `k` of precision `prec` (TPMG_F64, TPMG_F32 or TPMG_DW) `reps` times on the
 * operator's own workspace buffers of that precision (whatever they hold, e.g. after a solve) and
 * writes the mean duration of one launch in ms (CUDA events on `stream`) to *ms. Synchronises
 * `stream`. Allocates the workspace of `prec` if needed. */
tpmg_status tpmg_time_kernel(tpmg_op* op, tpmg_precision prec, tpmg_kernel k, int reps, double* ms,
                             void* stream);
/* Number of kernel launches this library has issued since the process started (a graph replay
 * counts every kernel node it contains). */
unsigned long long tpmg_kernel_launches(void);
/* Arithmetic rate of the current GPU, the denominator of the ALU rooflines (the paper's kernels
 * are bandwidth-bound on its K20X, Sec. 4; on a part with a narrow FP64 pipe the same per-cell
 * arithmetic can bind first). which: 0 = FP64 fused multiply-add, 1 = FP64 add, 2 = FP64 multiply,
 * 3 = FP32 fused multiply-add. Runs a full-occupancy grid of independent dependent chains `reps`
 * times (after one warm-up) on the legacy default stream and writes the best launch's operations
 * per second (one operation = one instruction's result per thread, so a multiply-add counts once)
 * to *ops_per_s and its duration in ms to *ms_per_launch (may be NULL). Allocates and frees a small
 * sink buffer; synchronises the device. */
tpmg_status tpmg_measure_alu_rate(int which, int reps, double* ops_per_s, double* ms_per_launch);

/* ---------------------------------------------------------------- autotuning
 * The plane-pipelined Smooth has TPMG_NUM_VARIANTS variants: tile shapes (columns per block x ring
 * depth) with the Thomas stack in shared memory (0-2), persistent ones with the stack in global
 * scratch (3, 4), persistent ones with two columns per thread that steer L2 residency of the stack
 * with eviction hints (5-7), and, in FP32 only, one warp per tile of 128 x 1 or 128 x 2 columns with
 * four columns per thread and the Thomas factors 1/m_k formed in registers (8-11: one-row tiles;
 * one-row tiles run as overlapping forward/backward stages; two-row tiles; one-row tiles with a
 * shallower ring). A level that was never tuned or set takes, in FP32, variant 8 where the level
 * fits one tile per resident warp (nx % 128 == 0), else 5; double-word takes 6 where nx % 64 == 0;
 * otherwise variant 3 (native FP64: variant 0). Variants 8-11 in other precisions run the default.
 * tpmg_autotune times each of them `reps` times on every level of precision `prec` (on the
 * operator's workspace, CUDA events on `stream`) and keeps the fastest per level; if variants_out
 * is not NULL it receives the choice of level l in variants_out[l] (host array of L+1 ints).
 * tpmg_set_variant sets one level's choice (e.g. from a saved tuning table). Both invalidate the
 * operator's cached CUDA graphs. Variants change the schedule, not the per-cell arithmetic (only the
 * grouping of the residual norm's partial sums differs). */
#define TPMG_NUM_VARIANTS 12
tpmg_status tpmg_autotune(tpmg_op* op, tpmg_precision prec, int reps, int* variants_out, void* stream);
tpmg_status tpmg_set_variant(tpmg_op* op, tpmg_precision prec, int level, int variant);

/* ---------------------------------------------------------------- learned preconditioner stage
 * A 3-D convolutional network used as an extra preconditioner stage inside flexible CG (an
 * extension of the method: the paper's preconditioners are the line solve and the V-cycle).
 * Architecture: cin (1 or 2) -> 16 -> 16 -> 16 -> 1 channels, 3x3x3 kernels, ReLU after the first
 * three layers, periodic padding in x and y and zero padding in z (the problem's boundaries).
 * Parameters: tpmg_nn_nparams(cin) floats, flat W1 b1 W2 b2 W3 b3 W4 b4 with W[co][ci][dz][dy][dx].
 * Inference and training run in BF16 with FP32 accumulation on the tensor cores (all four layers of
 * the forward pass where nx % 128 == 0 and ny % 4 == 0, the 16 -> 16 layers and their gradients
 * otherwise); FP32 master weights; Adam (lr given, beta 0.9/0.999, eps 1e-8).
 * Network inputs x are DEVICE fp32, channels-last (cin values per cell, cell index (k*ny+j)*nx+i);
 * outputs and targets DEVICE fp32 (one value per cell). Grids need nx % 64 == 0 and ny % 2 == 0. */
typedef struct tpmg_nn tpmg_nn;
int tpmg_nn_nparams(int cin);
/* params_host: HOST array of nparams floats, or NULL for all zeros */
tpmg_status tpmg_nn_create(int cin, const float* params_host, tpmg_nn** out);
tpmg_status tpmg_nn_destroy(tpmg_nn* nn);
tpmg_status tpmg_nn_get_params(const tpmg_nn* nn, float* host);
/* replaces the parameters and resets the Adam moments */
tpmg_status tpmg_nn_set_params(tpmg_nn* nn, const float* host);
tpmg_status tpmg_nn_forward(tpmg_nn* nn, int nx, int ny, int nz, const float* x, float* out, void* stream);
/* loss = mean over cells of (NN(x) - target)^2 into the DEVICE double *loss_out; its gradient
 * w.r.t. the parameters into the DEVICE array grad_out (nparams floats) if not NULL */
tpmg_status tpmg_nn_loss_grad(tpmg_nn* nn, int nx, int ny, int nz, const float* x, const float* target,
                              double* loss_out, float* grad_out, void* stream);
/* one Adam step on the loss above */
tpmg_status tpmg_nn_train_step(tpmg_nn* nn, int nx, int ny, int nz, const float* x, const float* target,
                               double lr, double* loss_out, void* stream);
/* Residual loss for the operator op (its finest level, FP32 arithmetic; the grid is op's, with the
 * network's nx % 64 == 0 and ny even rule): with r the input's channel 0, y = NN(x) and D = diag(A),
 * loss = mean over cells of (r - A D^{-1} y)^2 -- the mean square of the residual that the
 * correction D^{-1} y leaves, which is what the learned stage's acceptance test compares -- into
 * the DEVICE double *loss_out, and its parameter gradient (through
 * dLoss/dy = -2 D^{-1} A (r - A D^{-1} y) / n) into grad_out (DEVICE, nparams floats) if not NULL.
 * x as in tpmg_nn_forward. */
tpmg_status tpmg_nn_loss_grad_residual(tpmg_nn* nn, tpmg_op* op, const float* x, double* loss_out, float* grad_out,
                                       void* stream);
/* one Adam step on the residual loss */
tpmg_status tpmg_nn_train_step_residual(tpmg_nn* nn, tpmg_op* op, const float* x, double lr, double* loss_out,
                                        void* stream);
/* Training pair from an iterate u_k of a solve on op's finest level with exact solution u_star and
 * residual r (DEVICE doubles, one per cell): x = (r/rms(r) and, if cin == 2, aux per column (DEVICE
 * fp32, ny*nx)) in BF16-rounded fp32, target = D (u_star - u_k)/rms(r) with D = diag(A) -- the
 * error in the network's output unit (target_out may be NULL, then u_star and u_k may be too).
 * Synchronises `stream`; allocates its scratch (a training utility). */
tpmg_status tpmg_nn_make_pair(tpmg_op* op, int cin, const double* r, const double* u_star, const double* u_k,
                              const float* aux, float* x_out, float* target_out, void* stream);
/* Flexible CG with truncation 1 (Notay's FCG(1)) for A u = f on the finest level, double-word
 * vectors; preconditioner: one FP32 V-cycle z1 of r (the mixed solver's inner cycle, prm's
 * smoothing parameters) and, if nn is not NULL, the learned correction
 * z = z1 + rms(r1) D^{-1} NN(r1/rms(r1)), r1 = r - A z1, D = diag(A) (the network answers in units
 * of a Jacobi step), kept only when ||r - A z|| < ||r1|| (else z = z1).
 * aux: DEVICE fp32 second input channel per column (2-channel networks), else NULL.
 * *nn_accepted (host, may be NULL) receives how many learned corrections were kept. Stops on
 * Eq. (10) like the other solvers; same return values as tpmg_mg_solve. */
tpmg_status tpmg_fcg_solve(tpmg_op* op, tpmg_nn* nn, const float* aux, const tpmg_params* prm, const double* f,
                           double* u, tpmg_info* info, int* nn_accepted, void* stream);

/* ---------------------------------------------------------------- allocation-free variant
 * The paper has no counterpart: this entry point exists for callers that must not allocate device
 * memory while they run -- applications whose framework already owns nearly all device memory
 * through its own pool (a raw cudaMalloc there can fail or fragment that pool) and latency-critical
 * loops where cudaMalloc's implicit device synchronisation is not acceptable. Every other entry
 * point allocates workspace inside its operator; this one needs no operator and allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).
 *
 * r = f - A u and *norm_out = ||r||_2 on one nx x ny x nz level, native FP64, with A as in the
 * header comment: cx, cy the horizontal couplings, v a DEVICE array of ny*nx vertical couplings
 * (index j*nx + i); u, f, r DEVICE arrays of nz*ny*nx doubles (x fastest, r must not overlap u or
 * f); norm_out a DEVICE double. Same kernels and results as tpmg_residual(op, L, TPMG_F64, ...).
 *
 * Scratch: one partial sum per thread block in a fixed file-scope device array of
 * TPMG_NOALLOC_MAX_BLOCKS doubles (512 KB), held by every GPU that loads the library until the
 * process exits. The number of blocks is that of the residual kernel the grid takes: at most 1024
 * on grids of at most 4096 columns; on grids with nx a multiple of 64, even ny and 16-byte aligned
 * u, f, r (the two-column persistent sweep) at most 16 per SM whatever the size; otherwise
 * (nx/32)*(ny/4) blocks for nx a multiple of 32 and ny of 4, else one per 32 x 4 columns rounded
 * up. A call needing more than TPMG_NOALLOC_MAX_BLOCKS (above about 8.4 million columns on the
 * last two kinds of grid) is rejected with TPMG_ERR_ARG and a message in
 * tpmg_noalloc_last_error() before anything is launched. All calls share the array and each call
 * overwrites the entries it reads before reading them, so no clearing is needed; calls that
 * overlap on the GPU (on different streams or host threads without ordering) race on it and must
 * be serialised. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of the process; make
 * that first call before any stream capture, and do not use this entry point on a device after a
 * cudaDeviceReset there (the kept address would belong to the destroyed context). */
#define TPMG_NOALLOC_MAX_BLOCKS 65536
tpmg_status tpmg_residual_norm_noalloc(int nx, int ny, int nz, double cx, double cy, const double* v,
                                       const double* u, const double* f, double* r, double* norm_out,
                                       void* stream);
const char* tpmg_noalloc_last_error(void);

/* ---------------------------------------------------------------- the cubed-sphere panel operator
 * The paper's own operator: Eq. (1) (Sec. 2.1) discretised by cell-centred finite volumes on one
 * gnomonic cubed-sphere panel (Sec. 2.1.1: homogeneous Dirichlet on the panel boundary, Neumann at
 * r = 1 and r = 1 + H), in the factorised form of Eq. (14):
 *   A_{T,T'} = alpha_{TT'} I,   A_T = |T| diag(a) - alpha_T I + |T| tridiag(-(b + c), b, c),
 * with |T| the cell's area on the unit sphere (exact), alpha_{TT'} = -omega2 |e| / d for each face
 * (|e| the edge's great-circle length, d the great-circle distance of the cell centres; a face on the
 * panel boundary couples to a ghost value of 0), alpha_T their sum, and the radial vectors of nz
 * cells on [1, 1 + H]: a_k = (r_{k+1/2}^3 - r_{k-1/2}^3) / (3 h_z), b_k = -omega2 lambda2
 * r_{k-1/2}^2 / h_z^2, c_k = -omega2 lambda2 r_{k+1/2}^2 / h_z^2 (b_0 = c_{nz-1} = 0), h_z = H / nz.
 * The equations are integrated over the cells. Coarse levels rediscretise the same panel (Sec. 3.1).
 * The panel [-extent, extent]^2 of cube-face coordinates (extent 1: a whole cube face) maps to the
 * sphere by (X, Y, 1) / sqrt(1 + X^2 + Y^2). The unit entry points and CG are native FP64.
 *
 * tpmg_cg_solve on a panel operator (TPMG_F64) runs line-preconditioned CG with the fused SpMV and
 * Tridiag kernels of Sec. 3.1 on the panel stencil.
 * tpmg_mg_solve on a panel operator runs Algorithm 1 in native FP64 (prm->prec TPMG_F64) or as
 * iterative refinement (TPMG_MIXED): outer residual r = f - A u in FP64, one FP32 V-cycle on A e = r
 * (geometry and Thomas factors rounded once from the FP64 ones), u += e in FP64, until the FP64
 * residual meets prm->tol. Other precisions return TPMG_ERR_ARG. The cycle's kernels:
 * RestrictSmooth sums the 2 x 2 children's residuals (the integrated residual of the coarse cell),
 * Prolongate is bilinear in the logical grid with a ghost value of 0 beyond the panel. Fields are
 * DEVICE doubles, nz*ny*nx per level, x fastest. The unit entry points below run one kernel on level
 * `level` (1 = coarsest) on the caller's stream; norm_out (DEVICE double or NULL) receives
 * ||f - A u||. Errors: TPMG_ERR_ARG (not a panel operator, level out of range, NULL field). */
tpmg_status tpmg_create_panel_operator(const tpmg_grid* g, double omega2, double lambda2, double H,
                                       double extent, tpmg_op** out);
/* the geometry of level `level` as computed by the library: HOST arrays |T| (ny*nx), x-face
 * coefficients (ny*(nx+1), index j*(nx+1) + i for the face between cells i-1 and i) and y-face
 * coefficients ((ny+1)*nx, index j*nx + i for the face between rows j-1 and j); any may be NULL */
tpmg_status tpmg_panel_level_geometry(const tpmg_op* op, int level, double* area, double* ax, double* ay);
tpmg_status tpmg_panel_apply_A(tpmg_op* op, int level, const double* x, double* y, void* stream);
/* x = M^{-1} b, M the column blocks A_T (vertical line relaxation, Sec. 2.2) */
tpmg_status tpmg_panel_line_solve(tpmg_op* op, int level, const double* b, double* x, void* stream);
/* u_out = u + rho M^{-1}(f - A u) (Eq. (11)); u_out must not overlap u */
tpmg_status tpmg_panel_smooth(tpmg_op* op, int level, double rho, const double* u, const double* f,
                              double* u_out, double* norm_out, void* stream);
tpmg_status tpmg_panel_residual(tpmg_op* op, int level, const double* u, const double* f, double* r,
                                double* norm_out, void* stream);
/* f_c = R r_fine (sum of the children), u_c = rho M_c^{-1} f_c on the coarse level `level` */
tpmg_status tpmg_panel_restrict_smooth(tpmg_op* op, int level, double rho, const double* r_fine, double* f_c,
                                       double* u_c, void* stream);
/* u_f += P u_c with u_f on level `level` and u_c on level - 1 */
tpmg_status tpmg_panel_prolongate(tpmg_op* op, int level, const double* u_c, double* u_f, void* stream);

/* Batched solve: nprob independent problems (each its own operator, all on one device, no operator
 * twice) solved together by one cooperative persistent kernel -- the mixed-precision iterative
 * refinement of tpmg_mg_solve (prm->prec must be TPMG_MIXED) with the steps of every problem's
 * FP32 V-cycle interleaved phase by phase, a bounded grid barrier between phases (prm->timeout_s)
 * and a per-problem convergence mask. f[b], u[b]: DEVICE double fields of problem b's finest level;
 * infos: NULL or nprob entries (ms = the whole batch). The tables and a CUDA graph of the whole
 * solve (conversions, the persistent launch) are built on the first call for a set of operators
 * and parameters and replayed afterwards. Returns TPMG_ERR_TIMEOUT if a barrier wait ran out (the
 * device stays usable), TPMG_ERR_NONFINITE or TPMG_ERR_NOT_CONVERGED if any problem ended so. */
tpmg_status tpmg_mg_solve_batched(int nprob, tpmg_op* const* ops, const tpmg_params* prm,
                                  const double* const* f, double* const* u, tpmg_info* infos, void* stream);

const char* tpmg_status_string(tpmg_status s);
/* Message of the last error in the calling thread ("" if none). */
const char* tpmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TPMG_H */
