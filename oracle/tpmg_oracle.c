/*
 * tpmg_oracle.c -- the ORACLE: a plain, slow, obviously correct FP64 CPU implementation of the
 * tensor-product multigrid and line-preconditioned CG method of Mueller, Scheichl & Vainikko,
 * "Petascale elliptic solvers for anisotropic PDEs on GPU clusters" (arXiv:1402.3545).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test-suite, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py may load it. The product (the CUDA library) never calls it and shares no code,
 * header, table or helper with it.
 *
 * Problem (Sec. 2.1.1, flat-box form of Eq. (6) "TridiagonalPDE"), periodic horizontally and with
 * homogeneous Neumann conditions at the top and bottom (Sec. 2.1, below Eq. (2)):
 *   (A x)_{ijk} = (1 + 2cx + 2cy + v_ij * nvert(k)) x_{ijk}
 *                 - cx (x_{i-1,j,k} + x_{i+1,j,k}) - cy (x_{i,j-1,k} + x_{i,j+1,k})
 *                 - v_ij (x_{i,j,k-1} [k>0] + x_{i,j,k+1} [k<nz-1])
 * with cx = omega^2/hx^2, cy = omega^2/hy^2, v_ij = omega^2 lambda^2(x_i,y_j)/hz^2 and
 * nvert(k) = number of existing vertical neighbours (2 inside, 1 at a Neumann end: the mirror
 * ghost cell of the cell-centred discretisation). Horizontal indices wrap periodically.
 *
 * Storage: every 3-D field is a contiguous array of nz*ny*nx doubles with x fastest,
 * index (k*ny + j)*nx + i (x-contiguous, as in Eq. (13) "MemoryMapSingleGPU").
 * The vertical coefficient v is an array of ny*nx doubles (one value per column), index j*nx + i.
 *
 * Multigrid level numbering follows Sec. 2.2: level 1 is the coarsest, level L the finest.
 * Coarse level l has half the horizontal cells of level l+1 in each direction, the same nz,
 * cx^(l) = cx^(l+1)/4, cy^(l) = cy^(l+1)/4 (the horizontal mesh width doubles) and v^(l) the
 * average of the 2x2 children's v (the rediscretised vertical coefficient).
 *
 * Functions whose result has no independent closed form are marked "parity unpinned" where that
 * applies; the pins for everything else live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads: the loops over cells or columns may run on several host threads (OpenMP, when the
 * library is built with it). Every cell or column is computed by the same code whichever thread
 * takes it, so results do not depend on the thread count; the dot products and norms run on one
 * thread in index order, so they do not either. orc_set_threads(n) sets the count (n >= 1) and
 * returns the count in effect. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define ORC_MAX_LEVELS 16

static size_t idx3(int nx, int ny, int i, int j, int k) {
    return ((size_t)k * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i;
}

static int wrap(int i, int n) {
    if (i < 0) return i + n;
    if (i >= n) return i - n;
    return i;
}

/* y = A x : the matrix-free 7-point operator (Sec. 2.1.1 flat-box entries; Sec. 3.1 Eq. (14)
 * "LocalMatrixStencil" with |T| = 1, a = 1, alpha_{TT'} diag(d) = -cx or -cy, b = c = -v). */
void orc_apply_A(int nx, int ny, int nz, double cx, double cy, const double *v,
                 const double *x, double *y) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double vij = v[(size_t)j * nx + i];
                double diag = 1.0 + 2.0 * cx + 2.0 * cy;
                double vert = 0.0;
                if (k > 0) {
                    diag += vij;
                    vert += x[idx3(nx, ny, i, j, k - 1)];
                }
                if (k < nz - 1) {
                    diag += vij;
                    vert += x[idx3(nx, ny, i, j, k + 1)];
                }
                double xw = x[idx3(nx, ny, wrap(i - 1, nx), j, k)];
                double xe = x[idx3(nx, ny, wrap(i + 1, nx), j, k)];
                double xs = x[idx3(nx, ny, i, wrap(j - 1, ny), k)];
                double xn = x[idx3(nx, ny, i, wrap(j + 1, ny), k)];
                y[idx3(nx, ny, i, j, k)] = diag * x[idx3(nx, ny, i, j, k)] - cx * (xw + xe) -
                                           cy * (xs + xn) - vij * vert;
            }
}

/* x = M^{-1} b : vertical line relaxation. M is block diagonal with one tridiagonal block A_T
 * per column (the first term of Eq. (6); Sec. 2.2), i.e. the diagonal of A plus the vertical
 * couplings. Each block is solved by the Thomas algorithm in textbook order: forward
 * elimination k = 0..nz-1, then back substitution k = nz-1..0. */
void orc_line_solve(int nx, int ny, int nz, double cx, double cy, const double *v,
                    const double *b, double *x) {
#pragma omp parallel
    {
    double *cp = (double *)malloc(sizeof(double) * (size_t)nz);
    double *dp = (double *)malloc(sizeof(double) * (size_t)nz);
#pragma omp for collapse(2) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double vij = v[(size_t)j * nx + i];
            for (int k = 0; k < nz; ++k) {
                double diag = 1.0 + 2.0 * cx + 2.0 * cy;
                if (k > 0) diag += vij;
                if (k < nz - 1) diag += vij;
                double lower = (k > 0) ? -vij : 0.0;     /* coefficient of x_{k-1} */
                double upper = (k < nz - 1) ? -vij : 0.0; /* coefficient of x_{k+1} */
                double rhs = b[idx3(nx, ny, i, j, k)];
                if (k == 0) {
                    cp[k] = upper / diag;
                    dp[k] = rhs / diag;
                } else {
                    double den = diag - lower * cp[k - 1];
                    cp[k] = upper / den;
                    dp[k] = (rhs - lower * dp[k - 1]) / den;
                }
            }
            x[idx3(nx, ny, i, j, nz - 1)] = dp[nz - 1];
            for (int k = nz - 2; k >= 0; --k)
                x[idx3(nx, ny, i, j, k)] = dp[k] - cp[k] * x[idx3(nx, ny, i, j, k + 1)];
        }
    free(cp);
    free(dp);
    }
}

/* r = f - A u : the Residual kernel of Sec. 3.1. */
void orc_residual(int nx, int ny, int nz, double cx, double cy, const double *v,
                  const double *u, const double *f, double *r) {
    size_t n = (size_t)nx * ny * nz;
    orc_apply_A(nx, ny, nz, cx, cy, v, u, r);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) r[p] = f[p] - r[p];
}

/* u_out = u + rho M^{-1} (f - A u) : one block-Jacobi smoothing step, Eq. (11)
 * "MultigridSmoother". u_out may not alias u. */
void orc_smooth(int nx, int ny, int nz, double cx, double cy, const double *v, double rho,
                const double *u, const double *f, double *u_out) {
    size_t n = (size_t)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    orc_residual(nx, ny, nz, cx, cy, v, u, f, r);
    orc_line_solve(nx, ny, nz, cx, cy, v, r, z);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) u_out[p] = u[p] + rho * z[p];
    free(r);
    free(z);
}

/* f_c = R r_f : cell-average restriction in the horizontal direction only (Sec. 2.2,
 * text after Eq. (12)); the coarse cell (I,J) averages its 2x2 children. nxf, nyf even. */
void orc_restrict(int nxf, int nyf, int nz, const double *rf, double *fc) {
    int nxc = nxf / 2, nyc = nyf / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int J = 0; J < nyc; ++J)
            for (int I = 0; I < nxc; ++I) {
                double s = rf[idx3(nxf, nyf, 2 * I, 2 * J, k)] +
                           rf[idx3(nxf, nyf, 2 * I + 1, 2 * J, k)] +
                           rf[idx3(nxf, nyf, 2 * I, 2 * J + 1, k)] +
                           rf[idx3(nxf, nyf, 2 * I + 1, 2 * J + 1, k)];
                fc[idx3(nxc, nyc, I, J, k)] = 0.25 * s;
            }
}

/* u_f += P u_c : horizontal (bi)linear interpolation of cell-centred data (Sec. 2.2, text after
 * Eq. (12)). The fine cell 2I+a (a in {0,1}) lies a quarter of a coarse width from the centre of
 * coarse cell I, towards coarse cell I-1 (a = 0) or I+1 (a = 1): weights 3/4 and 1/4 per
 * direction, i.e. 9/16, 3/16, 3/16, 1/16 in 2-D. Coarse indices wrap periodically. */
void orc_prolongate_add(int nxc, int nyc, int nz, const double *uc, double *uf) {
    int nxf = 2 * nxc, nyf = 2 * nyc;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nyf; ++j)
            for (int i = 0; i < nxf; ++i) {
                int I = i / 2, J = j / 2;
                int I2 = wrap((i % 2 == 0) ? I - 1 : I + 1, nxc);
                int J2 = wrap((j % 2 == 0) ? J - 1 : J + 1, nyc);
                double val = 0.75 * 0.75 * uc[idx3(nxc, nyc, I, J, k)] +
                             0.25 * 0.75 * uc[idx3(nxc, nyc, I2, J, k)] +
                             0.75 * 0.25 * uc[idx3(nxc, nyc, I, J2, k)] +
                             0.25 * 0.25 * uc[idx3(nxc, nyc, I2, J2, k)];
                uf[idx3(nxf, nyf, i, j, k)] += val;
            }
}

/* v_c(I,J) = average of the four children's v (coarse-level vertical coefficient). */
void orc_coarsen_v(int nxf, int nyf, const double *vf, double *vc) {
    int nxc = nxf / 2, nyc = nyf / 2;
    for (int J = 0; J < nyc; ++J)
        for (int I = 0; I < nxc; ++I)
            vc[(size_t)J * nxc + I] =
                0.25 * (vf[(size_t)(2 * J) * nxf + 2 * I] + vf[(size_t)(2 * J) * nxf + 2 * I + 1] +
                        vf[(size_t)(2 * J + 1) * nxf + 2 * I] +
                        vf[(size_t)(2 * J + 1) * nxf + 2 * I + 1]);
}

double orc_dot(size_t n, const double *a, const double *b) {
    double s = 0.0;
    for (size_t p = 0; p < n; ++p) s += a[p] * b[p];
    return s;
}

double orc_norm2(size_t n, const double *a) { return sqrt(orc_dot(n, a, a)); }

/* ------------------------------------------------------------------------------------------ */
/* Multigrid hierarchy and V-cycle (Sec. 2.2, Algorithm 1).                                     */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int L, nz;
    int nx[ORC_MAX_LEVELS + 1], ny[ORC_MAX_LEVELS + 1];
    double cx[ORC_MAX_LEVELS + 1], cy[ORC_MAX_LEVELS + 1];
    double *v[ORC_MAX_LEVELS + 1];
    double *u[ORC_MAX_LEVELS + 1], *f[ORC_MAX_LEVELS + 1], *r[ORC_MAX_LEVELS + 1];
    double *tmp[ORC_MAX_LEVELS + 1];
    int nu_pre, nu_post, n_coarse;
    double rho;
} orc_mg;

static size_t lvl_n(const orc_mg *mg, int l) {
    return (size_t)mg->nx[l] * (size_t)mg->ny[l] * (size_t)mg->nz;
}

/* Builds the hierarchy for a fine grid nx x ny x nz with L levels. The fine-level u and f
 * pointers are attached later by the solver; coarse-level vectors are owned here. */
static int mg_setup(orc_mg *mg, int nx, int ny, int nz, int L, double cx, double cy,
                    const double *v) {
    if (L < 1 || L > ORC_MAX_LEVELS) return -1;
    if (nx % (1 << (L - 1)) != 0 || ny % (1 << (L - 1)) != 0) return -1;
    memset(mg, 0, sizeof(*mg));
    mg->L = L;
    mg->nz = nz;
    for (int l = L; l >= 1; --l) {
        mg->nx[l] = (l == L) ? nx : mg->nx[l + 1] / 2;
        mg->ny[l] = (l == L) ? ny : mg->ny[l + 1] / 2;
        mg->cx[l] = (l == L) ? cx : mg->cx[l + 1] / 4.0;
        mg->cy[l] = (l == L) ? cy : mg->cy[l + 1] / 4.0;
        size_t ncol = (size_t)mg->nx[l] * mg->ny[l];
        mg->v[l] = (double *)malloc(sizeof(double) * ncol);
        if (l == L)
            memcpy(mg->v[l], v, sizeof(double) * ncol);
        else
            orc_coarsen_v(mg->nx[l + 1], mg->ny[l + 1], mg->v[l + 1], mg->v[l]);
        size_t n = lvl_n(mg, l);
        mg->r[l] = (double *)calloc(n, sizeof(double));
        mg->tmp[l] = (double *)calloc(n, sizeof(double));
        if (l < L) {
            mg->u[l] = (double *)calloc(n, sizeof(double));
            mg->f[l] = (double *)calloc(n, sizeof(double));
        }
    }
    return 0;
}

static void mg_free(orc_mg *mg) {
    for (int l = 1; l <= mg->L; ++l) {
        free(mg->v[l]);
        free(mg->r[l]);
        free(mg->tmp[l]);
        if (l < mg->L) {
            free(mg->u[l]);
            free(mg->f[l]);
        }
    }
}

/* One smoothing step in place on level l (via a temporary: u <- u + rho M^{-1}(f - A u)). */
static void mg_smooth(orc_mg *mg, int l) {
    size_t n = lvl_n(mg, l);
    orc_smooth(mg->nx[l], mg->ny[l], mg->nz, mg->cx[l], mg->cy[l], mg->v[l], mg->rho, mg->u[l],
               mg->f[l], mg->tmp[l]);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) mg->u[l][p] = mg->tmp[l][p];
}

/* Restriction of the next finer level's residual followed by the first smoothing step from a
 * zero initial guess, u = rho M^{-1} f (the fused "RestrictSmooth" step of Algorithm 1). */
static void mg_restrict_smooth(orc_mg *mg, int l) {
    size_t n = lvl_n(mg, l);
    orc_restrict(mg->nx[l + 1], mg->ny[l + 1], mg->nz, mg->r[l + 1], mg->f[l]);
    orc_line_solve(mg->nx[l], mg->ny[l], mg->nz, mg->cx[l], mg->cy[l], mg->v[l], mg->f[l],
                   mg->u[l]);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) mg->u[l][p] *= mg->rho;
}

/* Algorithm 1 (VCycle), with nu_pre pre- and nu_post post-smoothing steps on every level and
 * n_coarse smoothing steps in total on the coarsest level (the first of which is fused with
 * the restriction). With L == 1 the cycle is n_coarse smoothing steps on the only level. */
static void mg_vcycle(orc_mg *mg, int l) {
    int L = mg->L;
    if (L == 1) {
        for (int s = 0; s < mg->n_coarse; ++s) mg_smooth(mg, 1);
        return;
    }
    if (l == 1) {
        mg_restrict_smooth(mg, 1);
        for (int s = 1; s < mg->n_coarse; ++s) mg_smooth(mg, 1);
        return;
    }
    if (l == L) {
        for (int s = 0; s < mg->nu_pre; ++s) mg_smooth(mg, l);
    } else {
        mg_restrict_smooth(mg, l);
        for (int s = 1; s < mg->nu_pre; ++s) mg_smooth(mg, l);
    }
    orc_residual(mg->nx[l], mg->ny[l], mg->nz, mg->cx[l], mg->cy[l], mg->v[l], mg->u[l],
                 mg->f[l], mg->r[l]);
    mg_vcycle(mg, l - 1);
    orc_prolongate_add(mg->nx[l - 1], mg->ny[l - 1], mg->nz, mg->u[l - 1], mg->u[l]);
    for (int s = 0; s < mg->nu_post; ++s) mg_smooth(mg, l);
}

/* One V-cycle on the fine level: u is updated in place. Returns 0 on success. */
int orc_vcycle(int nx, int ny, int nz, int L, double cx, double cy, const double *v,
               int nu_pre, int nu_post, int n_coarse, double rho, const double *f, double *u) {
    orc_mg mg;
    if (mg_setup(&mg, nx, ny, nz, L, cx, cy, v) != 0) return -1;
    mg.nu_pre = nu_pre;
    mg.nu_post = nu_post;
    mg.n_coarse = n_coarse;
    mg.rho = rho;
    mg.u[L] = u;
    mg.f[L] = (double *)f;
    mg_vcycle(&mg, L);
    mg_free(&mg);
    return 0;
}

/* Multigrid solve (Sec. 2.2): repeated V-cycles from the initial guess in u until
 * ||f - A u|| / ||f - A u_0|| < tol (Eq. (10) "epsilonTolerance") or max_iter cycles.
 * history (length max_iter+1, may be NULL) receives the relative residual before the first and
 * after every cycle. Returns the number of cycles done, or -1 on bad arguments; *converged is
 * set to 1 if the tolerance was met. */
int orc_mg_solve(int nx, int ny, int nz, int L, double cx, double cy, const double *v,
                 int nu_pre, int nu_post, int n_coarse, double rho, double tol, int max_iter,
                 const double *f, double *u, double *history, int *converged) {
    orc_mg mg;
    if (mg_setup(&mg, nx, ny, nz, L, cx, cy, v) != 0) return -1;
    mg.nu_pre = nu_pre;
    mg.nu_post = nu_post;
    mg.n_coarse = n_coarse;
    mg.rho = rho;
    mg.u[L] = u;
    mg.f[L] = (double *)f;
    size_t n = lvl_n(&mg, L);
    double *r = (double *)malloc(sizeof(double) * n);
    orc_residual(nx, ny, nz, cx, cy, v, u, f, r);
    double r0 = orc_norm2(n, r);
    int it = 0;
    *converged = 0;
    if (history) history[0] = 1.0;
    if (r0 == 0.0) {
        *converged = 1;
    } else {
        while (it < max_iter) {
            mg_vcycle(&mg, L);
            ++it;
            orc_residual(nx, ny, nz, cx, cy, v, u, f, r);
            double rel = orc_norm2(n, r) / r0;
            if (history) history[it] = rel;
            if (rel < tol) {
                *converged = 1;
                break;
            }
        }
    }
    free(r);
    mg_free(&mg);
    return it;
}

/* ------------------------------------------------------------------------------------------ */
/* Preconditioned CG (Sec. 2.2, Eqs. (8)-(9)), textbook form (Saad, Alg. 9.1), M = vertical line */
/* relaxation. The fused GPU ordering of Sec. 3.1 is algebraically the same iteration.         */
/* ------------------------------------------------------------------------------------------ */
int orc_cg_solve(int nx, int ny, int nz, double cx, double cy, const double *v, double tol,
                 int max_iter, const double *f, double *u, double *history, int *converged) {
    size_t n = (size_t)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    orc_residual(nx, ny, nz, cx, cy, v, u, f, r);
    double r0 = orc_norm2(n, r);
    orc_line_solve(nx, ny, nz, cx, cy, v, r, z);
    memcpy(p, z, sizeof(double) * n);
    double rz = orc_dot(n, r, z);
    int it = 0;
    *converged = 0;
    if (history) history[0] = 1.0;
    if (r0 == 0.0) {
        *converged = 1;
    } else {
        while (it < max_iter) {
            orc_apply_A(nx, ny, nz, cx, cy, v, p, q);
            double alpha = rz / orc_dot(n, p, q);
#pragma omp parallel for schedule(static)
            for (size_t s = 0; s < n; ++s) {
                u[s] += alpha * p[s];
                r[s] -= alpha * q[s];
            }
            ++it;
            double rel = orc_norm2(n, r) / r0;
            if (history) history[it] = rel;
            if (rel < tol) {
                *converged = 1;
                break;
            }
            orc_line_solve(nx, ny, nz, cx, cy, v, r, z);
            double rz_new = orc_dot(n, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
#pragma omp parallel for schedule(static)
            for (size_t s = 0; s < n; ++s) p[s] = z[s] + beta * p[s];
        }
    }
    free(r);
    free(z);
    free(p);
    free(q);
    return it;
}

/* ------------------------------------------------------------------------------------------ */
/* Iterative refinement around V-cycles (mixed-precision outer loop): r = f - A u,              */
/* e = V-cycle(A e = r, e_0 = 0), u += e, until ||r||/||r_0|| < tol. The oracle runs the inner  */
/* cycle in FP64; it is the mathematical algorithm the FP32-inner GPU solver approximates.      */
/* Pinned by dense LU (it converges to A^{-1} f) and by the multigrid iteration it must equal  */
/* (the V-cycle is linear, so one cycle on the correction equation gives the next iterate).    */
/* ------------------------------------------------------------------------------------------ */
int orc_ir_solve(int nx, int ny, int nz, int L, double cx, double cy, const double *v,
                 int nu_pre, int nu_post, int n_coarse, double rho, double tol, int max_iter,
                 const double *f, double *u, double *history, int *converged) {
    orc_mg mg;
    if (mg_setup(&mg, nx, ny, nz, L, cx, cy, v) != 0) return -1;
    mg.nu_pre = nu_pre;
    mg.nu_post = nu_post;
    mg.n_coarse = n_coarse;
    mg.rho = rho;
    size_t n = lvl_n(&mg, L);
    double *r = (double *)malloc(sizeof(double) * n);
    double *e = (double *)malloc(sizeof(double) * n);
    mg.u[L] = e;
    mg.f[L] = r;
    orc_residual(nx, ny, nz, cx, cy, v, u, f, r);
    double r0 = orc_norm2(n, r);
    int it = 0;
    *converged = 0;
    if (history) history[0] = 1.0;
    if (r0 == 0.0) {
        *converged = 1;
    } else {
        while (it < max_iter) {
            memset(e, 0, sizeof(double) * n);
            mg_vcycle(&mg, L);
#pragma omp parallel for schedule(static)
            for (size_t s = 0; s < n; ++s) u[s] += e[s];
            ++it;
            orc_residual(nx, ny, nz, cx, cy, v, u, f, r);
            double rel = orc_norm2(n, r) / r0;
            if (history) history[it] = rel;
            if (rel < tol) {
                *converged = 1;
                break;
            }
        }
    }
    free(r);
    free(e);
    mg_free(&mg);
    return it;
}
