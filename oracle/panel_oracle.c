/*
 * panel_oracle.c -- ORACLE (test infrastructure) of the paper's own operator: the model equation
 * Eq. (1) discretised by cell-centred finite volumes on one panel of a gnomonic cubed-sphere grid
 * with homogeneous Dirichlet conditions on the panel's horizontal boundary (Sec. 2.1.1), in the
 * factorised form of Eq. (14) "LocalMatrixStencil":
 *
 *   A_{T,T'} = alpha_{TT'} diag(d),
 *   A_T      = |T| diag(a) - alpha_T diag(d) + |T| tridiag(-(b + c), b, c),   alpha_T = sum of the
 *              alpha_{TT'} over the four faces of T (d = 1: the tangential term needs no radial
 *              weight once integrated over the cell),
 *
 * so that, for cell T = (i, j) and level k,
 *   (A u)_{T,k} = (|T| (a_k - b_k - c_k) - alpha_T) u_{T,k} + sum_{T'} alpha_{TT'} u_{T',k}
 *                 + |T| (b_k u_{T,k-1} + c_k u_{T,k+1}),
 * with b_0 = 0 and c_{nz-1} = 0 (Neumann top and bottom) and a neighbour across the panel boundary
 * holding the value 0 (its face coefficient still counts in alpha_T). Only the geometry's numbers
 * enter here; oracle/panel.py computes them from the panel and the radial grid.
 *
 * Only the test-suite, __graft_entry__.smoke() and bench.py's CPU legs may load this code; it shares
 * nothing with the CUDA library. Loops over cells and columns may run on several host threads
 * (OpenMP, as in tpmg_oracle.c); the norms and dot products run in index order on one thread.
 *
 * Arrays: fields nz*ny*nx doubles, x fastest (as in tpmg_oracle.c); area[j*nx + i] = |T|;
 * ax[j*(nx+1) + i] = alpha of the x-face between cells i-1 and i of row j (i = 0 and i = nx are the
 * boundary faces); ay[j*nx + i] = alpha of the y-face between rows j-1 and j of column i
 * (j = 0..ny); a, b, c: nz entries each.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PO_MAX_LEVELS 16

static size_t pidx(int nx, int ny, int i, int j, int k) {
    return ((size_t)k * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i;
}

typedef struct {
    int nx, ny, nz;
    const double *area, *ax, *ay, *a, *b, *c;
} po_level;

static double alpha_T(const po_level *g, int i, int j) {
    return g->ax[(size_t)j * (g->nx + 1) + i] + g->ax[(size_t)j * (g->nx + 1) + i + 1] +
           g->ay[(size_t)j * g->nx + i] + g->ay[(size_t)(j + 1) * g->nx + i];
}

/* y = A x (Eq. (14)). */
static void po_apply(const po_level *g, const double *x, double *y) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double T = g->area[(size_t)j * nx + i];
                const double aW = g->ax[(size_t)j * (nx + 1) + i], aE = g->ax[(size_t)j * (nx + 1) + i + 1];
                const double aS = g->ay[(size_t)j * nx + i], aN = g->ay[(size_t)(j + 1) * nx + i];
                double s = (T * (g->a[k] - g->b[k] - g->c[k]) - (aW + aE + aS + aN)) * x[pidx(nx, ny, i, j, k)];
                if (i > 0) s += aW * x[pidx(nx, ny, i - 1, j, k)];
                if (i < nx - 1) s += aE * x[pidx(nx, ny, i + 1, j, k)];
                if (j > 0) s += aS * x[pidx(nx, ny, i, j - 1, k)];
                if (j < ny - 1) s += aN * x[pidx(nx, ny, i, j + 1, k)];
                if (k > 0) s += T * g->b[k] * x[pidx(nx, ny, i, j, k - 1)];
                if (k < nz - 1) s += T * g->c[k] * x[pidx(nx, ny, i, j, k + 1)];
                y[pidx(nx, ny, i, j, k)] = s;
            }
}

/* x = M^{-1} r with M the column blocks A_T (vertical line relaxation, Sec. 2.2): Thomas per
 * column, forward elimination k = 0..nz-1, then back substitution. */
static void po_line_solve(const po_level *g, const double *r, double *x) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel
    {
    double *cp = (double *)malloc(sizeof(double) * (size_t)nz);
    double *dp = (double *)malloc(sizeof(double) * (size_t)nz);
#pragma omp for collapse(2) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double T = g->area[(size_t)j * nx + i], aT = alpha_T(g, i, j);
            for (int k = 0; k < nz; ++k) {
                const double diag = T * (g->a[k] - g->b[k] - g->c[k]) - aT;
                const double lower = (k > 0) ? T * g->b[k] : 0.0, upper = (k < nz - 1) ? T * g->c[k] : 0.0;
                const double rhs = r[pidx(nx, ny, i, j, k)];
                if (k == 0) {
                    cp[k] = upper / diag;
                    dp[k] = rhs / diag;
                } else {
                    const double den = diag - lower * cp[k - 1];
                    cp[k] = upper / den;
                    dp[k] = (rhs - lower * dp[k - 1]) / den;
                }
            }
            x[pidx(nx, ny, i, j, nz - 1)] = dp[nz - 1];
            for (int k = nz - 2; k >= 0; --k)
                x[pidx(nx, ny, i, j, k)] = dp[k] - cp[k] * x[pidx(nx, ny, i, j, k + 1)];
        }
    free(cp);
    free(dp);
    }
}

static po_level level_of(int nx, int ny, int nz, const double *area, const double *ax, const double *ay,
                         const double *a, const double *b, const double *c) {
    po_level g = {nx, ny, nz, area, ax, ay, a, b, c};
    return g;
}

void orc_panel_apply_A(int nx, int ny, int nz, const double *area, const double *ax, const double *ay,
                       const double *a, const double *b, const double *c, const double *x, double *y) {
    po_level g = level_of(nx, ny, nz, area, ax, ay, a, b, c);
    po_apply(&g, x, y);
}

void orc_panel_line_solve(int nx, int ny, int nz, const double *area, const double *ax, const double *ay,
                          const double *a, const double *b, const double *c, const double *r, double *x) {
    po_level g = level_of(nx, ny, nz, area, ax, ay, a, b, c);
    po_line_solve(&g, r, x);
}

/* f_c = R r_f: the coarse cell's right-hand side is the sum of its 2 x 2 children's residuals. The
 * equations are integrated over the cells (Eq. (14) carries |T|), so this is the residual integrated
 * over the coarse cell: the paper's cell average of the residual density times the coarse cell. */
static void po_restrict(int nxf, int nyf, int nz, const double *rf, double *fc) {
    const int nxc = nxf / 2, nyc = nyf / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int J = 0; J < nyc; ++J)
            for (int I = 0; I < nxc; ++I)
                fc[pidx(nxc, nyc, I, J, k)] =
                    rf[pidx(nxf, nyf, 2 * I, 2 * J, k)] + rf[pidx(nxf, nyf, 2 * I + 1, 2 * J, k)] +
                    rf[pidx(nxf, nyf, 2 * I, 2 * J + 1, k)] + rf[pidx(nxf, nyf, 2 * I + 1, 2 * J + 1, k)];
}

/* u_f += P u_c: bilinear interpolation in the logical (i, j) grid, weights 3/4 and 1/4 per
 * direction as on the flat box (Sec. 2.2); a coarse neighbour beyond the panel boundary holds 0
 * (the homogeneous Dirichlet ghost of the operator). */
static void po_prolongate_add(int nxc, int nyc, int nz, const double *uc, double *uf) {
    const int nxf = 2 * nxc, nyf = 2 * nyc;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nyf; ++j)
            for (int i = 0; i < nxf; ++i) {
                const int I = i / 2, J = j / 2;
                const int I2 = (i % 2 == 0) ? I - 1 : I + 1, J2 = (j % 2 == 0) ? J - 1 : J + 1;
                const int in2 = I2 >= 0 && I2 < nxc, jn2 = J2 >= 0 && J2 < nyc;
                double val = 0.75 * 0.75 * uc[pidx(nxc, nyc, I, J, k)];
                if (in2) val += 0.25 * 0.75 * uc[pidx(nxc, nyc, I2, J, k)];
                if (jn2) val += 0.75 * 0.25 * uc[pidx(nxc, nyc, I, J2, k)];
                if (in2 && jn2) val += 0.25 * 0.25 * uc[pidx(nxc, nyc, I2, J2, k)];
                uf[pidx(nxf, nyf, i, j, k)] += val;
            }
}

void orc_panel_restrict(int nxf, int nyf, int nz, const double *rf, double *fc) { po_restrict(nxf, nyf, nz, rf, fc); }
void orc_panel_prolongate_add(int nxc, int nyc, int nz, const double *uc, double *uf) {
    po_prolongate_add(nxc, nyc, nz, uc, uf);
}

/* ---------------------------------------------------------------- multigrid (Algorithm 1)      */
typedef struct {
    int L, nu_pre, nu_post, n_coarse;
    double rho;
    po_level g[PO_MAX_LEVELS + 1];
    double *u[PO_MAX_LEVELS + 1], *f[PO_MAX_LEVELS + 1], *r[PO_MAX_LEVELS + 1], *t[PO_MAX_LEVELS + 1];
} po_mg;

static size_t po_n(const po_level *g) { return (size_t)g->nx * g->ny * g->nz; }

/* u <- u + rho M^{-1} (f - A u) on level l (Eq. (11)). */
static void po_smooth(po_mg *m, int l) {
    const po_level *g = &m->g[l];
    const size_t n = po_n(g);
    po_apply(g, m->u[l], m->r[l]);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) m->r[l][p] = m->f[l][p] - m->r[l][p];
    po_line_solve(g, m->r[l], m->t[l]);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) m->u[l][p] += m->rho * m->t[l][p];
}

static void po_residual(po_mg *m, int l) {
    const size_t n = po_n(&m->g[l]);
    po_apply(&m->g[l], m->u[l], m->r[l]);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) m->r[l][p] = m->f[l][p] - m->r[l][p];
}

/* restriction of level l+1's residual, then the first smoothing step from zero: u = rho M^{-1} f */
static void po_restrict_smooth(po_mg *m, int l) {
    const size_t n = po_n(&m->g[l]);
    po_restrict(m->g[l + 1].nx, m->g[l + 1].ny, m->g[l].nz, m->r[l + 1], m->f[l]);
    po_line_solve(&m->g[l], m->f[l], m->u[l]);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < n; ++p) m->u[l][p] *= m->rho;
}

static void po_vcycle(po_mg *m, int l) {
    const int L = m->L;
    if (L == 1) {
        for (int s = 0; s < m->n_coarse; ++s) po_smooth(m, 1);
        return;
    }
    if (l == 1) {
        po_restrict_smooth(m, 1);
        for (int s = 1; s < m->n_coarse; ++s) po_smooth(m, 1);
        return;
    }
    if (l == L) {
        for (int s = 0; s < m->nu_pre; ++s) po_smooth(m, l);
    } else {
        po_restrict_smooth(m, l);
        for (int s = 1; s < m->nu_pre; ++s) po_smooth(m, l);
    }
    po_residual(m, l);
    po_vcycle(m, l - 1);
    po_prolongate_add(m->g[l - 1].nx, m->g[l - 1].ny, m->g[l].nz, m->u[l - 1], m->u[l]);
    for (int s = 0; s < m->nu_post; ++s) po_smooth(m, l);
}

static double po_norm(size_t n, const double *x) {
    double s = 0.0;
    for (size_t p = 0; p < n; ++p) s += x[p] * x[p];
    return sqrt(s);
}

/* Multigrid solve: V-cycles from u until ||f - A u|| / ||f - A u_0|| < tol (Eq. (10)). Level l
 * (1 = coarsest, L = finest) has nx[l] x ny[l] columns and the geometry area[l], ax[l], ay[l]
 * (arrays of L+1 pointers, index 0 unused); a, b, c are shared by the levels. Returns the cycles. */
int orc_panel_mg_solve(int L, const int *nx, const int *ny, int nz, const double *const *area,
                       const double *const *ax, const double *const *ay, const double *a, const double *b,
                       const double *c, int nu_pre, int nu_post, int n_coarse, double rho, double tol,
                       int max_iter, const double *f, double *u, double *history, int *converged) {
    if (L < 1 || L > PO_MAX_LEVELS) return -1;
    po_mg m;
    memset(&m, 0, sizeof(m));
    m.L = L;
    m.nu_pre = nu_pre;
    m.nu_post = nu_post;
    m.n_coarse = n_coarse;
    m.rho = rho;
    for (int l = 1; l <= L; ++l) {
        m.g[l] = level_of(nx[l], ny[l], nz, area[l], ax[l], ay[l], a, b, c);
        const size_t n = po_n(&m.g[l]);
        m.r[l] = (double *)calloc(n, sizeof(double));
        m.t[l] = (double *)calloc(n, sizeof(double));
        if (l < L) {
            m.u[l] = (double *)calloc(n, sizeof(double));
            m.f[l] = (double *)calloc(n, sizeof(double));
        }
    }
    m.u[L] = u;
    m.f[L] = (double *)f;
    const size_t n = po_n(&m.g[L]);
    double *r = (double *)malloc(sizeof(double) * n);
    po_apply(&m.g[L], u, r);
    for (size_t p = 0; p < n; ++p) r[p] = f[p] - r[p];
    const double r0 = po_norm(n, r);
    int it = 0;
    *converged = 0;
    if (history) history[0] = 1.0;
    if (r0 == 0.0) {
        *converged = 1;
    } else {
        while (it < max_iter) {
            po_vcycle(&m, L);
            ++it;
            po_apply(&m.g[L], u, r);
            for (size_t p = 0; p < n; ++p) r[p] = f[p] - r[p];
            const double rel = po_norm(n, r) / r0;
            if (history) history[it] = rel;
            if (rel < tol) {
                *converged = 1;
                break;
            }
        }
    }
    free(r);
    for (int l = 1; l <= L; ++l) {
        free(m.r[l]);
        free(m.t[l]);
        if (l < L) {
            free(m.u[l]);
            free(m.f[l]);
        }
    }
    return it;
}

/* Line-preconditioned CG (Sec. 2.2), textbook form, on the panel operator. */
int orc_panel_cg_solve(int nx, int ny, int nz, const double *area, const double *ax, const double *ay,
                       const double *a, const double *b, const double *c, double tol, int max_iter, const double *f,
                       double *u, double *history, int *converged) {
    po_level g = level_of(nx, ny, nz, area, ax, ay, a, b, c);
    const size_t n = po_n(&g);
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
    po_apply(&g, u, r);
    for (size_t s = 0; s < n; ++s) r[s] = f[s] - r[s];
    const double r0 = po_norm(n, r);
    po_line_solve(&g, r, z);
    memcpy(p, z, sizeof(double) * n);
    double rz = 0.0;
    for (size_t s = 0; s < n; ++s) rz += r[s] * z[s];
    int it = 0;
    *converged = 0;
    if (history) history[0] = 1.0;
    if (r0 == 0.0) {
        *converged = 1;
    } else {
        while (it < max_iter) {
            po_apply(&g, p, q);
            double pq = 0.0;
            for (size_t s = 0; s < n; ++s) pq += p[s] * q[s];
            const double alpha = rz / pq;
            for (size_t s = 0; s < n; ++s) {
                u[s] += alpha * p[s];
                r[s] -= alpha * q[s];
            }
            ++it;
            const double rel = po_norm(n, r) / r0;
            if (history) history[it] = rel;
            if (rel < tol) {
                *converged = 1;
                break;
            }
            po_line_solve(&g, r, z);
            double rz_new = 0.0;
            for (size_t s = 0; s < n; ++s) rz_new += r[s] * z[s];
            const double beta = rz_new / rz;
            rz = rz_new;
            for (size_t s = 0; s < n; ++s) p[s] = z[s] + beta * p[s];
        }
    }
    free(r);
    free(z);
    free(p);
    free(q);
    return it;
}
