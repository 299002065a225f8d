/*
 * nn_oracle.c -- ORACLE (test infrastructure only) for the learned preconditioner stage and
 * flexible CG. Plain FP64 loops. Only the test-suite, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load it; the CUDA library shares no code with it.
 *
 * Network (the learned stage of the extended method): 4 convolution layers with 3x3x3 kernels,
 * channels Cin -> 16 -> 16 -> 16 -> 1, ReLU after the first three. Fields are channel-first,
 * x fastest: element (c, k, j, i) at ((c*nz + k)*ny + j)*nx + i. Weights W[co][ci][dz][dy][dx]
 * (offsets -1..1 stored at 0..2), bias b[co]. The convolution is a cross-correlation:
 *   y[co](k,j,i) = b[co] + sum_ci sum_d W[co][ci][d] x[ci](k+dz, j+dy, i+dx)
 * with periodic wrap in i and j (the horizontal boundary of the elliptic problem) and zero padding
 * in k (beyond the Neumann ends).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static int nn_wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

static size_t fidx(int nx, int ny, int nz, int c, int k, int j, int i) {
    return (((size_t)c * nz + k) * ny + j) * (size_t)nx + i;
}

/* y = conv(x) + b, optional ReLU. x: cin channels, y: cout channels. */
void orc_conv3d_fwd(int nx, int ny, int nz, int cin, int cout, const double *W, const double *b,
                    int relu, const double *x, double *y) {
    for (int co = 0; co < cout; ++co)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double s = b ? b[co] : 0.0;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dz = -1; dz <= 1; ++dz) {
                            int kk = k + dz;
                            if (kk < 0 || kk >= nz) continue;
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    double w = W[((((size_t)co * cin + ci) * 3 + dz + 1) * 3 + dy + 1) * 3 + dx + 1];
                                    s += w * x[fidx(nx, ny, nz, ci, kk, nn_wrap(j + dy, ny), nn_wrap(i + dx, nx))];
                                }
                        }
                    if (relu && s < 0.0) s = 0.0;
                    y[fidx(nx, ny, nz, co, k, j, i)] = s;
                }
}

/* Gradients of one convolution layer given dy (gradient w.r.t. its output, after the ReLU mask
 * has been applied by the caller): dx (may be NULL), dW, db (accumulated: +=). */
void orc_conv3d_bwd(int nx, int ny, int nz, int cin, int cout, const double *W, const double *x,
                    const double *dy, double *dx, double *dW, double *db) {
    if (dx) memset(dx, 0, sizeof(double) * (size_t)cin * nx * ny * nz);
    for (int co = 0; co < cout; ++co)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double g = dy[fidx(nx, ny, nz, co, k, j, i)];
                    if (db) db[co] += g;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dz = -1; dz <= 1; ++dz) {
                            int kk = k + dz;
                            if (kk < 0 || kk >= nz) continue;
                            for (int dyy = -1; dyy <= 1; ++dyy)
                                for (int dxx = -1; dxx <= 1; ++dxx) {
                                    size_t widx = ((((size_t)co * cin + ci) * 3 + dz + 1) * 3 + dyy + 1) * 3 + dxx + 1;
                                    size_t xi = fidx(nx, ny, nz, ci, kk, nn_wrap(j + dyy, ny), nn_wrap(i + dxx, nx));
                                    dW[widx] += g * x[xi];
                                    if (dx) dx[xi] += g * W[widx];
                                }
                        }
                }
}

/* The 4-layer network. params: W1 b1 W2 b2 W3 b3 W4 b4 concatenated (cin -> 16 -> 16 -> 16 -> 1).
 * acts (optional, 3*16*n doubles) receives the post-ReLU activations of layers 1..3. */
static size_t nn_nparams(int cin) { return 16 * cin * 27 + 16 + 2 * (16 * 16 * 27 + 16) + 16 * 27 + 1; }

size_t orc_nn_nparams(int cin) { return nn_nparams(cin); }

void orc_nn_forward(int nx, int ny, int nz, int cin, const double *params, const double *x, double *out,
                    double *acts) {
    size_t n = (size_t)nx * ny * nz;
    const double *W1 = params, *b1 = W1 + 16 * cin * 27, *W2 = b1 + 16, *b2 = W2 + 16 * 16 * 27,
                 *W3 = b2 + 16, *b3 = W3 + 16 * 16 * 27, *W4 = b3 + 16, *b4 = W4 + 16 * 27;
    double *a1 = acts ? acts : (double *)malloc(sizeof(double) * 3 * 16 * n);
    double *a2 = a1 + 16 * n, *a3 = a2 + 16 * n;
    orc_conv3d_fwd(nx, ny, nz, cin, 16, W1, b1, 1, x, a1);
    orc_conv3d_fwd(nx, ny, nz, 16, 16, W2, b2, 1, a1, a2);
    orc_conv3d_fwd(nx, ny, nz, 16, 16, W3, b3, 1, a2, a3);
    orc_conv3d_fwd(nx, ny, nz, 16, 1, W4, b4, 0, a3, out);
    if (!acts) free(a1);
}

/* Backpropagation through the four layers: given the forward activations (acts, as filled by
 * orc_nn_forward) and d4 = dLoss/dout, the gradient w.r.t. all parameters (grad, overwritten). */
static void nn_backward(int nx, int ny, int nz, int cin, const double *params, const double *x,
                        const double *acts, const double *d4, double *grad) {
    size_t n = (size_t)nx * ny * nz;
    const double *W2 = params + 16 * cin * 27 + 16, *W3 = W2 + 16 * 16 * 27 + 16,
                 *W4 = W3 + 16 * 16 * 27 + 16;
    double *gW1 = grad, *gb1 = gW1 + 16 * cin * 27, *gW2 = gb1 + 16, *gb2 = gW2 + 16 * 16 * 27,
           *gW3 = gb2 + 16, *gb3 = gW3 + 16 * 16 * 27, *gW4 = gb3 + 16, *gb4 = gW4 + 16 * 27;
    const double *W1 = params;
    memset(grad, 0, sizeof(double) * nn_nparams(cin));
    const double *a1 = acts, *a2 = a1 + 16 * n, *a3 = a2 + 16 * n;
    double *d3 = (double *)malloc(sizeof(double) * 16 * n);
    double *d2 = (double *)malloc(sizeof(double) * 16 * n);
    orc_conv3d_bwd(nx, ny, nz, 16, 1, W4, a3, d4, d3, gW4, gb4);
    for (size_t p = 0; p < 16 * n; ++p) if (a3[p] <= 0.0) d3[p] = 0.0;  /* ReLU of layer 3 */
    orc_conv3d_bwd(nx, ny, nz, 16, 16, W3, a2, d3, d2, gW3, gb3);
    for (size_t p = 0; p < 16 * n; ++p) if (a2[p] <= 0.0) d2[p] = 0.0;
    orc_conv3d_bwd(nx, ny, nz, 16, 16, W2, a1, d2, d3, gW2, gb2);
    for (size_t p = 0; p < 16 * n; ++p) if (a1[p] <= 0.0) d3[p] = 0.0;
    orc_conv3d_bwd(nx, ny, nz, cin, 16, W1, x, d3, NULL, gW1, gb1);
    free(d3);
    free(d2);
}

/* Loss = mean over cells of (out - target)^2 and its gradient w.r.t. all parameters (grad, nparams
 * doubles, overwritten). Returns the loss. */
double orc_nn_loss_grad(int nx, int ny, int nz, int cin, const double *params, const double *x,
                        const double *target, double *grad) {
    size_t n = (size_t)nx * ny * nz;
    double *acts = (double *)malloc(sizeof(double) * 3 * 16 * n);
    double *out = (double *)malloc(sizeof(double) * n);
    double *d4 = (double *)malloc(sizeof(double) * n);
    orc_nn_forward(nx, ny, nz, cin, params, x, out, acts);
    double loss = 0.0;
    for (size_t p = 0; p < n; ++p) {
        double e = out[p] - target[p];
        loss += e * e;
        d4[p] = 2.0 * e / (double)n;
    }
    loss /= (double)n;
    nn_backward(nx, ny, nz, cin, params, x, acts, d4, grad);
    free(acts);
    free(out);
    free(d4);
    return loss;
}

void orc_apply_A(int nx, int ny, int nz, double cx, double cy, const double *v, const double *x, double *y);

/* D = diag(A) per cell: 1 + 2cx + 2cy plus v for each vertical neighbour inside the column. The
 * network's output is measured in units of D^{-1} (a Jacobi step): the learned correction is
 * s D^{-1} NN(r/s), so NN's targets are O(1) whatever the mesh width and lambda^2. */
static void diag_inv(int nx, int ny, int nz, double cx, double cy, const double *v, double *dinv) {
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double vij = v[(size_t)j * nx + i];
                double d = 1.0 + 2.0 * cx + 2.0 * cy + (k > 0 ? vij : 0.0) + (k < nz - 1 ? vij : 0.0);
                dinv[((size_t)k * ny + j) * nx + i] = 1.0 / d;
            }
}

void orc_diag_inv(int nx, int ny, int nz, double cx, double cy, const double *v, double *dinv) {
    diag_inv(nx, ny, nz, cx, cy, v, dinv);
}

/* Residual loss: with r = x[0] (the normalised residual channel), y = NN(x) and D = diag(A),
 *   loss = mean over cells of (r - A D^{-1} y)^2,
 * the mean square of the residual left after the correction D^{-1} y; A is the operator with
 * couplings cx, cy and v (per column). A is symmetric, so dLoss/dy = -2 D^{-1} A (r - A D^{-1} y) / n.
 * Returns the loss; grad (nparams doubles) is overwritten. */
double orc_nn_loss_grad_residual(int nx, int ny, int nz, int cin, double cx, double cy, const double *v,
                                 const double *params, const double *x, double *grad) {
    size_t n = (size_t)nx * ny * nz;
    double *acts = (double *)malloc(sizeof(double) * 3 * 16 * n);
    double *out = (double *)malloc(sizeof(double) * n);
    double *e = (double *)malloc(sizeof(double) * n);
    double *d4 = (double *)malloc(sizeof(double) * n);
    double *dinv = (double *)malloc(sizeof(double) * n);
    diag_inv(nx, ny, nz, cx, cy, v, dinv);
    orc_nn_forward(nx, ny, nz, cin, params, x, out, acts);
    for (size_t p = 0; p < n; ++p) out[p] *= dinv[p];
    orc_apply_A(nx, ny, nz, cx, cy, v, out, e);
    double loss = 0.0;
    for (size_t p = 0; p < n; ++p) {
        e[p] = x[p] - e[p];
        loss += e[p] * e[p];
    }
    loss /= (double)n;
    orc_apply_A(nx, ny, nz, cx, cy, v, e, d4);
    for (size_t p = 0; p < n; ++p) d4[p] *= -2.0 * dinv[p] / (double)n;
    nn_backward(nx, ny, nz, cin, params, x, acts, d4, grad);
    free(acts);
    free(out);
    free(e);
    free(d4);
    free(dinv);
    return loss;
}

/* One Adam step (Kingma & Ba, 2015) on n parameters: m, v moments, t = step number (1-based). */
void orc_adam_step(size_t n, double *theta, const double *g, double *m, double *v, int t, double lr,
                   double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (size_t p = 0; p < n; ++p) {
        m[p] = beta1 * m[p] + (1.0 - beta1) * g[p];
        v[p] = beta2 * v[p] + (1.0 - beta2) * g[p] * g[p];
        double mh = m[p] / c1, vh = v[p] / c2;
        theta[p] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Flexible CG with truncation m = 1 (Notay, SIAM J. Sci. Comput. 22, 2000): the search direction */
/* is z_i A-orthogonalised against the previous direction only, so a preconditioner that changes  */
/* from one application to the next is allowed.                                                   */
/* ------------------------------------------------------------------------------------------ */
void orc_line_solve(int nx, int ny, int nz, double cx, double cy, const double *v, const double *b, double *x);
int orc_vcycle(int nx, int ny, int nz, int L, double cx, double cy, const double *v, int nu_pre, int nu_post,
               int n_coarse, double rho, const double *f, double *u);
double orc_dot(size_t n, const double *a, const double *b);

typedef struct {
    int mode;           /* 0: z = M^{-1} r (line solve); 1: z = V-cycle(r); 2: V-cycle + learned stage */
    int L, nu_pre, nu_post, n_coarse;
    double rho;
    int cin;
    const double *params; /* network parameters (mode 2) */
    const double *aux;    /* second input channel (n values) or NULL */
    int nn_used, nn_rejected;
} orc_prec;

/* z = B(r). Mode 2: z1 = V-cycle(r), r1 = r - A z1, s = rms(r1) = ||r1|| / sqrt(n),
 * z = z1 + s D^{-1} NN(r1 / s) with D = diag(A) (the network sees a residual of unit mean square
 * and answers in units of a Jacobi step, whatever the grid size and coefficients); the learned
 * correction is dropped (z = z1) when ||r - A z|| >= ||r1|| or the result is not finite. */
static void fcg_precondition(int nx, int ny, int nz, double cx, double cy, const double *v, orc_prec *P,
                             const double *r, double *z, double *cand) {
    size_t n = (size_t)nx * ny * nz;
    if (P->mode == 0) {
        orc_line_solve(nx, ny, nz, cx, cy, v, r, z);
        return;
    }
    memset(z, 0, sizeof(double) * n);
    orc_vcycle(nx, ny, nz, P->L, cx, cy, v, P->nu_pre, P->nu_post, P->n_coarse, P->rho, r, z);
    if (P->mode != 2) return;
    double *Az = (double *)malloc(sizeof(double) * n);
    double *r1 = (double *)malloc(sizeof(double) * n);
    double *x = (double *)malloc(sizeof(double) * n * (size_t)P->cin);
    double *c = (double *)malloc(sizeof(double) * n);
    double *dinv = (double *)malloc(sizeof(double) * n);
    diag_inv(nx, ny, nz, cx, cy, v, dinv);
    orc_apply_A(nx, ny, nz, cx, cy, v, z, Az);
    for (size_t p = 0; p < n; ++p) r1[p] = r[p] - Az[p];
    double nr1 = sqrt(orc_dot(n, r1, r1));
    int accept = 0;
    if (nr1 > 0.0 && isfinite(nr1)) {
        double rms = nr1 / sqrt((double)n);
        for (size_t p = 0; p < n; ++p) x[p] = r1[p] / rms;
        if (P->cin > 1) memcpy(x + n, P->aux, sizeof(double) * n);
        orc_nn_forward(nx, ny, nz, P->cin, P->params, x, c, NULL);
        for (size_t p = 0; p < n; ++p) c[p] = z[p] + rms * dinv[p] * c[p];
        orc_apply_A(nx, ny, nz, cx, cy, v, c, Az);
        double s = 0.0;
        for (size_t p = 0; p < n; ++p) {
            double e = r[p] - Az[p];
            s += e * e;
        }
        s = sqrt(s);
        accept = isfinite(s) && s < nr1;
        if (cand) memcpy(cand, c, sizeof(double) * n);
        if (accept) memcpy(z, c, sizeof(double) * n);
    }
    P->nn_used += accept;
    P->nn_rejected += !accept;
    free(Az);
    free(r1);
    free(x);
    free(c);
    free(dinv);
}

/* One application of the preconditioner (test access): z = B(r); cand (may be NULL) receives the
 * learned candidate z1 + s D^{-1} NN(r1/s) of mode 2 whether or not it was kept. */
void orc_fcg_precondition(int nx, int ny, int nz, double cx, double cy, const double *v, orc_prec *P,
                          const double *r, double *z, double *cand) {
    fcg_precondition(nx, ny, nz, cx, cy, v, P, r, z, cand);
}

int orc_fcg_solve(int nx, int ny, int nz, double cx, double cy, const double *v, orc_prec *P, double tol,
                  int max_iter, const double *f, double *u, double *history, int *converged) {
    size_t n = (size_t)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
    orc_apply_A(nx, ny, nz, cx, cy, v, u, q);
    for (size_t s = 0; s < n; ++s) r[s] = f[s] - q[s];
    double r0 = sqrt(orc_dot(n, r, r));
    int it = 0;
    *converged = 0;
    if (history) history[0] = 1.0;
    if (r0 == 0.0) {
        *converged = 1;
    } else {
        fcg_precondition(nx, ny, nz, cx, cy, v, P, r, z, NULL);
        memcpy(p, z, sizeof(double) * n);
        orc_apply_A(nx, ny, nz, cx, cy, v, p, q);
        while (it < max_iter) {
            double pq = orc_dot(n, p, q);
            double alpha = orc_dot(n, p, r) / pq;
            for (size_t s = 0; s < n; ++s) {
                u[s] += alpha * p[s];
                r[s] -= alpha * q[s];
            }
            ++it;
            double rel = sqrt(orc_dot(n, r, r)) / r0;
            if (history) history[it] = rel;
            if (rel < tol) {
                *converged = 1;
                break;
            }
            if (it == max_iter) break;
            fcg_precondition(nx, ny, nz, cx, cy, v, P, r, z, NULL);
            double beta = orc_dot(n, z, q) / pq;
            for (size_t s = 0; s < n; ++s) p[s] = z[s] - beta * p[s];
            orc_apply_A(nx, ny, nz, cx, cy, v, p, q);
        }
    }
    free(r);
    free(z);
    free(p);
    free(q);
    return it;
}
