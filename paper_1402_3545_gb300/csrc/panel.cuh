// panel.cuh -- the cubed-sphere panel operator's level view and launchers (k_panel.cu), used by the
// C-ABI layer. Native FP64, and FP32 for the inner V-cycles of the mixed-precision solve.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace tpmg {

// One multigrid level of the panel operator (Eq. (14)) as the kernels see it, in value type T
// (double or float): nx x ny columns of nz cells, x fastest. Geometry: area[j*nx + i] = |T|;
// ax[j*(nx+1) + i] the coefficient alpha of the x-face between cells i-1 and i of row j (i = 0 and nx:
// the panel boundary); ay[j*nx + i] that of the y-face between rows j-1 and j (j = 0..ny). Radial
// vectors (nz each, shared by the levels): E = a - b - c, B = -b, C = -c with B[0] = C[nz-1] = 0 and
// C[k] = B[k+1]. Thomas factors per cell: inv = 1/m_k, fl = |T| B_k / m_k, fw = |T| C_k / m_k.
template <class T>
struct PanelLvT {
    int nx, ny, nz;
    const T* area;
    const T* ax;
    const T* ay;
    const T* E;
    const T* B;
    const T* C;
    const T* inv;
    const T* fl;
    const T* fw;
};
typedef PanelLvT<double> PanelLv;

enum { PANEL_SMOOTH = 0, PANEL_RESIDUAL = 1, PANEL_LINESOLVE = 2, PANEL_APPLY = 3 };

void launch_panel_factors(const PanelLv& L, double* inv, double* fl, double* fw, cudaStream_t s);
// mode PANEL_*: Smooth (coef = rho) and Residual write partial sums of ||f - A u||^2 when partials is
// non-null; the line solve takes its right-hand side in u and scales by coef. Returns the number of
// thread blocks (= partial sums written).
template <class T>
int launch_panel_sweep(int mode, const PanelLvT<T>& L, double coef, const T* u, const T* f, T* out, double* partials,
                       const int* done, cudaStream_t s);
// r = f - A u in FP64 stored as FP32 (the mixed solve's outer residual), partial sums of ||r||^2
int launch_panel_residual_to_f32(const PanelLv& L, const double* u, const double* f, float* r, double* partials,
                                 const int* done, cudaStream_t s);
template <class T>
void launch_panel_restrict_smooth(const PanelLvT<T>& Lc, double rho, const T* rf, T* fc, T* uc, const int* done,
                                  cudaStream_t s);
template <class T>
void launch_panel_prolongate(int nxc, int nyc, int nz, const T* uc, T* uf, const int* done, cudaStream_t s);
// fused CG kernels on the finest level (Sec. 3.1): SpMV writes one partial sum of <p, q> per block,
// Tridiag those of <r, r> and then of <r, z> (panel_blocks(nx, ny) each)
struct Scalars;
int panel_blocks(int nx, int ny);
void launch_panel_cg_spmv(const PanelLv& L, const Scalars* sc, double* u, double* p, const double* z, double* q,
                          double* partials, cudaStream_t s);
void launch_panel_cg_tridiag(const PanelLv& L, const Scalars* sc, double* r, const double* q, double* z,
                             double* partials, cudaStream_t s);

}  // namespace tpmg
