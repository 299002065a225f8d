// fcg.cuh -- device scalars and launchers of flexible CG (k_fcg.cu), used by the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "kernels.cuh"

namespace tpmg {

static constexpr int FCG_MAX_BLOCKS = 152 * 8;

struct FcgScalars {
    double r0, rel, tol, alpha, beta, pq, r1sq;
    int iters, max_iter, done, converged, nonfinite, keep, accepted, rejected;
};
enum { FCG_INIT_NORM = 0, FCG_ALPHA = 1, FCG_CHECK = 2, FCG_BETA = 3, FCG_R1 = 4, FCG_DECIDE = 5 };

int fcg_apply(const Lv<PolDW>& L, const float2* p, const float2* r, float2* q, double* partials, cudaStream_t s);
int fcg_update(size_t n, const FcgScalars* sc, float2* u, const float2* p, float2* r, const float2* q, double* partials,
               cudaStream_t s);
int fcg_dot(size_t n, const float2* a, const float2* b, double* partials, cudaStream_t s);
void fcg_direction(size_t n, const FcgScalars* sc, const float2* z, float2* p, cudaStream_t s);
// c = z1 + rms(r1) D^{-1} y (D = diag(A) from cx, cy and the per-column couplings v32)
void fcg_learned(size_t n, size_t ncol, int nz, double cx, double cy, const float* v32, const FcgScalars* sc,
                 const float2* z1, const float* y, float2* c, cudaStream_t s);
void fcg_select(size_t n, const FcgScalars* sc, const float2* c, const float2* z1, float2* z, cudaStream_t s);
void fcg_dw_from_f32(size_t n, const float* a, float2* b, cudaStream_t s);
void fcg_f32_from_dw(size_t n, const float2* a, float* b, cudaStream_t s);
void fcg_scalar(int mode, const double* partials, int nparts, FcgScalars* sc, double* history, cudaStream_t s);
void fcg_init(FcgScalars* sc, double tol, int max_iter, cudaStream_t s);

}  // namespace tpmg
