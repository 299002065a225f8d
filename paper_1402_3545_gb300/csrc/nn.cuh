// nn.cuh -- device buffers and launchers of the learned stage (k_nn.cu), used by the C-ABI layer.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace tpmg {

enum { EPI_RELU = 0, EPI_MASK = 1 };

// Parameters (fp32 master, flat: W1 b1 W2 b2 W3 b3 W4 b4 with W[co][ci][tap]) and activations of
// one network. Activation buffers hold ncap cells (16 channels each, channels-last bf16).
struct NNBufs {
    int cin;
    int nparams;
    float* params;  // master weights
    float* grad;
    float* adam_m;
    float* adam_v;
    __nv_bfloat16 *w1, *w2f, *w2b, *w3f, *w3b, *w4;  // bf16 copies (forward / transposed layouts)
    size_t ncap;
    __nv_bfloat16 *a1, *a2, *a3;  // post-ReLU activations of layers 1..3
    __nv_bfloat16 *d1, *d2;       // gradient buffers of the hidden layers
    __nv_bfloat16* x;             // network input (cin channels)
    float* out;                   // network output
    float* d4;                    // gradient of the output
    float* tmp;                   // scratch field (residual loss)
    float* part;                  // per-block partial sums of the weight gradients
    double* dpart;                // per-block partial sums of the loss
    int* err;                     // set by a tensor-core convolution whose wait ran out of time
};

void nn_prepare_weights(const NNBufs& b, cudaStream_t s);
// out = NN(x); requires nx % 64 == 0 and ny % 2 == 0
void nn_forward(const NNBufs& b, int nx, int ny, int nz, const __nv_bfloat16* x, float* out, cudaStream_t s);
// gradient of the loss w.r.t. all parameters into grad, given d4 = dLoss/dout (forward done before)
void nn_backward(const NNBufs& b, int nx, int ny, int nz, const __nv_bfloat16* x, const float* d4, float* grad,
                 cudaStream_t s);
int nn_grad_blocks(size_t n);
void nn_mse(const float* out, const float* target, float* d4, double* partials, size_t n, int nblocks, cudaStream_t s);
// residual loss: e = x[channel 0] - q (q = A NN(x)), tmp = -2 e / n, partial sums of e^2 / n
void nn_res_loss(const __nv_bfloat16* x, int cin, const float* q, float* tmp, double* partials, size_t n, int nblocks,
                 cudaStream_t s);
void nn_adam(int n, float* theta, const float* g, float* m, float* v, float lr, int t, cudaStream_t s);
// network input from a residual r (fp64 or double-word), normalised by its root-mean-square
// (sum of squares in *sumsq); optional training target D (ea - eb) / rms with D = diag(A) of the
// level (cx, cy, per-column couplings v32)
void nn_make_input_f64(size_t n, size_t ncol, int nz, int cin, const double* r, const float* aux, const double* sumsq,
                       __nv_bfloat16* x, const double* ea, const double* eb, double cx, double cy, const float* v32,
                       float* target, cudaStream_t s);
void nn_make_input_dw(size_t n, size_t ncol, int nz, int cin, const float2* r, const float* aux, const double* sumsq,
                      __nv_bfloat16* x, cudaStream_t s);
// out = D^{-1} in
void nn_scale_dinv(size_t n, size_t ncol, int nz, double cx, double cy, const float* v32, const float* in, float* out,
                   cudaStream_t s);

}  // namespace tpmg
