// k_nn.cu -- the learned preconditioner stage: a 4-layer 3-D convolutional network (cin -> 16 ->
// 16 -> 16 -> 1, 3x3x3 kernels, ReLU after the first three layers, periodic padding in x and y,
// zero padding in z), its training kernels and Adam.
//
// Activations are channels-last BF16 (16 channels = 32 bytes per cell, cell index (k*ny + j)*nx + i);
// weights are BF16 copies of FP32 master parameters; all sums accumulate in FP32.
// The 16 -> 16 layers are implicit GEMMs on the tensor cores: a block computes a tile of 64 x 2
// cells of one plane; each warp owns 16 consecutive cells (the M = 16 rows of mma.m16n8k16), the
// K dimension runs over the 27 taps x 16 input channels, N = 16 output channels (two n8 tiles).
// The input tile with its one-cell halo (66 x 4 x 3 cells) and the 27 x 16 x 16 weights are staged
// in shared memory and fed to the MMAs with ldmatrix. The same kernel computes the data gradient
// of the backward pass with flipped, transposed weights and a ReLU-mask epilogue. The weight
// gradients of the 16 -> 16 layers are tensor-core GEMMs too (cells are the K dimension).
#include <cuda_bf16.h>

#include <type_traits>

#include "kernels.cuh"
#include "nn.cuh"

namespace tpmg {

__device__ __forceinline__ int nwrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldm_x4(unsigned addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldm_x4_t(unsigned addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
// D = A B + D, A 16x16 (row), B 16x8 (col), bf16 inputs, f32 accumulate
__device__ __forceinline__ void mma16816(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

static constexpr int TXC = 64, TYC = 2;              // cells per block tile (x, y)
static constexpr int HX = TXC + 2, HY = TYC + 2;     // halo tile
static constexpr int HCELLS = HX * HY * 3;           // 3 planes
static constexpr int HALO_BYTES = HCELLS * 32;       // 16 bf16 per cell
static constexpr int W_BYTES = 27 * 16 * 16 * 2;

// Loads the 66 x 4 x 3 halo tile of a 16-channel activation around plane k (zero beyond z ends).
__device__ void load_halo16(const __nv_bfloat16* __restrict__ act, int nx, int ny, int nz, int x0, int y0, int k,
                            unsigned char* H) {
    const int tid = threadIdx.x;
    for (int q = tid; q < HCELLS * 2; q += blockDim.x) {
        const int v = q >> 1, half = q & 1;
        const int xx = v % HX, yy = (v / HX) % HY, dz = v / (HX * HY);
        const int kk = k - 1 + dz;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (kk >= 0 && kk < nz) {
            const int i = nwrap(x0 - 1 + xx, nx), j = nwrap(y0 - 1 + yy, ny);
            const size_t p = ((size_t)kk * ny + j) * nx + i;
            val = __ldg(reinterpret_cast<const uint4*>(act + p * 16) + half);
        }
        reinterpret_cast<uint4*>(H)[q] = val;
    }
}

// ---------------------------------------------------------------- 16 -> 16 convolution (tensor cores)
// EPI_RELU: out = bf16(relu(acc + bias)); EPI_MASK: out = bf16(mask > 0 ? acc : 0) (data gradient)
template <int EPI>
__global__ void __launch_bounds__(256) k_conv16(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wt,
                                                const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask,
                                                __nv_bfloat16* __restrict__ out, int nx, int ny, int nz) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* H = smem;
    unsigned char* Ws = smem + HALO_BYTES;
    const int x0 = blockIdx.x * TXC, y0 = blockIdx.y * TYC, k = blockIdx.z;
    for (int q = threadIdx.x; q < W_BYTES / 16; q += blockDim.x)
        reinterpret_cast<uint4*>(Ws)[q] = __ldg(reinterpret_cast<const uint4*>(Wt) + q);
    load_halo16(in, nx, ny, nz, x0, y0, k, H);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int yw = warp >> 2, xw = (warp & 3) * 16;
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    const int ar = lane & 15, acol = (lane >> 4) * 8;                       // A: row, column block
    const int bco = ((lane >> 4) << 3) + (lane & 7), bci = ((lane >> 3) & 1) * 8;  // B: out, in channel
#pragma unroll 1
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll 1
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int tap = (dz * 3 + dy) * 3 + dx;
                const int cell = (dz * HY + yw + dy) * HX + xw + ar + dx;
                uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
                ldm_x4(saddr(H + cell * 32 + acol * 2), a0, a1, a2, a3);
                ldm_x4(saddr(Ws + ((tap * 16 + bco) * 16 + bci) * 2), b0, b1, b2, b3);
                mma16816(c0, a0, a1, a2, a3, b0, b1);
                mma16816(c1, a0, a1, a2, a3, b2, b3);
            }
    // epilogue: lane holds cells g, g+8 and channel pairs 2t, 2t+1 (+8 for the second n tile)
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    const int y = y0 + yw;
    if (y >= ny) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int x = x0 + xw + g + 8 * h;
        if (x >= nx) continue;
        const size_t p = ((size_t)k * ny + y) * nx + x;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const float* c = nt ? c1 : c0;
            const int co = t2 + 8 * nt;
            float v0 = c[2 * h], v1 = c[2 * h + 1];
            if (EPI == EPI_RELU) {
                v0 = fmaxf(v0 + __ldg(bias + co), 0.f);
                v1 = fmaxf(v1 + __ldg(bias + co + 1), 0.f);
            } else {
                const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + p * 16 + co);
                if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
                if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
            }
            *reinterpret_cast<__nv_bfloat162*>(out + p * 16 + co) = __floats2bfloat162_rn(v0, v1);
        }
    }
}

// ---------------------------------------------------------------- first layer: cin -> 16 (SIMT)
template <int CIN>
__global__ void __launch_bounds__(256) k_conv_first(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                    const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                    int nx, int ny, int nz) {
    __shared__ float w[16 * CIN * 27];
    for (int q = threadIdx.x; q < 16 * CIN * 27; q += blockDim.x) w[q] = __bfloat162float(W[q]);
    __syncthreads();
    const size_t n = (size_t)nx * ny * nz;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((size_t)nx * ny));
    float acc[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) acc[co] = __ldg(bias + co);
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = k + dz;
        if (kk < 0 || kk >= nz) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int tap = ((dz + 1) * 3 + dy + 1) * 3 + dx + 1;
                const size_t q = ((size_t)kk * ny + nwrap(j + dy, ny)) * nx + nwrap(i + dx, nx);
#pragma unroll
                for (int ci = 0; ci < CIN; ++ci) {
                    const float xv = __bfloat162float(in[q * CIN + ci]);
#pragma unroll
                    for (int co = 0; co < 16; ++co) acc[co] = fmaf(w[(co * CIN + ci) * 27 + tap], xv, acc[co]);
                }
            }
    }
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) o[co] = __float2bfloat16_rn(fmaxf(acc[co], 0.f));
    reinterpret_cast<uint4*>(out + p * 16)[0] = reinterpret_cast<uint4*>(o)[0];
    reinterpret_cast<uint4*>(out + p * 16)[1] = reinterpret_cast<uint4*>(o)[1];
}

// ---------------------------------------------------------------- last layer: 16 -> 1 (SIMT)
__global__ void __launch_bounds__(256) k_conv_last(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ bias, float* __restrict__ out, int nx,
                                                   int ny, int nz) {
    __shared__ float w[16 * 27];
    for (int q = threadIdx.x; q < 16 * 27; q += blockDim.x) w[q] = __bfloat162float(W[q]);
    __syncthreads();
    const size_t n = (size_t)nx * ny * nz;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((size_t)nx * ny));
    float acc = __ldg(bias);
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = k + dz;
        if (kk < 0 || kk >= nz) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int tap = ((dz + 1) * 3 + dy + 1) * 3 + dx + 1;
                const size_t q = ((size_t)kk * ny + nwrap(j + dy, ny)) * nx + nwrap(i + dx, nx);
                __align__(16) __nv_bfloat16 a[16];
                reinterpret_cast<uint4*>(a)[0] = __ldg(reinterpret_cast<const uint4*>(in + q * 16));
                reinterpret_cast<uint4*>(a)[1] = __ldg(reinterpret_cast<const uint4*>(in + q * 16) + 1);
#pragma unroll
                for (int ci = 0; ci < 16; ++ci) acc = fmaf(w[ci * 27 + tap], __bfloat162float(a[ci]), acc);
            }
    }
    out[p] = acc;
}

// ---------------------------------------------------------------- backward of the last layer
// d3[ci](p) = mask(a3) * sum_d W4[ci][d] d4(p - d): the transposed 16 <- 1 convolution
__global__ void __launch_bounds__(256) k_bwd_last(const float* __restrict__ d4, const __nv_bfloat16* __restrict__ W,
                                                  const __nv_bfloat16* __restrict__ a3, __nv_bfloat16* __restrict__ d3,
                                                  int nx, int ny, int nz) {
    __shared__ float w[16 * 27];
    for (int q = threadIdx.x; q < 16 * 27; q += blockDim.x) w[q] = __bfloat162float(W[q]);
    __syncthreads();
    const size_t n = (size_t)nx * ny * nz;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((size_t)nx * ny));
    float acc[16];
#pragma unroll
    for (int ci = 0; ci < 16; ++ci) acc[ci] = 0.f;
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = k - dz;
        if (kk < 0 || kk >= nz) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int tap = ((dz + 1) * 3 + dy + 1) * 3 + dx + 1;
                const float g = __ldg(d4 + ((size_t)kk * ny + nwrap(j - dy, ny)) * nx + nwrap(i - dx, nx));
#pragma unroll
                for (int ci = 0; ci < 16; ++ci) acc[ci] = fmaf(w[ci * 27 + tap], g, acc[ci]);
            }
    }
    __align__(16) __nv_bfloat16 m[16], o[16];
    reinterpret_cast<uint4*>(m)[0] = __ldg(reinterpret_cast<const uint4*>(a3 + p * 16));
    reinterpret_cast<uint4*>(m)[1] = __ldg(reinterpret_cast<const uint4*>(a3 + p * 16) + 1);
#pragma unroll
    for (int ci = 0; ci < 16; ++ci) o[ci] = __float2bfloat16_rn(__bfloat162float(m[ci]) > 0.f ? acc[ci] : 0.f);
    reinterpret_cast<uint4*>(d3 + p * 16)[0] = reinterpret_cast<uint4*>(o)[0];
    reinterpret_cast<uint4*>(d3 + p * 16)[1] = reinterpret_cast<uint4*>(o)[1];
}

// ---------------------------------------------------------------- weight gradient, 16 -> 16 layers
// dW[co][ci][tap] = sum_p dy[co](p) x[ci](p + d): per tap a GEMM (16 co) x (cells) x (16 ci) on the
// tensor cores; warp w accumulates the taps w, w+8, w+16, w+24 over the block's tiles, then writes
// one partial sum per (block, tap, co, ci).
__global__ void __launch_bounds__(256) k_dw16(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
                                              float* __restrict__ partials, int nx, int ny, int nz) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* H = smem;
    unsigned char* D = smem + HALO_BYTES;  // 128 cells x 16 channels of dy
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float acc[4][2][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const int tiles_x = nx / TXC, tiles_y = ny / TYC;
    const long ntiles = (long)tiles_x * tiles_y * nz;
    const int q8 = lane >> 3, rr = lane & 7;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = (int)(t % tiles_x), ty = (int)((t / tiles_x) % tiles_y), k = (int)(t / ((long)tiles_x * tiles_y));
        const int x0 = tx * TXC, y0 = ty * TYC;
        __syncthreads();
        load_halo16(x, nx, ny, nz, x0, y0, k, H);
        for (int q = threadIdx.x; q < TXC * TYC * 2; q += blockDim.x) {
            const int v = q >> 1, half = q & 1;
            const int xx = v % TXC, yy = v / TXC;
            const size_t p = ((size_t)k * ny + y0 + yy) * nx + x0 + xx;
            reinterpret_cast<uint4*>(D)[q] = __ldg(reinterpret_cast<const uint4*>(dy + p * 16) + half);
        }
        __syncthreads();
        // 8 chunks of 16 cells: (row, 16-cell column block)
#pragma unroll 1
        for (int ch = 0; ch < 8; ++ch) {
            const int yw = ch >> 2, xc = (ch & 3) * 16;
            // A = dy^T (co x cells): stored [cell][co] -> transposed load
            uint32_t a0, a1, a2, a3;
            {
                const int cellrow = (q8 >> 1) * 8 + rr, coff = (q8 & 1) * 8;
                ldm_x4_t(saddr(D + ((yw * TXC + xc + cellrow) * 16 + coff) * 2), a0, a1, a2, a3);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int tap = warp + 8 * s;
                if (tap >= 27) break;
                const int dz = tap / 9, dyy = (tap / 3) % 3, dxx = tap % 3;
                // B = shifted x (cells x ci): stored [cell][ci] -> transposed load
                const int cellrow = (q8 & 1) * 8 + rr, cioff = (q8 >> 1) * 8;
                const int cell = (dz * HY + yw + dyy) * HX + xc + cellrow + dxx;
                uint32_t b0, b1, b2, b3;
                ldm_x4_t(saddr(H + (cell * 16 + cioff) * 2), b0, b1, b2, b3);
                mma16816(acc[s][0], a0, a1, a2, a3, b0, b1);
                mma16816(acc[s][1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int tap = warp + 8 * s;
        if (tap >= 27) break;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = g + 8 * h, ci = t2 + 8 * nt;
                float* dst = partials + (size_t)blockIdx.x * (16 * 16 * 27);
                dst[(co * 16 + ci) * 27 + tap] = acc[s][nt][2 * h];
                dst[(co * 16 + ci + 1) * 27 + tap] = acc[s][nt][2 * h + 1];
            }
    }
}

// ---------------------------------------------------------------- weight gradient of thin layers
// dW[co][ci][tap] for a layer with CIN inputs and COUT outputs where one side is thin: one thread per
// weight, a block per slice of cells, one partial sum per (block, weight). x: CIN channels-last bf16;
// dy: COUT channels (bf16 channels-last, or fp32 when COUT == 1).
template <int CIN, int COUT, bool DYF32>
__global__ void k_dw_thin(const __nv_bfloat16* __restrict__ x, const void* __restrict__ dyv, float* __restrict__ partials,
                          int nx, int ny, int nz, size_t cells_per_block) {
    constexpr int NW = COUT * CIN * 27;
    const size_t n = (size_t)nx * ny * nz;
    const size_t p0 = blockIdx.x * cells_per_block, p1 = p0 + cells_per_block < n ? p0 + cells_per_block : n;
    for (int wi = threadIdx.x; wi < NW; wi += blockDim.x) {
        const int co = wi / (CIN * 27), ci = (wi / 27) % CIN, tap = wi % 27;
        const int dz = tap / 9 - 1, dyy = (tap / 3) % 3 - 1, dxx = tap % 3 - 1;
        float s = 0.f;
        for (size_t p = p0; p < p1; ++p) {
            const int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((size_t)nx * ny));
            const int kk = k + dz;
            if (kk < 0 || kk >= nz) continue;
            const float g = DYF32 ? __ldg(reinterpret_cast<const float*>(dyv) + p)
                                  : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(dyv)[p * COUT + co]);
            const size_t q = ((size_t)kk * ny + nwrap(j + dyy, ny)) * nx + nwrap(i + dxx, nx);
            s = fmaf(g, __bfloat162float(x[q * CIN + ci]), s);
        }
        partials[(size_t)blockIdx.x * NW + wi] = s;
    }
}

// per-channel sums of dy (bias gradients): one partial per (block, channel)
template <int C, bool F32>
__global__ void k_chansum(const void* __restrict__ dyv, float* __restrict__ partials, size_t n, size_t cells_per_block) {
    __shared__ float red[256];
    const size_t p0 = blockIdx.x * cells_per_block, p1 = p0 + cells_per_block < n ? p0 + cells_per_block : n;
    for (int c = 0; c < C; ++c) {
        float s = 0.f;
        for (size_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
            s += F32 ? __ldg(reinterpret_cast<const float*>(dyv) + p)
                     : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(dyv)[p * C + c]);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * C + c] = red[0];
        __syncthreads();
    }
}

// out[e] = sum over blocks b of partials[b * nelem + e] (fixed order)
__global__ void k_reduce_partials(const float* __restrict__ partials, int nblocks, int nelem, float* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nelem) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * nelem + e];
    out[e] = (float)s;
}

// ---------------------------------------------------------------- parameters
// master fp32 params (flat, W[co][ci][tap] per layer) -> bf16 weights: W1, W4 as stored; W2, W3 as
// [tap][co][ci] for the forward GEMM and [tap'][ci][co] with tap' the mirrored tap for the data
// gradient (transposed convolution).
__global__ void k_prepare_weights(const float* __restrict__ params, int cin, __nv_bfloat16* __restrict__ w1,
                                  __nv_bfloat16* __restrict__ w2f, __nv_bfloat16* __restrict__ w2b,
                                  __nv_bfloat16* __restrict__ w3f, __nv_bfloat16* __restrict__ w3b,
                                  __nv_bfloat16* __restrict__ w4) {
    const int n1 = 16 * cin * 27, n2 = 16 * 16 * 27, n4 = 16 * 27;
    const float* W1 = params;
    const float* W2 = W1 + n1 + 16;
    const float* W3 = W2 + n2 + 16;
    const float* W4 = W3 + n2 + 16;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
        if (e < n1) w1[e] = __float2bfloat16_rn(W1[e]);
        if (e < n4) w4[e] = __float2bfloat16_rn(W4[e]);
        const int co = e / (16 * 27), ci = (e / 27) % 16, tap = e % 27;
        const int mirror = 26 - tap;
        w2f[(tap * 16 + co) * 16 + ci] = __float2bfloat16_rn(W2[e]);
        w3f[(tap * 16 + co) * 16 + ci] = __float2bfloat16_rn(W3[e]);
        w2b[(mirror * 16 + ci) * 16 + co] = __float2bfloat16_rn(W2[e]);
        w3b[(mirror * 16 + ci) * 16 + co] = __float2bfloat16_rn(W3[e]);
    }
}

// Adam (Kingma & Ba 2015) on fp32 master parameters
__global__ void k_adam(int n, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    theta[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// partial sums of the loss mean (out - target)^2 (each block's sum divided by n); d4 = 2 (out - target) / n
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ target, float* __restrict__ d4,
                      double* __restrict__ partials, size_t n) {
    double s = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const float e = out[p] - target[p];
        d4[p] = 2.f * e / (float)n;
        s += (double)e * e;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0] / (double)n;
}

// residual loss: e = r - q with r the input's channel 0 and q = A NN(x); tmp = -2 e / n (A tmp is
// then the loss gradient w.r.t. the output); partial sums of e^2 / n per block
__global__ void k_res_loss(const __nv_bfloat16* __restrict__ x, int cin, const float* __restrict__ q,
                           float* __restrict__ tmp, double* __restrict__ partials, size_t n) {
    double s = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const float e = __bfloat162float(x[p * cin]) - q[p];
        tmp[p] = -2.f * e / (float)n;
        s += (double)e * e;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0] / (double)n;
}

// network input from a residual: channel 0 = r / rms(r) (rms from *sumsq), channel 1 = aux per
// column; optional target D (ea - eb) / rms(r) (the error of an iterate, exact solution minus
// iterate, in the network's output unit D^{-1}; D from cx2cy2 = 2cx + 2cy and v32 per column)
template <class SR>
__global__ void k_make_input(size_t n, size_t ncol, int nz, int cin, const SR* __restrict__ r,
                             const float* __restrict__ aux, const double* __restrict__ sumsq,
                             __nv_bfloat16* __restrict__ x, const double* __restrict__ ea,
                             const double* __restrict__ eb, float cx2cy2, const float* __restrict__ v32,
                             float* __restrict__ target) {
    const double rms = sqrt(*sumsq / (double)n);
    const double inv = rms > 0.0 ? 1.0 / rms : 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        double rv;
        if constexpr (std::is_same<SR, double>::value) rv = r[p];
        else rv = (double)r[p].x + (double)r[p].y;
        x[p * cin] = __float2bfloat16_rn((float)(rv * inv));
        if (cin > 1) x[p * cin + 1] = __float2bfloat16_rn(aux[p % ncol]);
        if (target) {
            const float dinv = diag_inv_f32(cx2cy2, v32[p % ncol], (int)(p / ncol), nz);
            target[p] = (float)((ea[p] - eb[p]) * inv) / dinv;
        }
    }
}

// out = D^{-1} in (D = diag(A) of an FP32 level)
__global__ void k_scale_dinv(size_t n, size_t ncol, int nz, float cx2cy2, const float* __restrict__ v32,
                             const float* __restrict__ in, float* __restrict__ out) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        out[p] = in[p] * diag_inv_f32(cx2cy2, __ldg(v32 + p % ncol), (int)(p / ncol), nz);
}

// ================================================================ host launchers
void nn_prepare_weights(const NNBufs& b, cudaStream_t s) {
    k_prepare_weights<<<27, 256, 0, s>>>(b.params, b.cin, b.w1, b.w2f, b.w2b, b.w3f, b.w3b, b.w4);
    note_launch();
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256); }

void nn_forward(const NNBufs& b, int nx, int ny, int nz, const __nv_bfloat16* x, float* out, cudaStream_t s) {
    const size_t n = (size_t)nx * ny * nz;
    const float* b1 = b.params + 16 * b.cin * 27;
    const float* b2 = b1 + 16 + 16 * 16 * 27;
    const float* b3 = b2 + 16 + 16 * 16 * 27;
    const float* b4 = b3 + 16 + 16 * 27;
    if (b.cin == 1) k_conv_first<1><<<blocks_for(n), 256, 0, s>>>(x, b.w1, b1, b.a1, nx, ny, nz);
    else k_conv_first<2><<<blocks_for(n), 256, 0, s>>>(x, b.w1, b1, b.a1, nx, ny, nz);
    note_launch();
    const size_t smem = HALO_BYTES + W_BYTES;
    cudaFuncSetAttribute(k_conv16<EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grd(nx / TXC, ny / TYC, nz);
    k_conv16<EPI_RELU><<<grd, 256, smem, s>>>(b.a1, b.w2f, b2, nullptr, b.a2, nx, ny, nz);
    note_launch();
    k_conv16<EPI_RELU><<<grd, 256, smem, s>>>(b.a2, b.w3f, b3, nullptr, b.a3, nx, ny, nz);
    note_launch();
    k_conv_last<<<blocks_for(n), 256, 0, s>>>(b.a3, b.w4, b4, out, nx, ny, nz);
    note_launch();
}

int nn_grad_blocks(size_t n) {
    size_t b = (n + 4095) / 4096;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

void nn_backward(const NNBufs& b, int nx, int ny, int nz, const __nv_bfloat16* x, const float* d4, float* grad,
                 cudaStream_t s) {
    const size_t n = (size_t)nx * ny * nz;
    const int cin = b.cin;
    const int n1 = 16 * cin * 27, n2 = 16 * 16 * 27, n4 = 16 * 27;
    float* gW1 = grad;
    float* gb1 = gW1 + n1;
    float* gW2 = gb1 + 16;
    float* gb2 = gW2 + n2;
    float* gW3 = gb2 + 16;
    float* gb3 = gW3 + n2;
    float* gW4 = gb3 + 16;
    float* gb4 = gW4 + n4;
    const int nb = nn_grad_blocks(n);
    const size_t cpb = (n + nb - 1) / nb;
    // layer 4: dW4, db4 and d3 = mask(a3) * W4^T d4
    k_dw_thin<16, 1, true><<<nb, 128, 0, s>>>(b.a3, d4, b.part, nx, ny, nz, cpb);
    k_reduce_partials<<<(n4 + 255) / 256, 256, 0, s>>>(b.part, nb, n4, gW4);
    k_chansum<1, true><<<nb, 256, 0, s>>>(d4, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 1, gb4);
    k_bwd_last<<<blocks_for(n), 256, 0, s>>>(d4, b.w4, b.a3, b.d1, nx, ny, nz);
    for (int q = 0; q < 5; ++q) note_launch();
    const size_t smem = HALO_BYTES + W_BYTES;
    cudaFuncSetAttribute(k_conv16<EPI_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const size_t smem_dw = HALO_BYTES + TXC * TYC * 32;
    cudaFuncSetAttribute(k_dw16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dw);
    dim3 grd(nx / TXC, ny / TYC, nz);
    // layer 3: dW3 from (a2, d3); d2 = mask(a2) * conv(d3, W3 flipped)
    k_dw16<<<nb, 256, smem_dw, s>>>(b.a2, b.d1, b.part, nx, ny, nz);
    k_reduce_partials<<<(n2 + 255) / 256, 256, 0, s>>>(b.part, nb, n2, gW3);
    k_chansum<16, false><<<nb, 256, 0, s>>>(b.d1, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 16, gb3);
    k_conv16<EPI_MASK><<<grd, 256, smem, s>>>(b.d1, b.w3b, nullptr, b.a2, b.d2, nx, ny, nz);
    // layer 2: dW2 from (a1, d2); d1 = mask(a1) * conv(d2, W2 flipped)
    k_dw16<<<nb, 256, smem_dw, s>>>(b.a1, b.d2, b.part, nx, ny, nz);
    k_reduce_partials<<<(n2 + 255) / 256, 256, 0, s>>>(b.part, nb, n2, gW2);
    k_chansum<16, false><<<nb, 256, 0, s>>>(b.d2, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 16, gb2);
    k_conv16<EPI_MASK><<<grd, 256, smem, s>>>(b.d2, b.w2b, nullptr, b.a1, b.d1, nx, ny, nz);
    // layer 1: dW1 from (x, d1)
    if (cin == 1) k_dw_thin<1, 16, false><<<nb, 128, 0, s>>>(x, b.d1, b.part, nx, ny, nz, cpb);
    else k_dw_thin<2, 16, false><<<nb, 128, 0, s>>>(x, b.d1, b.part, nx, ny, nz, cpb);
    k_reduce_partials<<<(n1 + 255) / 256, 256, 0, s>>>(b.part, nb, n1, gW1);
    k_chansum<16, false><<<nb, 256, 0, s>>>(b.d1, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 16, gb1);
    for (int q = 0; q < 14; ++q) note_launch();
}

void nn_mse(const float* out, const float* target, float* d4, double* partials, size_t n, int nblocks, cudaStream_t s) {
    k_mse<<<nblocks, 256, 0, s>>>(out, target, d4, partials, n);
    note_launch();
}

void nn_res_loss(const __nv_bfloat16* x, int cin, const float* q, float* tmp, double* partials, size_t n, int nblocks,
                 cudaStream_t s) {
    k_res_loss<<<nblocks, 256, 0, s>>>(x, cin, q, tmp, partials, n);
    note_launch();
}

void nn_adam(int n, float* theta, const float* g, float* m, float* v, float lr, int t, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(n, theta, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
    note_launch();
}

void nn_make_input_f64(size_t n, size_t ncol, int nz, int cin, const double* r, const float* aux, const double* sumsq,
                       __nv_bfloat16* x, const double* ea, const double* eb, double cx, double cy, const float* v32,
                       float* target, cudaStream_t s) {
    k_make_input<double><<<blocks_for(n) < 4096 ? blocks_for(n) : 4096, 256, 0, s>>>(
        n, ncol, nz, cin, r, aux, sumsq, x, ea, eb, (float)(2.0 * cx + 2.0 * cy), v32, target);
    note_launch();
}
void nn_make_input_dw(size_t n, size_t ncol, int nz, int cin, const float2* r, const float* aux, const double* sumsq,
                      __nv_bfloat16* x, cudaStream_t s) {
    k_make_input<float2><<<blocks_for(n) < 4096 ? blocks_for(n) : 4096, 256, 0, s>>>(
        n, ncol, nz, cin, r, aux, sumsq, x, nullptr, nullptr, 0.f, nullptr, nullptr);
    note_launch();
}
void nn_scale_dinv(size_t n, size_t ncol, int nz, double cx, double cy, const float* v32, const float* in, float* out,
                   cudaStream_t s) {
    k_scale_dinv<<<blocks_for(n) < 4096 ? blocks_for(n) : 4096, 256, 0, s>>>(n, ncol, nz, (float)(2.0 * cx + 2.0 * cy),
                                                                             v32, in, out);
    note_launch();
}

}  // namespace tpmg
