// k_nn.cu -- the learned preconditioner stage: a 4-layer 3-D convolutional network (cin -> 16 ->
// 16 -> 16 -> 1, 3x3x3 kernels, ReLU after the first three layers, periodic padding in x and y,
// zero padding in z), its training kernels and Adam.
//
// Activations are channels-last BF16 (16 channels = 32 bytes per cell, cell index (k*ny + j)*nx + i);
// weights are BF16 copies of FP32 master parameters; all sums accumulate in FP32.
// Where nx is a multiple of 128 (and ny of 4), every layer is an implicit GEMM on the fifth-generation
// tensor cores (tcgen05, accumulators in tensor memory) in one rolling scheme over the z planes:
// k_conv16_roll (the 16 -> 16 layers, their data gradient, and the 2 -> 16 first layer) and
// k_last_roll (16 -> 1). Other shapes use mma.sync kernels: k_conv16z (16 -> 16: tiles of 64 x 2
// cells, each warp 16 consecutive cells as the M = 16 rows of mma.m16n8k16, K over the 27 taps x 16
// input channels, operands by ldmatrix), k_first_z / k_first_tc2 and k_last_proj. The weight
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

// ---------------------------------------------------------------- 16 -> 16, marching in z
// The same implicit GEMM as k_conv16, but a persistent block stages the weights once and walks
// whole columns of tiles: it keeps the planes k-1, k, k+1 of its 66 x 4 halo tile in a 4-slot ring
// and fetches plane k+2 with cp.async while the tensor cores work on plane k, so every input plane
// is read once per tile (not three times) and the loads overlap the MMAs.
__device__ __forceinline__ unsigned sa_nn(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa_nn(dst)), "l"(src));
}
__device__ __forceinline__ void cp4nn(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa_nn(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit_nn() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait_nn() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

static constexpr int PLANE_CELLS = HX * HY;        // 66 x 4 cells of one halo plane
static constexpr int PLANE_BYTES = PLANE_CELLS * 32;

// Shared-memory offset of the 16-byte half `h` of 32-byte row `r` (a cell's 16 channels, or a
// weight row): the halves of rows 4..7 (mod 8) swap places, so the 8 rows an ldmatrix phase reads
// (32 bytes apart) fall on 8 distinct groups of 4 banks instead of 2-way conflicts.
__device__ __forceinline__ int swz(int r, int h) { return r * 32 + ((h ^ ((r >> 2) & 1)) << 4); }

// MT m-tiles (16 cells each) per warp: the weight fragment of a tap is loaded once for MT tiles
template <int EPI, int MT>
__global__ void __launch_bounds__(256 / MT) k_conv16z(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wt,
                                                      const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask,
                                                      __nv_bfloat16* __restrict__ out, int nx, int ny, int nz) {
    constexpr int WPR = 4 / MT;  // warps per tile row
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* Ws = smem;
    unsigned char* ring = smem + W_BYTES;  // 4 planes
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int q = tid; q < W_BYTES / 16; q += blockDim.x)
        *reinterpret_cast<uint4*>(Ws + swz(q >> 1, q & 1)) = __ldg(reinterpret_cast<const uint4*>(Wt) + q);
    const int tiles_x = nx / TXC, ntiles = tiles_x * (ny / TYC);
    const int yw = warp / WPR, xw = (warp % WPR) * 16 * MT;
    const int ar = lane & 15, acol = (lane >> 4) * 8;
    const int bco = ((lane >> 4) << 3) + (lane & 7), bci = ((lane >> 3) & 1) * 8;
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    float bco0 = 0.f, bco1 = 0.f, bco8 = 0.f, bco9 = 0.f;
    if (EPI == EPI_RELU) {
        bco0 = __ldg(bias + t2);
        bco1 = __ldg(bias + t2 + 1);
        bco8 = __ldg(bias + t2 + 8);
        bco9 = __ldg(bias + t2 + 9);
    }
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TXC, y0 = (tile / tiles_x) * TYC;
        // plane kk of the tile into ring slot (kk + 1) & 3 (zeros beyond the z ends)
        auto load_plane = [&](int kk) {
            unsigned char* P = ring + ((kk + 1) & 3) * PLANE_BYTES;
            for (int q = tid; q < PLANE_CELLS * 2; q += blockDim.x) {
                const int v = q >> 1, half = q & 1;
                const int xx = v % HX, yy = v / HX;
                if (kk >= 0 && kk < nz) {
                    const int i = nwrap(x0 - 1 + xx, nx), j = nwrap(y0 - 1 + yy, ny);
                    cp16(P + swz(v, half), in + (((size_t)kk * ny + j) * nx + i) * 16 + half * 8);
                } else {
                    *reinterpret_cast<uint4*>(P + swz(v, half)) = make_uint4(0, 0, 0, 0);
                }
            }
            cp_commit_nn();
        };
        __syncthreads();  // the previous tile's ring (and, first time, the weights) are settled
        load_plane(-1);
        load_plane(0);
        load_plane(1);
        for (int k = 0; k < nz; ++k) {
            load_plane(k + 2);  // into the slot of plane k-2, read by nobody now
            cp_wait_nn<1>();    // planes up to k+1 have landed (this thread's copies)
            __syncthreads();    // ... and every other thread's
            float c[MT][2][4];
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) c[m][nt][e] = 0.f;
#pragma unroll 1
            for (int dz = 0; dz < 3; ++dz) {
                const unsigned char* H = ring + ((k + dz) & 3) * PLANE_BYTES;  // plane k - 1 + dz
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int tap = (dz * 3 + dy) * 3 + dx;
                        uint32_t b0, b1, b2, b3;
                        ldm_x4(saddr(Ws + swz(tap * 16 + bco, bci >> 3)), b0, b1, b2, b3);
#pragma unroll
                        for (int m = 0; m < MT; ++m) {
                            const int cell = (yw + dy) * HX + xw + 16 * m + ar + dx;
                            uint32_t a0, a1, a2, a3;
                            ldm_x4(saddr(H + swz(cell, acol >> 3)), a0, a1, a2, a3);
                            mma16816(c[m][0], a0, a1, a2, a3, b0, b1);
                            mma16816(c[m][1], a0, a1, a2, a3, b2, b3);
                        }
                    }
            }
            const int y = y0 + yw;
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int x = x0 + xw + 16 * m + g + 8 * h;
                    const size_t p = ((size_t)k * ny + y) * nx + x;
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        const int co = t2 + 8 * nt;
                        float v0 = c[m][nt][2 * h], v1 = c[m][nt][2 * h + 1];
                        if (EPI == EPI_RELU) {
                            v0 = fmaxf(v0 + (nt ? bco8 : bco0), 0.f);
                            v1 = fmaxf(v1 + (nt ? bco9 : bco1), 0.f);
                        } else {
                            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + p * 16 + co);
                            if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                            if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                        }
                        *reinterpret_cast<__nv_bfloat162*>(out + p * 16 + co) = __floats2bfloat162_rn(v0, v1);
                    }
                }
            __syncthreads();  // the slot of plane k-1 is refilled by the next step's load
        }
        cp_wait_nn<0>();
    }
}

static constexpr int CONV_MT = 2;  // m-tiles per warp of the 16 -> 16 convolution

static int conv16z_grid(int nx, int ny) {
    static int per_sm = 0, nsm = 0;
    const size_t smem = W_BYTES + 4 * PLANE_BYTES;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_conv16z<EPI_RELU, CONV_MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_conv16z<EPI_MASK, CONV_MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv16z<EPI_RELU, CONV_MT>, 256 / CONV_MT, smem);
        if (per_sm < 1) per_sm = 1;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    const int ntiles = (nx / TXC) * (ny / TYC);
    const int nb = per_sm * nsm;
    return nb < ntiles ? nb : ntiles;
}

// ---------------------------------------------------------------- 16 -> 16 on tcgen05: common parts
// Tiles of TR rows of TCX = 128 consecutive x cells (M = 128 per MMA); a halo plane of the tile is
// TR + 2 rows of 130 cells in shared memory, in the canonical no-swizzle K-major layout of the MMA
// operands: per row the two 8-channel K halves one after the other, 16-byte rows of 8 channels, 8
// cells per 128-byte core matrix, so the A operand of a tap's shift dx is the halo row viewed from
// cell dx (a 16-byte aligned view, no copy).
static constexpr int TCX = 128;                     // cells per tile row
static constexpr int TC_ROWC = TCX + 2;             // halo row cells
static constexpr int TC_HALF = TC_ROWC * 16;        // bytes of one K half of a halo row
static constexpr int TC_ROWB = 2 * TC_HALF;         // bytes of one halo row (both K halves)
static constexpr long long TC_SPIN = 1LL << 26;     // bound of every mbarrier wait

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start address >> 4 (bits 0-13), leading (K) byte offset >> 4 (16-29), stride (M/N) byte
    // offset >> 4 (32-45), descriptor version 1 (46-47), base offset 0, no swizzle (61-63 = 0)
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// kind::f16 instruction descriptors below: D FP32 (bit 4), A and B BF16 (bits 7, 10), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24

// bounded wait on an mbarrier phase that also returns (false) once *abort is set
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, const volatile int* abort) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// ---------------------------------------------------------------- 16 -> 16 on tcgen05, rolling planes
// The implicit GEMM with MMAs of up to N = 144. A tcgen05.mma with M = 128 and K = 16 whose operands
// come fresh from shared memory costs about the same up to N = 144 (measured: 69 cycles at N = 16,
// 48 and 96, 72 at 144, 128 at 256), so each MMA should produce many output columns. One input view
// -- plane p, halo row h, shift dx -- feeds nine outputs: rows h-2, h-1, h (taps dy = 2, 1, 0) of
// output planes p+1, p, p-1 (taps dz = 0, 1, 2). The accumulators of three consecutive output planes
// live in tensor memory by residue q = plane mod 3, row-major: column 48 r + 16 q + channel for tile
// row r, so the outputs of a view inside the tile are contiguous columns (N = 144 for the inner
// rows, 96 or 48 for the two halo rows at each end, whose other outputs lie outside the tile); B holds
// the nine taps' weights in that order, rotated with p mod 3 (3 rotations x 3 shifts = 9 matrices),
// and a narrower MMA reads the rows of B it needs. Per input plane 3 (TR + 2) MMAs; after them output
// plane p-1 is complete and the input plane is never read again, so the z padding needs no planes.
// Tiles of TR = 4 rows: a block works on two tiles at once, plane by plane in turn, each with its own
// window of 48 TR columns, so the MMAs of one tile run while the epilogue drains the other's window.
// Tiles of TR = 8 rows (fewer MMAs per row; one window of 384 columns): the epilogue hands rows 0-3
// and 4-7 back on separate barriers, and the MMA thread issues the views of the first rows while the
// others drain. The first layer (FIRST) folds the three shifts into K (2 channels x 3 shifts = 6 of
// K = 16): one MMA per halo row. Roles:
//   producer warps (4): copy the input planes into a ring of SLOTS planes with cp.async, each
//     thread's copies followed by cp.async.mbarrier.arrive on the slot's `full` mbarrier (first
//     layer: raw rows into a ring of their own, then each producer writes its cell's operand rows);
//   one MMA thread: per input plane waits for it (`full`) and for the epilogue to have zeroed the
//     residue block it opens in its tile's window (`acce` of that window), issues the MMAs, commits
//     to the window's `accf` and releases the plane's slot (`empty`, by tcgen05.commit);
//   epilogue warps (4 per group of tile rows, TR / 4 rows per thread): per input plane p drain output
//     plane p-1 of the tile (and, after the tile's last plane, plane nz-1), round it to BF16 (bias +
//     ReLU first in the forward pass), zero the drained residue blocks (after the last plane all
//     three), arrive on `acce`, then (with the backward pass's ReLU mask) write the warp's BF16
//     staging buffer, which the warp's lane 0 writes out by a bulk copy (TMA) of its 32 cells.
// Every wait is bounded and also gives up once another role has given up (a shared abort flag), which
// raises the error flag.
static constexpr int RL_NPROD = 128;
static constexpr int RL_BB = 144 * 32;  // one B matrix: [K half][144 rows][8 ci]
static constexpr int RL_WB = 9 * RL_BB;
__host__ __device__ constexpr uint32_t rl_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}
template <int TR, bool FIRST = false>
struct RlShape {
    // epilogue: one warp per lane quarter and row group, ERW row groups; a thread drains rows
    // erow, erow + ERW, ... (RPT of them)
    static constexpr int ERW = TR < 4 ? TR : 4;
    static constexpr int RPT = TR / ERW;
    static constexpr int NEPI = 128 * ERW;
    static constexpr int NPROD = RL_NPROD;  // producer threads (the full barrier's arrival count)
    static constexpr int NT = NEPI + 32 + NPROD;
    // weights: nine B matrices (rotation, dx); the first layer folds dx into K: three (rotation)
    static constexpr int WB = FIRST ? 3 * RL_BB : RL_WB;
    // one halo row of the A ring: 130 cells x 16 channels (both K halves), or for the first layer the
    // 128 cells of an operand row (K half 0: dx x 2 channels, K half 1 zero)
    static constexpr int ROWB = FIRST ? 2 * TCX * 16 : TC_ROWB;
    static constexpr int PLANEB = (TR + 2) * ROWB;
    // operand planes in flight or waiting (two rows: three, so that two blocks share an SM)
    static constexpr int SLOTS = FIRST ? 3 : (TR == 4 ? 6 : 3);
    // first layer: raw halo rows (130 cells x 2 BF16 channels, 12 bytes of padding on either side,
    // the 128 interior cells 16-byte aligned) in a ring of RAW planes
    static constexpr int RAWROW = 32 + TCX * 4;
    static constexpr int RAW = FIRST ? 8 : 0;
    static constexpr int RAWB = (TR + 2) * RAWROW;
    static constexpr int STAGE = NEPI * 32;  // 1 KB of BF16 output per epilogue warp
    // output staging buffers per epilogue warp: up to NSTG of a warp's 1 KB bulk stores are in flight,
    // which is what hides the write latency
    static constexpr int NSTG = 2;
    static constexpr int SMEM = WB + SLOTS * PLANEB + RAW * RAWB + NSTG * STAGE;
    static constexpr int WIN_COLS = 48 * TR;     // one tile's window of three output planes
    // two windows (a pair of tiles in turn) where the tensor memory holds them, else one
    static constexpr int NWIN = 2 * WIN_COLS <= 512 ? 2 : 1;
    static constexpr int TMEM_COLS = NWIN * WIN_COLS <= 256 ? 256 : 512;
    static_assert(TR >= 2 && TR % ERW == 0 && NWIN * WIN_COLS <= 512, "windows");
};

template <int EPI, int TR, bool FIRST = false>
__global__ void __launch_bounds__(RlShape<TR, FIRST>::NT) k_conv16_roll(const __nv_bfloat16* __restrict__ in,
                                                                 const __nv_bfloat16* __restrict__ Wt,
                                                                 const float* __restrict__ bias,
                                                                 const __nv_bfloat16* __restrict__ mask,
                                                                 __nv_bfloat16* __restrict__ out, int nx, int ny,
                                                                 int nz, int* err) {
    typedef RlShape<TR, FIRST> SH;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[SH::SLOTS], empty[SH::SLOTS], accf[2], acce[2];
    __shared__ uint32_t tmem_base;
    __shared__ float bsh[16];
    __shared__ volatile int abort;
    __shared__ volatile int pstat[2];  // first layer: the producers' verdict on step q, slot q & 1
    unsigned char* Ws = smem;
    unsigned char* ring = smem + SH::WB;
    unsigned char* raw = ring + SH::SLOTS * SH::PLANEB;  // first layer only
    unsigned char* stage = raw + SH::RAW * SH::RAWB;     // NSTG output staging buffers
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if constexpr (FIRST) {
        // B matrix (rotation rot), row 48 j + 16 q + co, K index 2 dx + ci (K 6 .. 15 zero): tap
        // dy = 2 - j, dz = (rot + 1 - q) mod 3 of W1[co][ci][tap]
        for (int e = tid; e < 3 * 144 * 16; e += SH::NT) {
            const int rot = e / 2304, n = (e >> 4) % 144, k = e & 15;
            const int j = n / 48, qq = (n / 16) % 3, co = n & 15;
            float wv = 0.f;
            if (k < 6) {
                const int dx = k >> 1, ci = k & 1, dy = 2 - j, dz = (rot + 4 - qq) % 3;
                wv = __bfloat162float(Wt[(co * 2 + ci) * 27 + (dz * 3 + dy) * 3 + dx]);
            }
            *reinterpret_cast<__nv_bfloat16*>(Ws + rot * RL_BB + (k >> 3) * (RL_BB / 2) + n * 16 + (k & 7) * 2) =
                __float2bfloat16_rn(wv);
        }
        // the operand ring starts at zero; its K half 1 is never written again
        for (int i = tid; i < SH::SLOTS * SH::PLANEB / 16; i += SH::NT)
            reinterpret_cast<uint4*>(ring)[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        // B matrix (rotation rot, shift dx), row 48 j + 16 q + co: tap dy = 2 - j, dz = (rot + 1 - q) mod 3
        for (int e = tid; e < 9 * 9 * 32; e += SH::NT) {
            const int mtx = e / 288, blk = (e / 32) % 9, co = (e >> 1) & 15, h = e & 1;
            const int rot = mtx / 3, dx = mtx % 3, j = blk / 3, qq = blk % 3;
            const int dy = 2 - j, dz = (rot + 4 - qq) % 3, tap = (dz * 3 + dy) * 3 + dx;
            *reinterpret_cast<uint4*>(Ws + mtx * RL_BB + h * (RL_BB / 2) + (blk * 16 + co) * 16) =
                __ldg(reinterpret_cast<const uint4*>(Wt + (tap * 16 + co) * 16 + h * 8));
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "n"(SH::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid < 16) bsh[tid] = (EPI == EPI_RELU) ? __ldg(bias + tid) : 0.f;
    if (tid == 0) {
        for (int s = 0; s < SH::SLOTS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[s])), "n"(SH::NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])));
        }
        for (int w = 0; w < 2; ++w) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&accf[w])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&acce[w])), "n"(SH::NEPI / 32));
        }
        abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");  // the weights, written by plain stores, for the MMAs
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // an epilogue warp zeroes its 32 lanes of tile row `row` in residue block q of window w
    auto zero_block = [&](int w, int q, int row) {
        const uint32_t z = 0;
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                tmem + w * SH::WIN_COLS + 48 * row + 16 * q + ((uint32_t)((warp & 3) * 32) << 16)),
            "r"(z)
            : "memory");
    };
    if (tid < SH::NEPI) {  // the windows start at zero; afterwards a block is zeroed as it is drained
        for (int w = 0; w < SH::NWIN; ++w)
            for (int rr = 0; rr < SH::RPT; ++rr)
                for (int q = 0; q < 3; ++q) zero_block(w, q, (warp >> 2) + SH::ERW * rr);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int tiles_x = nx / TCX, ntiles = tiles_x * (ny / TR);
    const int G = (int)gridDim.x;
    bool ok = true;
    // the block's tiles in pairs (t, t + G), t = blockIdx.x + 2 G i; a pair runs its planes in turn
    // (tile 0 of the pair, tile 1, next plane ...); a pair whose second tile does not exist runs alone
    if (tid >= SH::NEPI + 32) {
        if constexpr (FIRST) {
            // ---- producers, first layer: the pair's planes in turn. A plane's halo rows (130 cells x 2
            // BF16 channels) arrive by cp.async in a ring of RAW planes, DQ steps ahead; then each
            // producer writes the operand row of its cell: K = (dx, ci) for the shifts dx = 0 .. 2, the
            // three 4-byte channel pairs of cells x-1 .. x+1 side by side
            constexpr int CPR = TCX * 4 / 16 + 2;  // copies per halo row: 32 of 16 bytes, two halo cells
            constexpr int NCH = (TR + 2) * CPR, CPT = (NCH + SH::NPROD - 1) / SH::NPROD;
            constexpr int DQ = SH::RAW - 2;  // a raw slot is refilled two steps after it was read
            const int ptid = tid - (SH::NEPI + 32);
            int it0 = blockIdx.x, ip = 0, iw = 0, iq = 0;  // the next step to copy: pair, plane, tile
            auto issue = [&]() {
                if (it0 < ntiles) {
                    const int tile = it0 + iw * G;
                    const int x0 = (tile % tiles_x) * TCX, y0 = (tile / tiles_x) * TR;
                    unsigned char* R = raw + (iq % SH::RAW) * SH::RAWB;
                    const __nv_bfloat16* base = in + (size_t)ip * ny * nx * 2;
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const int qq = ptid + SH::NPROD * c;
                        if (qq < NCH) {
                            const int rr = qq / CPR, k = qq % CPR;
                            const size_t row = (size_t)nwrap(y0 - 1 + rr, ny) * nx;
                            unsigned char* d = R + rr * SH::RAWROW;
                            if (k < CPR - 2) cp16(d + 16 + 16 * k, base + (row + x0) * 2 + 8 * k);
                            else if (k == CPR - 2) cp4nn(d + 12, base + (row + nwrap(x0 - 1, nx)) * 2);
                            else cp4nn(d + 16 + TCX * 4, base + (row + nwrap(x0 + TCX, nx)) * 2);
                        }
                    }
                    ++iq;
                    const int nt = SH::NWIN == 2 && it0 + G < ntiles ? 2 : 1;
                    if (++iw == nt) {
                        iw = 0;
                        if (++ip == nz) {
                            ip = 0;
                            it0 += SH::NWIN * G;
                        }
                    }
                }
                cp_commit_nn();  // one group per step, empty past the block's last step
            };
            int nsteps = 0;
            for (int t0 = blockIdx.x; t0 < ntiles; t0 += SH::NWIN * G)
                nsteps += nz * (SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1);
            for (int i = 0; i < DQ; ++i) issue();
            for (int q = 0; q < nsteps; ++q) {
                issue();              // step q + DQ
                cp_wait_nn<DQ>();     // this thread's copies of step q have landed
                const int slot = q % SH::SLOTS;
                // one thread waits for the operand slot; the barrier hands its verdict (and, with the
                // other producers' copies, the whole raw plane) to all, so that all leave together
                if (ptid == 0)
                    pstat[q & 1] =
                        (q < SH::SLOTS || ws_wait(saddr(&empty[slot]), ((q / SH::SLOTS) - 1) & 1, &abort)) ? 1 : 0;
                asm volatile("bar.sync 1, %0;" ::"n"(SH::NPROD) : "memory");
                if (!pstat[q & 1]) {
                    ok = false;
                    break;
                }
                const unsigned char* R = raw + (q % SH::RAW) * SH::RAWB;
                unsigned char* A = ring + slot * SH::PLANEB;
                constexpr int HS = SH::NPROD / TCX;  // producers per cell: rows h0, h0 + HS, ...
                const int cell = ptid % TCX, h0 = ptid / TCX;
#pragma unroll
                for (int h = h0; h < TR + 2; h += HS) {
                    const uint32_t* r = reinterpret_cast<const uint32_t*>(R + h * SH::RAWROW + 12) + cell;
                    *reinterpret_cast<uint4*>(A + h * SH::ROWB + cell * 16) = make_uint4(r[0], r[1], r[2], 0u);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the operand, for the MMAs
                mbar_arrive(saddr(&full[slot]));
            }
            cp_wait_nn<0>();
        } else {
            // ---- producers: the pair's planes in turn into slot q % SLOTS of the ring
            const int ptid = tid - (SH::NEPI + 32);
            constexpr int NCH = (TR + 2) * TC_ROWC * 2, CPT = (NCH + SH::NPROD - 1) / SH::NPROD;
            int ch_dst[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int qq = ptid + SH::NPROD * c;
                ch_dst[c] = qq < NCH ? ((qq >> 1) / TC_ROWC) * TC_ROWB + (qq & 1) * TC_HALF + ((qq >> 1) % TC_ROWC) * 16 : -1;
            }
            int q = 0;
            for (int t0 = blockIdx.x; t0 < ntiles && ok; t0 += SH::NWIN * G) {
                const int nt = SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1;
                uint32_t src[SH::NWIN][CPT];  // element offsets within a plane (the caller keeps a plane below 2^32)
#pragma unroll
                for (int w = 0; w < SH::NWIN; ++w) {
                    const int tile = w < nt ? t0 + w * G : t0;
                    const int x0 = (tile % tiles_x) * TCX, y0 = (tile / tiles_x) * TR;
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const int qq = ptid + SH::NPROD * c;
                        const int hh = qq & 1, cc = (qq >> 1) % TC_ROWC, rr = (qq >> 1) / TC_ROWC;
                        src[w][c] = ((uint32_t)nwrap(y0 - 1 + rr, ny) * nx + nwrap(x0 - 1 + cc, nx)) * 16 + hh * 8;
                    }
                }
                for (int p = 0; p < nz && ok; ++p) {
                    for (int w = 0; w < nt; ++w, ++q) {
                        const int slot = q % SH::SLOTS;
                        if (q >= SH::SLOTS && !ws_wait(saddr(&empty[slot]), ((q / SH::SLOTS) - 1) & 1, &abort)) {
                            ok = false;
                            break;
                        }
                        unsigned char* P = ring + slot * SH::PLANEB;
                        const __nv_bfloat16* base = in + (size_t)p * ny * nx * 16;
#pragma unroll
                        for (int c = 0; c < CPT; ++c)
                            if (ch_dst[c] >= 0) cp16(P + ch_dst[c], base + src[w][c]);
                        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(&full[slot]))
                                     : "memory");
                    }
                }
            }
            cp_wait_nn<0>();
        }
    } else if (warp == SH::NEPI / 32) {
        // ---- MMA thread: one step per input plane of a tile, into that tile's window
        if (lane == 0) {
            const uint64_t dw0 = tc_desc(saddr(Ws), RL_BB / 2, 128);
            unsigned s = 0, cnt[2] = {0, 0};
            for (int t0 = blockIdx.x; t0 < ntiles && ok; t0 += SH::NWIN * G) {
                const int nt = SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1;
                for (int p = 0; p < nz && ok; ++p) {
                    for (int w = 0; w < nt; ++w, ++s) {
                        const int slot = s % SH::SLOTS;
                        // one window with two rows per epilogue thread: the epilogue hands the drained
                        // rows 0 .. ERW-1 back on acce[0] and the rest on acce[1], so that the views of
                        // the first rows go in while the last rows drain
                        constexpr bool SPLIT = SH::NWIN == 1 && SH::RPT == 2;
                        if (!ws_wait(saddr(&full[slot]), (s / SH::SLOTS) & 1, &abort) ||
                            (cnt[w] >= 1 && !ws_wait(saddr(&acce[w]), (cnt[w] - 1) & 1, &abort))) {
                            ok = false;
                            break;
                        }
                        // the plane's copies, observed through the barrier, ordered before the tensor
                        // core's reads; the zeroed window before its writes
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint64_t dp = tc_desc(saddr(ring + slot * SH::PLANEB), FIRST ? TCX * 16 : TC_HALF, 128);
                        const uint32_t win = tmem + w * SH::WIN_COLS;
                        const int rot = p % 3;
                        // the views of halo rows hlo .. hhi-1 (halo row h feeds tile rows h-2+j, j in [jlo, jhi])
                        auto views = [&](int hlo, int hhi) {
#pragma unroll
                            for (int h = hlo; h < hhi; ++h) {
                                const int jlo = h < 2 ? 2 - h : 0, jhi = h > TR - 1 ? TR + 1 - h : 2;
                                const uint32_t d = win + 48 * (h - 2 + jlo), idesc = rl_idesc(48 * (jhi - jlo + 1));
                                if constexpr (FIRST) {  // one MMA per halo row: K spans the three shifts
                                    const uint64_t da = dp + (uint64_t)((h * SH::ROWB) >> 4);
                                    const uint64_t db = dw0 + (uint64_t)((rot * RL_BB + 48 * jlo * 16) >> 4);
                                    asm volatile(
                                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                        "l"(da), "l"(db), "r"(idesc), "r"(1));
                                } else {
#pragma unroll
                                    for (int dx = 0; dx < 3; ++dx) {
                                        const uint64_t da = dp + (uint64_t)(((h * TC_ROWB) + dx * 16) >> 4);
                                        const uint64_t db = dw0 + (uint64_t)((((rot * 3 + dx) * RL_BB) + 48 * jlo * 16) >> 4);
                                        asm volatile(
                                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                            "l"(da), "l"(db), "r"(idesc), "r"(1));
                                    }
                                }
                            }
                        };
                        if constexpr (SPLIT) {
                            views(0, SH::ERW);  // tile rows up to ERW-1 (acce[0], waited above)
                            if (cnt[w] >= 1 && !ws_wait(saddr(&acce[1]), (cnt[w] - 1) & 1, &abort)) {
                                tc_commit(saddr(&accf[w]));  // the final wait covers the MMAs issued
                                ++cnt[w];
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;");
                            views(SH::ERW, TR + 2);
                        } else {
                            views(0, TR + 2);
                        }
                        tc_commit(saddr(&accf[w]));
                        tc_commit(saddr(&empty[slot]));  // the input plane has no later reader
                        ++cnt[w];
                    }
                }
            }
            // no MMA may be in flight when the tensor memory is freed (a bounded wait, abort or not)
            for (int w = 0; w < 2; ++w)
                if (cnt[w] > 0) tc_wait(saddr(&accf[w]), (cnt[w] - 1) & 1);
        }
    } else {
        // ---- epilogue: thread (erow, ecell) owns one cell of tile rows erow, erow + ERW, ...
        const int erow = warp >> 2, ecell = (warp & 3) * 32 + lane;
        constexpr bool SPLIT = SH::NWIN == 1 && SH::RPT == 2;  // rows handed back in two groups
        auto load16 = [&](int w, int q, int row, float (&v)[16]) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tmem + w * SH::WIN_COLS + 48 * row + 16 * q + ((uint32_t)((warp & 3) * 32) << 16)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
        };
        // a cell's 16 channels for output, rounded to BF16 and packed (forward: bias and ReLU first);
        // done before the window is handed back, so that a thread holds 8 registers per row, not 16
        auto pack = [&](float (&v)[16], uint4& o0, uint4& o1) {
            if (EPI == EPI_RELU) {
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = fmaxf(v[c] + bsh[c], 0.f);
            }
            __nv_bfloat162* h0 = reinterpret_cast<__nv_bfloat162*>(&o0);
            __nv_bfloat162* h1 = reinterpret_cast<__nv_bfloat162*>(&o1);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                h0[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
                h1[c] = __floats2bfloat162_rn(v[8 + 2 * c], v[8 + 2 * c + 1]);
            }
        };
        // output plane o of a tile: (data gradient: the ReLU mask, zeroing the rounded values, which
        // gives the bits of zeroing before the rounding) the warp's 32 cells (1 KB of BF16) into its
        // staging buffer `nemit % NSTG`, then one bulk copy (TMA) of them to global memory issued by the
        // warp's lane 0; a buffer is rewritten once the copy issued from it NSTG emits earlier has read it
        unsigned nemit = 0;
        auto emit = [&](int o, int x0, int y0, int row, uint4 o0, uint4 o1) {
            const size_t pidx = ((size_t)o * ny + y0 + row) * nx + x0 + ecell;
            if (EPI == EPI_MASK) {
                const uint4 m0 = __ldg(reinterpret_cast<const uint4*>(mask + pidx * 16));
                const uint4 m1 = __ldg(reinterpret_cast<const uint4*>(mask + pidx * 16 + 8));
                const __nv_bfloat16* mk0 = reinterpret_cast<const __nv_bfloat16*>(&m0);
                const __nv_bfloat16* mk1 = reinterpret_cast<const __nv_bfloat16*>(&m1);
                __nv_bfloat16* b0 = reinterpret_cast<__nv_bfloat16*>(&o0);
                __nv_bfloat16* b1 = reinterpret_cast<__nv_bfloat16*>(&o1);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (!(__bfloat162float(mk0[c]) > 0.f)) b0[c] = __float2bfloat16_rn(0.f);
                    if (!(__bfloat162float(mk1[c]) > 0.f)) b1[c] = __float2bfloat16_rn(0.f);
                }
            }
            unsigned char* B = stage + (nemit % SH::NSTG) * SH::STAGE + warp * 1024;
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(SH::NSTG - 1) : "memory");
            __syncwarp();  // the buffer's last copy has read it
            *reinterpret_cast<uint4*>(B + lane * 32) = o0;
            *reinterpret_cast<uint4*>(B + lane * 32 + 16) = o1;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stores, for the bulk copy
            __syncwarp();
            if (lane == 0) {
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], 1024;" ::"l"(out + (pidx - lane) * 16),
                             "r"(saddr(B))
                             : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
            ++nemit;
        };
        unsigned cnt[2] = {0, 0};
        for (int t0 = blockIdx.x; t0 < ntiles && ok; t0 += SH::NWIN * G) {
            const int nt = SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1;
            for (int p = 0; p < nz && ok; ++p) {
                for (int w = 0; w < nt; ++w) {
                    const int tile = t0 + w * G;
                    const int x0 = (tile % tiles_x) * TCX, y0 = (tile / tiles_x) * TR;
                    // the warp agrees on the bounded wait's outcome, so that it leaves or goes on as one
                    if (!__all_sync(0xffffffffu, ws_wait(saddr(&accf[w]), cnt[w] & 1, &abort))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    if (p < nz - 1) {
                        // output plane p-1 is complete: drain it from every row of the thread and zero
                        // its block, so that the tile's next MMAs may accumulate there; hand the window
                        // back before the (slower) output stores
                        uint4 oa[SH::RPT][2];
#pragma unroll
                        for (int rr = 0; rr < SH::RPT; ++rr) {
                            if (p >= 1) {
                                float v[16];
                                load16(w, (p - 1) % 3, erow + SH::ERW * rr, v);
                                pack(v, oa[rr][0], oa[rr][1]);
                            }
                            zero_block(w, (p + 2) % 3, erow + SH::ERW * rr);
                            if (SPLIT || rr == SH::RPT - 1) {  // rows handed back by groups (see the MMA thread)
                                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                                asm volatile("tcgen05.fence::before_thread_sync;");
                                __syncwarp();
                                if (lane == 0) mbar_arrive(saddr(&acce[SPLIT ? rr : w]));
                            }
                        }
                        if (p >= 1)
#pragma unroll
                            for (int rr = 0; rr < SH::RPT; ++rr) emit(p - 1, x0, y0, erow + SH::ERW * rr, oa[rr][0], oa[rr][1]);
                    } else {
                        // the tile's last plane: output planes p-1 and nz-1, then the whole window zeroed
                        // (including the block of the plane beyond the end)
#pragma unroll
                        for (int rr = 0; rr < SH::RPT; ++rr) {
                            const int row = erow + SH::ERW * rr;
                            float va[16], vb[16];
                            uint4 a0, a1, b0, b1;
                            if (p >= 1) {
                                load16(w, (p - 1) % 3, row, va);
                                pack(va, a0, a1);
                            }
                            load16(w, (nz - 1) % 3, row, vb);
                            pack(vb, b0, b1);
                            zero_block(w, 0, row);
                            zero_block(w, 1, row);
                            zero_block(w, 2, row);
                            if (p >= 1) emit(p - 1, x0, y0, row, a0, a1);
                            emit(nz - 1, x0, y0, row, b0, b1);
                        }
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(saddr(&acce[w]));
                            if (SPLIT) mbar_arrive(saddr(&acce[1]));
                        }
                    }
                    ++cnt[w];
                }
            }
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the output has been written
    }
    if (!ok) {
        abort = 1;
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(SH::TMEM_COLS));
}

// Blocks of a kernel that fit on one SM by its registers, shared memory and thread slots (the
// occupancy query answers one for the tensor-memory kernels here where a launch holds two), capped
// by the tensor memory: 512 columns per SM, and tcgen05.alloc of a block beyond them would wait.
static int blocks_per_sm(const void* fn, int nt, int smem, int tmem_cols) {
    int dev = 0, regs_sm = 0, smem_sm = 0, resv = 0, thr_sm = 0;
    cudaGetDevice(&dev);
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, fn);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int warps = (nt + 31) / 32, regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int k = regs_sm / (warps * regs_warp);
    const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + resv), by_thr = thr_sm / nt;
    if (by_smem < k) k = by_smem;
    if (by_thr < k) k = by_thr;
    if (k > 512 / tmem_cols) k = 512 / tmem_cols;
    return k < 1 ? 1 : k;
}

template <int TR, bool FIRST = false>
static int conv16_roll_grid(int nx, int ny) {
    typedef RlShape<TR, FIRST> SH;
    static int nsm = 0, per_sm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const void* fr = (const void*)k_conv16_roll<EPI_RELU, TR, FIRST>;
        cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM);
        cudaFuncSetAttribute(fr, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        per_sm = blocks_per_sm(fr, SH::NT, SH::SMEM, SH::TMEM_COLS);
        if constexpr (!FIRST) {  // the masked variant (backward pass) shares the grid
            const void* fm = (const void*)k_conv16_roll<EPI_MASK, TR, FIRST>;
            cudaFuncSetAttribute(fm, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM);
            cudaFuncSetAttribute(fm, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            const int b = blocks_per_sm(fm, SH::NT, SH::SMEM, SH::TMEM_COLS);
            if (b < per_sm) per_sm = b;
        }
    }
    const int ntiles = (nx / TCX) * (ny / TR), nb = per_sm * nsm;
    return nb < ntiles ? nb : ntiles;
}

// one 16 -> 16 layer: the rolling-plane tcgen05 kernel when nx is a multiple of 128 (tiles of eight
// rows where they give every SM one, else four, two where ny % 4 == 2), else the mma.sync one
static int sm_count() {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    return nsm;
}

template <int EPI>
static void conv16(const NNBufs& b, const __nv_bfloat16* in, const __nv_bfloat16* W, const float* bias,
                   const __nv_bfloat16* mask, __nv_bfloat16* out, int nx, int ny, int nz, cudaStream_t s) {
    const int nsm = sm_count();
    if (nx % TCX == 0 && ny % 2 == 0 && (size_t)nx * ny * 16 < ((size_t)1 << 32)) {
        // 8-row tiles (fewer MMAs per row, one window) where they still give every SM a tile
        if (ny % 8 == 0 && (nx / TCX) * (ny / 8) >= nsm)
            k_conv16_roll<EPI, 8><<<conv16_roll_grid<8>(nx, ny), RlShape<8>::NT, RlShape<8>::SMEM, s>>>(
                in, W, bias, mask, out, nx, ny, nz, b.err);
        else if (ny % 4 == 0)
            k_conv16_roll<EPI, 4><<<conv16_roll_grid<4>(nx, ny), RlShape<4>::NT, RlShape<4>::SMEM, s>>>(
                in, W, bias, mask, out, nx, ny, nz, b.err);
        else
            k_conv16_roll<EPI, 2><<<conv16_roll_grid<2>(nx, ny), RlShape<2>::NT, RlShape<2>::SMEM, s>>>(
                in, W, bias, mask, out, nx, ny, nz, b.err);
    } else {
        const size_t smemz = W_BYTES + 4 * PLANE_BYTES;
        k_conv16z<EPI, CONV_MT><<<conv16z_grid(nx, ny), 256 / CONV_MT, smemz, s>>>(in, W, bias, mask, out, nx, ny, nz);
    }
    note_launch();
}

// ---------------------------------------------------------------- thin layers, marching in z
// The one-channel first layer (1 -> 16) and the weight gradients of the first and last layers in
// the persistent z-marching form of k_conv16z: a block of 128 threads owns a 64 x 2 tile, one cell
// per thread, keeps the input planes k-1, k, k+1 (one-cell halo) in a 4-slot ring and the weights
// in shared memory as FP32, so every input value is read from memory once per tile and the weight
// reads are shared-memory broadcasts. (The two-channel first layer and the last layer run on the
// tensor cores: k_first_tc2, k_last_proj.)
static constexpr int TCELLS = TXC * TYC;  // 128 cells per tile plane

// thin input (C = 1 or 2 channels, bf16): plane kk of the tile into ring slot (kk + 1) & 3
template <int C>
__device__ __forceinline__ void load_thin(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* ring, int nx, int ny,
                                          int nz, int x0, int y0, int kk) {
    __nv_bfloat16* P = ring + ((kk + 1) & 3) * (PLANE_CELLS * C);
    for (int q = threadIdx.x; q < PLANE_CELLS; q += blockDim.x) {
        const int xx = q % HX, yy = q / HX;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (kk >= 0 && kk < nz) {
                const int i = nwrap(x0 - 1 + xx, nx), j = nwrap(y0 - 1 + yy, ny);
                v = in[(((size_t)kk * ny + j) * nx + i) * C + c];
            }
            P[q * C + c] = v;
        }
    }
}
// 16-channel input: plane kk into slot (kk + 1) & 3 with 16-byte cp.async (zeros beyond the ends)
__device__ __forceinline__ void load_wide(const __nv_bfloat16* __restrict__ in, unsigned char* ring, int nx, int ny,
                                          int nz, int x0, int y0, int kk) {
    unsigned char* P = ring + ((kk + 1) & 3) * PLANE_BYTES;
    for (int q = threadIdx.x; q < PLANE_CELLS * 2; q += blockDim.x) {
        const int v = q >> 1, half = q & 1;
        const int xx = v % HX, yy = v / HX;
        if (kk >= 0 && kk < nz) {
            const int i = nwrap(x0 - 1 + xx, nx), j = nwrap(y0 - 1 + yy, ny);
            cp16(P + swz(v, half), in + (((size_t)kk * ny + j) * nx + i) * 16 + half * 8);
        } else {
            *reinterpret_cast<uint4*>(P + swz(v, half)) = make_uint4(0, 0, 0, 0);
        }
    }
    cp_commit_nn();
}

static int thin_grid(int nx, int ny, int cap) {
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (nx / TXC) * (ny / TYC);
    int nb = nsm * 8;
    if (nb > cap) nb = cap;
    return nb < ntiles ? nb : ntiles;
}

// a1 = relu(conv(x, W1) + b1); W1 (bf16, [co][ci][tap]) held as FP32 [tap][ci][co]
template <int CIN>
__global__ void __launch_bounds__(128) k_first_z(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                 const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                 int nx, int ny, int nz) {
    __shared__ __align__(16) float w[27 * CIN * 16];
    __shared__ __align__(16) __nv_bfloat16 ring[4 * PLANE_CELLS * CIN];
    const int tid = threadIdx.x;
    for (int q = tid; q < 16 * CIN * 27; q += blockDim.x) {
        const int co = q / (CIN * 27), ci = (q / 27) % CIN, tap = q % 27;
        w[(tap * CIN + ci) * 16 + co] = __bfloat162float(W[q]);
    }
    float bs[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) bs[co] = __ldg(bias + co);
    const int tiles_x = nx / TXC, ntiles = tiles_x * (ny / TYC);
    const int cx = tid % TXC, cy = tid / TXC;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TXC, y0 = (tile / tiles_x) * TYC;
        __syncthreads();
        load_thin<CIN>(in, ring, nx, ny, nz, x0, y0, -1);
        load_thin<CIN>(in, ring, nx, ny, nz, x0, y0, 0);
        for (int k = 0; k < nz; ++k) {
            load_thin<CIN>(in, ring, nx, ny, nz, x0, y0, k + 1);
            __syncthreads();
            float acc[16];
#pragma unroll
            for (int co = 0; co < 16; ++co) acc[co] = bs[co];
#pragma unroll 1
            for (int dz = 0; dz < 3; ++dz) {
                const __nv_bfloat16* P = ring + ((k + dz) & 3) * (PLANE_CELLS * CIN);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int tap = (dz * 3 + dy) * 3 + dx;
                        const int cell = (cy + dy) * HX + cx + dx;
#pragma unroll
                        for (int ci = 0; ci < CIN; ++ci) {
                            const float xv = __bfloat162float(P[cell * CIN + ci]);
                            const float4* wv = reinterpret_cast<const float4*>(w + (tap * CIN + ci) * 16);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float4 ww = wv[q];
                                acc[4 * q] = fmaf(ww.x, xv, acc[4 * q]);
                                acc[4 * q + 1] = fmaf(ww.y, xv, acc[4 * q + 1]);
                                acc[4 * q + 2] = fmaf(ww.z, xv, acc[4 * q + 2]);
                                acc[4 * q + 3] = fmaf(ww.w, xv, acc[4 * q + 3]);
                            }
                        }
                    }
            }
            __align__(16) __nv_bfloat16 o[16];
#pragma unroll
            for (int co = 0; co < 16; ++co) o[co] = __float2bfloat16_rn(fmaxf(acc[co], 0.f));
            const size_t p = ((size_t)k * ny + y0 + cy) * nx + x0 + cx;
            reinterpret_cast<uint4*>(out + p * 16)[0] = reinterpret_cast<uint4*>(o)[0];
            reinterpret_cast<uint4*>(out + p * 16)[1] = reinterpret_cast<uint4*>(o)[1];
            __syncthreads();  // the slot of plane k-1 is refilled next
        }
    }
}

// ---------------------------------------------------------------- thin layers on the tensor cores
// First layer (2 -> 16) as one implicit GEMM per 16 cells: K = 27 taps x 2 channels, padded to 64
// (4 k16 blocks of 8 taps); an A fragment register holds the 2 channels of one cell and tap (one
// 32-bit shared load), the B fragments (the weights) stay in registers for the whole kernel. The
// input planes arrive through a 6-slot cp.async ring (planes k+2 .. k+4 in flight while plane k is
// computed; planes beyond the z ends are zeros), and the output tile is staged in shared memory, so
// it leaves in coalesced 16-byte stores instead of 4-byte pieces of 32-byte cells.
static constexpr int FP_SLOTS = 6;
static constexpr int FP_PLANE = PLANE_CELLS * 2;  // bf16 values of one halo plane (2 channels)
__global__ void __launch_bounds__(128) k_first_tc2(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ bias, __nv_bfloat16* __restrict__ out, int nx,
                                                   int ny, int nz) {
    __shared__ __align__(16) __nv_bfloat16 ring[FP_SLOTS * FP_PLANE];
    __shared__ __align__(16) __nv_bfloat16 stage[TCELLS * 16];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3, t2 = 2 * t;
    // B fragments: k = 2 j + ci within block kb <-> tap 8 kb + j; column n = output channel
    uint32_t bf[4][2][2];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int tap = 8 * kb + t + 4 * r, co = g + 8 * nt;
                __nv_bfloat162 v = __floats2bfloat162_rn(0.f, 0.f);
                if (tap < 27) {
                    v.x = W[(co * 2 + 0) * 27 + tap];
                    v.y = W[(co * 2 + 1) * 27 + tap];
                }
                bf[kb][nt][r] = *reinterpret_cast<uint32_t*>(&v);
            }
    const float bc0 = __ldg(bias + t2), bc1 = __ldg(bias + t2 + 1), bc8 = __ldg(bias + t2 + 8), bc9 = __ldg(bias + t2 + 9);
    const int tiles_x = nx / TXC, ntiles = tiles_x * (ny / TYC);
    const int yw = warp >> 1, xw = (warp & 1) * 32;
    // plane kk (-1 <= kk) of the tile's halo into slot (kk + 1) % FP_SLOTS, one group per plane
    auto issue = [&](int x0, int y0, int kk) {
        __nv_bfloat16* P = ring + ((kk + 1) % FP_SLOTS) * FP_PLANE;
        for (int q = tid; q < PLANE_CELLS; q += 128) {
            if (kk >= 0 && kk < nz) {
                const int i = nwrap(x0 - 1 + q % HX, nx), j = nwrap(y0 - 1 + q / HX, ny);
                cp4nn(P + 2 * q, in + (((size_t)kk * ny + j) * nx + i) * 2);
            } else {
                *reinterpret_cast<uint32_t*>(P + 2 * q) = 0u;
            }
        }
        cp_commit_nn();
    };
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TXC, y0 = (tile / tiles_x) * TYC;
        __syncthreads();  // the previous tile's ring and output stage are no longer read
        for (int kk = -1; kk <= 3; ++kk) issue(x0, y0, kk);
        for (int k = 0; k < nz; ++k) {
            issue(x0, y0, k + 4);
            cp_wait_nn<3>();  // planes k-1, k, k+1 have landed
            __syncthreads();
            float c[2][2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) c[m][nt][e] = 0.f;
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                uint32_t a[2][4];
#pragma unroll
                for (int r = 0; r < 2; ++r) {  // r = 0: taps 8 kb + t, r = 1: taps 8 kb + t + 4
                    const int tap = 8 * kb + t + 4 * r;
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                    const uint32_t* P = reinterpret_cast<const uint32_t*>(ring + ((k + dz) % FP_SLOTS) * FP_PLANE);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const int cell = (yw + dy) * HX + xw + 16 * m + g + dx;
                        a[m][2 * r] = tap < 27 ? P[cell] : 0u;
                        a[m][2 * r + 1] = tap < 27 ? P[cell + 8] : 0u;
                    }
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    mma16816(c[m][0], a[m][0], a[m][1], a[m][2], a[m][3], bf[kb][0][0], bf[kb][0][1]);
                    mma16816(c[m][1], a[m][0], a[m][1], a[m][2], a[m][3], bf[kb][1][0], bf[kb][1][1]);
                }
            }
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cell = yw * TXC + xw + 16 * m + g + 8 * h;
                    *reinterpret_cast<__nv_bfloat162*>(stage + cell * 16 + t2) =
                        __floats2bfloat162_rn(fmaxf(c[m][0][2 * h] + bc0, 0.f), fmaxf(c[m][0][2 * h + 1] + bc1, 0.f));
                    *reinterpret_cast<__nv_bfloat162*>(stage + cell * 16 + t2 + 8) =
                        __floats2bfloat162_rn(fmaxf(c[m][1][2 * h] + bc8, 0.f), fmaxf(c[m][1][2 * h + 1] + bc9, 0.f));
                }
            __syncthreads();  // the output tile is staged; the ring's planes k-1 .. k+1 are read
            for (int q = tid; q < TCELLS * 2; q += 128) {
                const int cell = q >> 1, half = q & 1;
                const size_t p = ((size_t)k * ny + y0 + cell / TXC) * nx + x0 + cell % TXC;
                *reinterpret_cast<uint4*>(out + p * 16 + half * 8) = *reinterpret_cast<const uint4*>(stage + cell * 16 + half * 8);
            }
        }
        cp_wait_nn<0>();
    }
}

// Last layer (16 -> 1) by in-plane tap projections: out[v] = b + sum over (dy, dx) of
// Q_{dy,dx}[v + (dy-1, dx-1)] with Q_{dy,dx}[c] = sum over dz and ci of W4[ci][dz,dy,dx] a_{k-1+dz}[c][ci].
// Per output plane k one small GEMM on the tensor cores forms Q for every cell of the tile's 66 x 4
// halo (M = 16 cells, K = 48: the three planes k-1 .. k+1 x 16 channels, N = the 9 in-plane taps
// padded to 16); Q goes to shared memory tap-major and each thread sums its cell's 9 shifted
// values. Against one MMA per tap with a single non-zero B column (the earlier form) this is 102
// instead of 216 MMAs per plane of a 128-cell tile, with 9 shared stores and loads per cell; the
// activation planes arrive through a 5-slot cp.async ring (planes beyond the z ends are zeros).
static constexpr int LP_CELLS = 272;  // 66 x 4 halo cells padded to 17 m16 tiles
static constexpr int LP_PS = 276;     // tap-row stride of Q (conflict-free stores and gathers)
static constexpr int LP_SLOTS = 5;    // planes k-1 .. k+1 read, k+2 and k+3 in flight
static constexpr size_t LP_SMEM = (size_t)LP_SLOTS * LP_CELLS * 32 + (size_t)9 * LP_PS * 4;

__global__ void __launch_bounds__(128) k_last_proj(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ bias, float* __restrict__ out, int nx,
                                                   int ny, int nz) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* ring = smem;
    float* Q = reinterpret_cast<float*>(smem + (size_t)LP_SLOTS * LP_CELLS * 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    // B fragments of W4 for k-block dz (16 channels) and n-tile nt: column n = dy*3 + dx (< 9)
    uint32_t bf[3][2][2];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int n = g + 8 * nt, tap = dz * 9 + n;
            __nv_bfloat162 b0 = __floats2bfloat162_rn(0.f, 0.f), b1 = b0;
            if (n < 9) {
                b0.x = W[t2 * 27 + tap];
                b0.y = W[(t2 + 1) * 27 + tap];
                b1.x = W[(t2 + 8) * 27 + tap];
                b1.y = W[(t2 + 9) * 27 + tap];
            }
            bf[dz][nt][0] = *reinterpret_cast<uint32_t*>(&b0);
            bf[dz][nt][1] = *reinterpret_cast<uint32_t*>(&b1);
        }
    const float b4 = __ldg(bias);
    const int tiles_x = nx / TXC, ntiles = tiles_x * (ny / TYC);
    const int tx = tid & 63, ty = tid >> 6;  // this thread's output cell of the 64 x 2 tile
    const int ar = lane & 15, ah = lane >> 4;
    // plane kk (-1 <= kk) of the tile's halo into ring slot (kk + 1) % LP_SLOTS: 16-byte halves of the
    // swizzled cell rows by cp.async, zeros beyond the z ends; one group per plane
    auto issue = [&](int x0, int y0, int kk) {
        unsigned char* S = ring + ((kk + 1) % LP_SLOTS) * (LP_CELLS * 32);
        for (int q = tid; q < PLANE_CELLS * 2; q += 128) {
            const int v = q >> 1, half = q & 1;
            if (kk >= 0 && kk < nz) {
                const int i = nwrap(x0 - 1 + v % HX, nx), j = nwrap(y0 - 1 + v / HX, ny);
                cp16(S + swz(v, half), in + (((size_t)kk * ny + j) * nx + i) * 16 + half * 8);
            } else {
                *reinterpret_cast<uint4*>(S + swz(v, half)) = make_uint4(0, 0, 0, 0);
            }
        }
        cp_commit_nn();
    };
    const size_t pl = (size_t)nx * ny;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TXC, y0 = (tile / tiles_x) * TYC;
        __syncthreads();  // the previous tile's ring and projections are no longer read
        for (int kk = -1; kk <= LP_SLOTS - 3; ++kk) issue(x0, y0, kk);
        const size_t orow = (size_t)(y0 + ty) * nx + x0 + tx;
        for (int k = 0; k < nz; ++k) {
            issue(x0, y0, k + LP_SLOTS - 2);
            cp_wait_nn<LP_SLOTS - 3>();  // planes k-1, k, k+1 have landed
            __syncthreads();             // ... for every thread; the last gather is done
            for (int mt = warp; mt < LP_CELLS / 16; mt += 4) {
                float c[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
                for (int dz = 0; dz < 3; ++dz) {  // plane k-1+dz sits in slot (k + dz) % LP_SLOTS
                    const unsigned char* S = ring + ((k + dz) % LP_SLOTS) * (LP_CELLS * 32);
                    uint32_t a0, a1, a2, a3;
                    ldm_x4(saddr(S + swz(mt * 16 + ar, ah)), a0, a1, a2, a3);
                    mma16816(c[0], a0, a1, a2, a3, bf[dz][0][0], bf[dz][0][1]);
                    mma16816(c[1], a0, a1, a2, a3, bf[dz][1][0], bf[dz][1][1]);
                }
                const int cell = mt * 16 + g;
                // n-tile 0 holds taps t2, t2+1; n-tile 1 tap 8 + t2 (only tap 8 is used)
                Q[t2 * LP_PS + cell] = c[0][0];
                Q[t2 * LP_PS + cell + 8] = c[0][2];
                Q[(t2 + 1) * LP_PS + cell] = c[0][1];
                Q[(t2 + 1) * LP_PS + cell + 8] = c[0][3];
                if (t2 == 0) {
                    Q[8 * LP_PS + cell] = c[1][0];
                    Q[8 * LP_PS + cell + 8] = c[1][2];
                }
            }
            __syncthreads();  // the plane's projections are complete
            float s = 0.f;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) s += Q[(dy * 3 + dx) * LP_PS + (ty + dy) * HX + tx + dx];
            out[(size_t)k * pl + orow] = s + b4;
        }
        cp_wait_nn<0>();
    }
}

// ---------------------------------------------------------------- last layer (16 -> 1) on tcgen05
// The rolling scheme of k_conv16_roll for one output channel: the view (input plane p, halo row h,
// shift dx) feeds rows h-2 .. h of output planes p+1, p, p-1, nine single-channel outputs, so one MMA
// of N = 16 (M = 128 cells, K = 16 channels; B columns 9 .. 15 zero) covers them. Each halo row h has
// its own 16 accumulator columns at 16 h (column 3 j + q: tile row h-2+j, residue q = plane mod 3), so
// output row r of a plane sums column 3 j + q of the blocks of rows r+2-j (j = 0, 1, 2). Per input
// plane 3 (TR + 2) MMAs; then output plane p-1 is complete. The epilogue warps (one per lane quarter,
// a thread owns one cell of every tile row) load the whole window of their lanes (all loads in
// flight, one wait), add each row's three columns, zero the drained residue's columns (all after the
// tile's last plane), store it back, hand it back and store the outputs (+ bias) in FP32. With TR = 4
// two windows of 16 (TR + 2) columns take a pair of tiles plane by plane in turn, so the tensor core
// fills one while the epilogue drains the other; with TR = 8 one window, handed back in groups of
// three blocks. Two blocks per SM. Producers and the bounded waits as in k_conv16_roll.
static constexpr int LR_NPROD = 64;
static constexpr int LR_BB = 16 * 32;  // one B matrix: [K half][16 rows][8 ci]
static constexpr int LR_WB = 9 * LR_BB;
static constexpr uint32_t LR_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
template <int TR>
struct LrShape {
    static constexpr int NT = 128 + 32 + LR_NPROD;  // epilogue warps, the MMA warp, the producers
    static constexpr int PLANEB = (TR + 2) * TC_ROWB;
    static constexpr int SLOTS = TR >= 8 ? 2 : 4;   // two blocks share an SM
    static constexpr int SMEM = LR_WB + SLOTS * PLANEB;
    static constexpr int WIN_COLS = 16 * (TR + 2);  // one block of 16 columns per halo row
    // two windows (a pair of tiles in turn) where two blocks per SM still fit the tensor memory
    static constexpr int NWIN = 2 * WIN_COLS <= 256 ? 2 : 1;
    static constexpr int TMEM_COLS = NWIN * WIN_COLS <= 128 ? 128 : 256;
    static_assert(NWIN * WIN_COLS <= TMEM_COLS, "windows");
};

template <int TR>
__global__ void __launch_bounds__(LrShape<TR>::NT, 2) k_last_roll(const __nv_bfloat16* __restrict__ in,
                                                               const __nv_bfloat16* __restrict__ W,
                                                               const float* __restrict__ bias,
                                                               float* __restrict__ out, int nx, int ny, int nz,
                                                               int* err) {
    typedef LrShape<TR> SH;
    extern __shared__ __align__(128) unsigned char smem[];
    // acce: per window, or with one window per group of three drained blocks (SPLIT)
    __shared__ __align__(8) uint64_t full[LrShape<TR>::SLOTS], empty[LrShape<TR>::SLOTS], accf[2], acce[4];
    constexpr int HH = 3, NG = (TR + 2 + HH - 1) / HH;  // the window's blocks in groups of three
    constexpr bool SPLIT = SH::NWIN == 1;
    static_assert(NG <= 4, "handover barriers");
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort;
    unsigned char* Ws = smem;
    unsigned char* ring = smem + LR_WB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // B matrix (rotation rot, shift dx): row n = 3 j + q (n < 9) is tap dy = 2 - j, dz = (rot + 1 - q)
    // mod 3 of W4[ci][tap]; rows 9 .. 15 zero
    for (int e = tid; e < 9 * 16 * 16; e += SH::NT) {
        const int mtx = e / 256, n = (e / 16) % 16, ci = e % 16;
        const int rot = mtx / 3, dx = mtx % 3, j = n / 3, qq = n % 3;
        float w = 0.f;
        if (n < 9) {
            const int dy = 2 - j, dz = (rot + 4 - qq) % 3;
            w = __bfloat162float(W[ci * 27 + (dz * 3 + dy) * 3 + dx]);
        }
        *reinterpret_cast<__nv_bfloat16*>(Ws + mtx * LR_BB + (ci >> 3) * (LR_BB / 2) + n * 16 + (ci & 7) * 2) =
            __float2bfloat16_rn(w);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "n"(SH::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < SH::SLOTS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[s])), "n"(LR_NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])));
        }
        for (int w = 0; w < 2; ++w) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&accf[w])));
        for (int g = 0; g < 4; ++g) asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(saddr(&acce[g])));
        abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const float b4 = __ldg(bias);
    const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // an epilogue warp's lane quarter
    auto ld16 = [&](int blk, uint32_t (&r)[16]) {  // the caller waits (tcgen05.wait::ld) before use
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tlane + 16 * blk));
    };
    auto st16 = [&](int blk, const uint32_t (&r)[16]) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                tlane + 16 * blk),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
            "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
            : "memory");
    };
    if (tid < 128) {  // the windows start at zero
        uint32_t z[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) z[c] = 0;
#pragma unroll
        for (int h = 0; h < SH::NWIN * (TR + 2); ++h) st16(h, z);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int tiles_x = nx / TCX, ntiles = tiles_x * (ny / TR);
    const int G = (int)gridDim.x;
    bool ok = true;
    // tiles in pairs (t, t + G) as in k_conv16_roll: while the epilogue drains one tile's window the
    // tensor core accumulates into the other's
    if (tid >= 128 + 32) {
        // ---- producers: the pair's planes in turn into slot q % SLOTS of the ring
        const int ptid = tid - (128 + 32);
        constexpr int NCH = (TR + 2) * TC_ROWC * 2, CPT = (NCH + LR_NPROD - 1) / LR_NPROD;
        int ch_dst[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int qq = ptid + LR_NPROD * c;
            ch_dst[c] = qq < NCH ? ((qq >> 1) / TC_ROWC) * TC_ROWB + (qq & 1) * TC_HALF + ((qq >> 1) % TC_ROWC) * 16 : -1;
        }
        int q = 0;
        for (int t0 = blockIdx.x; t0 < ntiles && ok; t0 += SH::NWIN * G) {
            const int nt = SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1;
            uint32_t src[SH::NWIN][CPT];  // element offsets within a plane (the caller keeps a plane below 2^32)
#pragma unroll
            for (int w = 0; w < SH::NWIN; ++w) {
                const int tile = w < nt ? t0 + w * G : t0;
                const int x0 = (tile % tiles_x) * TCX, y0 = (tile / tiles_x) * TR;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int qq = ptid + LR_NPROD * c;
                    const int hh = qq & 1, cc = (qq >> 1) % TC_ROWC, rr = (qq >> 1) / TC_ROWC;
                    src[w][c] = ((uint32_t)nwrap(y0 - 1 + rr, ny) * nx + nwrap(x0 - 1 + cc, nx)) * 16 + hh * 8;
                }
            }
            for (int p = 0; p < nz && ok; ++p) {
                for (int w = 0; w < nt; ++w, ++q) {
                    const int slot = q % SH::SLOTS;
                    if (q >= SH::SLOTS && !ws_wait(saddr(&empty[slot]), ((q / SH::SLOTS) - 1) & 1, &abort)) {
                        ok = false;
                        break;
                    }
                    unsigned char* P = ring + slot * SH::PLANEB;
                    const __nv_bfloat16* base = in + (size_t)p * ny * nx * 16;
#pragma unroll
                    for (int c = 0; c < CPT; ++c)
                        if (ch_dst[c] >= 0) cp16(P + ch_dst[c], base + src[w][c]);
                    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(&full[slot]))
                                 : "memory");
                }
            }
        }
        cp_wait_nn<0>();
    } else if (warp == 4) {
        // ---- MMA thread: one step per input plane of a tile, into that tile's window
        if (lane == 0) {
            const uint64_t dw0 = tc_desc(saddr(Ws), LR_BB / 2, 128);
            unsigned s = 0, cnt[2] = {0, 0};
            for (int t0 = blockIdx.x; t0 < ntiles && ok; t0 += SH::NWIN * G) {
                const int nt = SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1;
                for (int p = 0; p < nz && ok; ++p) {
                    for (int w = 0; w < nt; ++w, ++s) {
                        const int slot = s % SH::SLOTS;
                        if (!ws_wait(saddr(&full[slot]), (s / SH::SLOTS) & 1, &abort) ||
                            (cnt[w] >= 1 && !ws_wait(saddr(&acce[w]), (cnt[w] - 1) & 1, &abort))) {
                            ok = false;
                            break;
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint64_t dp = tc_desc(saddr(ring + slot * SH::PLANEB), TC_HALF, 128);
                        const uint32_t win = tmem + w * SH::WIN_COLS;
                        const int rot = p % 3;
                        // the views of halo rows hlo .. hhi-1 (block h of the window each)
                        auto views = [&](int hlo, int hhi) {
#pragma unroll
                            for (int h = hlo; h < hhi; ++h)
#pragma unroll
                                for (int dx = 0; dx < 3; ++dx) {
                                    const uint64_t db = dw0 + (uint64_t)(((rot * 3 + dx) * LR_BB) >> 4);
                                    const uint64_t da = dp + (uint64_t)(((h * TC_ROWB) + dx * 16) >> 4);
                                    asm volatile(
                                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(win + 16 * h),
                                        "l"(da), "l"(db), "r"(LR_IDESC), "r"(1));
                                }
                        };
                        if constexpr (SPLIT) {  // each group of blocks as soon as the epilogue has zeroed it
                            views(0, HH);  // group 0 (acce[0], waited above)
                            bool okg = true;
#pragma unroll
                            for (int g = 1; g < NG; ++g) {
                                if (okg && cnt[w] >= 1 && !ws_wait(saddr(&acce[g]), (cnt[w] - 1) & 1, &abort)) okg = false;
                                if (!okg) break;
                                asm volatile("tcgen05.fence::after_thread_sync;");
                                views(g * HH, (g + 1) * HH < TR + 2 ? (g + 1) * HH : TR + 2);
                            }
                            if (!okg) {
                                tc_commit(saddr(&accf[w]));  // the final wait covers the MMAs issued
                                ++cnt[w];
                                ok = false;
                                break;
                            }
                        } else {
                            views(0, TR + 2);
                        }
                        tc_commit(saddr(&accf[w]));
                        tc_commit(saddr(&empty[slot]));
                        ++cnt[w];
                    }
                }
            }
            for (int w = 0; w < 2; ++w)
                if (cnt[w] > 0) tc_wait(saddr(&accf[w]), (cnt[w] - 1) & 1);
        }
    } else {
        // ---- epilogue warps 0 .. 3: the thread owns cell `cell` of every tile row
        const int cell = (warp & 3) * 32 + lane;
        unsigned cnt[2] = {0, 0};
        for (int t0 = blockIdx.x; t0 < ntiles && ok; t0 += SH::NWIN * G) {
            const int nt = SH::NWIN == 2 && t0 + G < ntiles ? 2 : 1;
            for (int p = 0; p < nz && ok; ++p) {
                for (int w = 0; w < nt; ++w) {
                    const int tile = t0 + w * G;
                    const int x0 = (tile % tiles_x) * TCX, y0 = (tile / tiles_x) * TR;
                    // the warp agrees on the bounded wait's outcome, so that it leaves or goes on as one
                    if (!__all_sync(0xffffffffu, ws_wait(saddr(&accf[w]), cnt[w] & 1, &abort))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const bool last = p == nz - 1;
                    const int qa = (p + 2) % 3;   // residue of output plane p-1: drained (p >= 1) and zeroed
                    const int qb = (nz - 1) % 3;  // residue of output plane nz-1, drained after the last plane
                    float oa[TR], ob[TR];
#pragma unroll
                    for (int r = 0; r < TR; ++r) oa[r] = ob[r] = 0.f;
                    // the window of this lane in groups of three blocks, each group's loads in flight at once;
                    // with one window each group is handed back once zeroed
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                    uint32_t vv[HH][16];
#pragma unroll
                    for (int i = 0; i < HH; ++i)
                        if (g * HH + i < TR + 2) ld16(w * (TR + 2) + g * HH + i, vv[i]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int i = 0; i < HH; ++i) {
                        const int h = g * HH + i;
                        if (h >= TR + 2) continue;
                        uint32_t (&v)[16] = vv[i];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const int r = h - 2 + j;
                            if (r < 0 || r >= TR) continue;
                            const float a0 = __uint_as_float(v[3 * j]), a1 = __uint_as_float(v[3 * j + 1]),
                                        a2 = __uint_as_float(v[3 * j + 2]);
                            oa[r] += qa == 0 ? a0 : (qa == 1 ? a1 : a2);
                            ob[r] += qb == 0 ? a0 : (qb == 1 ? a1 : a2);
                        }
#pragma unroll
                        for (int c = 0; c < 9; ++c)
                            if (last || c % 3 == qa) v[c] = 0;
                        st16(w * (TR + 2) + h, v);
                    }
                    if (SPLIT || g == NG - 1) {
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(saddr(&acce[SPLIT ? g : w]));
                    }
                    }
#pragma unroll
                    for (int r = 0; r < TR; ++r) {
                        const size_t row = (size_t)(y0 + r) * nx + x0 + cell;
                        if (p >= 1) out[(size_t)(p - 1) * nx * ny + row] = oa[r] + b4;
                        if (last) out[(size_t)(nz - 1) * nx * ny + row] = ob[r] + b4;
                    }
                    ++cnt[w];
                }
            }
        }
    }
    if (!ok) {
        abort = 1;
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(SH::TMEM_COLS));
}

template <int TR>
static int last_roll_grid(int nx, int ny) {
    typedef LrShape<TR> SH;
    static int per_sm = 0, nsm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_last_roll<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM);
        cudaFuncSetAttribute(k_last_roll<TR>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        per_sm = blocks_per_sm((const void*)k_last_roll<TR>, SH::NT, SH::SMEM, SH::TMEM_COLS);
    }
    const int ntiles = (nx / TCX) * (ny / TR);
    const int nb = per_sm * nsm;
    return nb < ntiles ? nb : ntiles;
}

// partial weight gradient of the first layer: dW1[co][ci][tap] = sum_p d1[p][co] x[p + d(tap)][ci].
// Thread t < 27 CIN G owns one (ci, tap) for all 16 co over the cells of group t / (27 CIN)
// (G = 108 / (27 CIN) groups of the 128 tile cells); one partial per block and weight.
template <int CIN>
__global__ void __launch_bounds__(128) k_dwfirst_z(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
                                                   float* __restrict__ partials, int nx, int ny, int nz) {
    constexpr int NPAIR = 27 * CIN, G = 108 / NPAIR, CPG = TCELLS / G;
    __shared__ __align__(16) __nv_bfloat16 ring[4 * PLANE_CELLS * CIN];
    __shared__ __align__(16) __nv_bfloat16 dys[TCELLS * 16];
    const int tid = threadIdx.x;
    const bool act = tid < NPAIR * G;
    const int pair = tid % NPAIR, grp = tid / NPAIR;
    const int ci = pair % CIN, tap = pair / CIN;
    const int dz = tap / 9, dyy = (tap / 3) % 3, dxx = tap % 3;
    float acc[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) acc[co] = 0.f;
    const int tiles_x = nx / TXC, ntiles = tiles_x * (ny / TYC);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TXC, y0 = (tile / tiles_x) * TYC;
        __syncthreads();
        load_thin<CIN>(x, ring, nx, ny, nz, x0, y0, -1);
        load_thin<CIN>(x, ring, nx, ny, nz, x0, y0, 0);
        for (int k = 0; k < nz; ++k) {
            load_thin<CIN>(x, ring, nx, ny, nz, x0, y0, k + 1);
            for (int q = tid; q < TCELLS * 2; q += blockDim.x) {
                const int v = q >> 1, half = q & 1;
                const size_t p = ((size_t)k * ny + y0 + v / TXC) * nx + x0 + v % TXC;
                reinterpret_cast<uint4*>(dys)[q] = __ldg(reinterpret_cast<const uint4*>(dy + p * 16) + half);
            }
            __syncthreads();
            if (act) {
                const __nv_bfloat16* P = ring + ((k + dz) & 3) * (PLANE_CELLS * CIN);
                for (int cc = grp * CPG; cc < (grp + 1) * CPG; ++cc) {
                    const int cx = cc % TXC, cy = cc / TXC;
                    const float xv = __bfloat162float(P[((cy + dyy) * HX + cx + dxx) * CIN + ci]);
                    const uint4* g = reinterpret_cast<const uint4*>(dys + cc * 16);
#pragma unroll
                    for (int hq = 0; hq < 2; ++hq) {
                        const uint4 gv = g[hq];
                        const __nv_bfloat162* gb = reinterpret_cast<const __nv_bfloat162*>(&gv);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 f = __bfloat1622float2(gb[e]);
                            acc[8 * hq + 2 * e] = fmaf(f.x, xv, acc[8 * hq + 2 * e]);
                            acc[8 * hq + 2 * e + 1] = fmaf(f.y, xv, acc[8 * hq + 2 * e + 1]);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    // the groups of one (ci, tap) add up in shared memory, in group order
    __shared__ float red[108 * 16];
    if (act)
#pragma unroll
        for (int co = 0; co < 16; ++co) red[tid * 16 + co] = acc[co];
    __syncthreads();
    if (tid < NPAIR) {
        float* dst = partials + (size_t)blockIdx.x * (16 * CIN * 27);
        for (int co = 0; co < 16; ++co) {
            float sm = 0.f;
            for (int gq = 0; gq < G; ++gq) sm += red[(gq * NPAIR + tid) * 16 + co];
            dst[(co * CIN + ci) * 27 + tap] = sm;
        }
    }
}

// partial weight gradient of the last layer: dW4[ci][tap] = sum_p d4[p] a3[p + d(tap)][ci];
// thread t < 108 owns tap t % 27 for all 16 ci over the cells of group t / 27 (4 groups)
__global__ void __launch_bounds__(128) k_dwlast_z(const __nv_bfloat16* __restrict__ a3, const float* __restrict__ d4,
                                                  float* __restrict__ partials, int nx, int ny, int nz) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* ring = smem;
    float* ds = reinterpret_cast<float*>(smem + 4 * PLANE_BYTES);
    const int tid = threadIdx.x;
    const bool act = tid < 108;
    const int tap = tid % 27, grp = tid / 27;
    const int dz = tap / 9, dyy = (tap / 3) % 3, dxx = tap % 3;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.f;
    const int tiles_x = nx / TXC, ntiles = tiles_x * (ny / TYC);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TXC, y0 = (tile / tiles_x) * TYC;
        __syncthreads();
        load_wide(a3, ring, nx, ny, nz, x0, y0, -1);
        load_wide(a3, ring, nx, ny, nz, x0, y0, 0);
        load_wide(a3, ring, nx, ny, nz, x0, y0, 1);
        for (int k = 0; k < nz; ++k) {
            load_wide(a3, ring, nx, ny, nz, x0, y0, k + 2);
            {
                const int v = tid;
                const size_t p = ((size_t)k * ny + y0 + v / TXC) * nx + x0 + v % TXC;
                ds[v] = __ldg(d4 + p);
            }
            cp_wait_nn<1>();
            __syncthreads();
            if (act) {
                const unsigned char* P = ring + ((k + dz) & 3) * PLANE_BYTES;
                for (int cc = grp * 32; cc < grp * 32 + 32; ++cc) {
                    const int cx = cc % TXC, cy = cc / TXC;
                    const float g = ds[cc];
                    const int cell = (cy + dyy) * HX + cx + dxx;
#pragma unroll
                    for (int hq = 0; hq < 2; ++hq) {
                        const uint4 av = *reinterpret_cast<const uint4*>(P + swz(cell, hq));
                        const __nv_bfloat162* ab = reinterpret_cast<const __nv_bfloat162*>(&av);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 f = __bfloat1622float2(ab[e]);
                            acc[8 * hq + 2 * e] = fmaf(g, f.x, acc[8 * hq + 2 * e]);
                            acc[8 * hq + 2 * e + 1] = fmaf(g, f.y, acc[8 * hq + 2 * e + 1]);
                        }
                    }
                }
            }
            __syncthreads();
        }
        cp_wait_nn<0>();
    }
    float* red = reinterpret_cast<float*>(smem);  // the ring is no longer read
    __syncthreads();
    if (act)
#pragma unroll
        for (int c = 0; c < 16; ++c) red[tid * 16 + c] = acc[c];
    __syncthreads();
    if (tid < 27) {
        float* dst = partials + (size_t)blockIdx.x * (16 * 27);
        for (int c = 0; c < 16; ++c) {
            const float sm = (red[tid * 16 + c] + red[(27 + tid) * 16 + c]) + (red[(54 + tid) * 16 + c] + red[(81 + tid) * 16 + c]);
            dst[c * 27 + tid] = sm;
        }
    }
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

// persistent grid of a 128-thread thin-layer kernel over the 64 x 2 tiles: the blocks the SMs hold
// at once (so no block waits for another to finish all its tiles), at most one per tile
template <class K>
static int resident_grid(K kern, size_t smem, int nx, int ny) {
    int nsm = 0, dev = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem);
    if (occ < 1) occ = 1;
    const int ntiles = (nx / TXC) * (ny / TYC);
    const int nb = nsm * occ;
    return nb < ntiles ? nb : ntiles;
}

void nn_forward(const NNBufs& b, int nx, int ny, int nz, const __nv_bfloat16* x, float* out, cudaStream_t s) {
    const size_t n = (size_t)nx * ny * nz;
    const float* b1 = b.params + 16 * b.cin * 27;
    const float* b2 = b1 + 16 + 16 * 16 * 27;
    const float* b3 = b2 + 16 + 16 * 16 * 27;
    const float* b4 = b3 + 16 + 16 * 27;
    const int gt = thin_grid(nx, ny, 1 << 30);
    if (b.cin == 1) k_first_z<1><<<gt, 128, 0, s>>>(x, b.w1, b1, b.a1, nx, ny, nz);
    else if (nx % TCX == 0 && ny % 8 == 0 && (nx / TCX) * (ny / 8) >= sm_count())  // 8-row tiles fill the SMs
        k_conv16_roll<EPI_RELU, 8, true><<<conv16_roll_grid<8, true>(nx, ny), RlShape<8, true>::NT, RlShape<8, true>::SMEM,
                                           s>>>(x, b.w1, b1, nullptr, b.a1, nx, ny, nz, b.err);
    else if (nx % TCX == 0 && ny % 4 == 0)
        k_conv16_roll<EPI_RELU, 4, true><<<conv16_roll_grid<4, true>(nx, ny), RlShape<4, true>::NT, RlShape<4, true>::SMEM,
                                           s>>>(x, b.w1, b1, nullptr, b.a1, nx, ny, nz, b.err);
    else k_first_tc2<<<resident_grid(k_first_tc2, 0, nx, ny), 128, 0, s>>>(x, b.w1, b1, b.a1, nx, ny, nz);
    note_launch();
    conv16<EPI_RELU>(b, b.a1, b.w2f, b2, nullptr, b.a2, nx, ny, nz, s);
    conv16<EPI_RELU>(b, b.a2, b.w3f, b3, nullptr, b.a3, nx, ny, nz, s);
    if (nx % TCX == 0 && ny % 8 == 0 && (size_t)nx * ny * 16 < ((size_t)1 << 32) &&
        (nx / TCX) * (ny / 8) >= 2 * sm_count()) {  // 8-row tiles where they fill two blocks per SM
        k_last_roll<8><<<last_roll_grid<8>(nx, ny), LrShape<8>::NT, LrShape<8>::SMEM, s>>>(b.a3, b.w4, b4, out, nx, ny,
                                                                                        nz, b.err);
    } else if (nx % TCX == 0 && ny % 4 == 0 && (size_t)nx * ny * 16 < ((size_t)1 << 32)) {
        k_last_roll<4><<<last_roll_grid<4>(nx, ny), LrShape<4>::NT, LrShape<4>::SMEM, s>>>(b.a3, b.w4, b4, out, nx, ny,
                                                                                        nz, b.err);
    } else {
        static bool lp_attr = false;
        if (!lp_attr) {
            cudaFuncSetAttribute(k_last_proj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LP_SMEM);
            lp_attr = true;
        }
        k_last_proj<<<resident_grid(k_last_proj, LP_SMEM, nx, ny), 128, LP_SMEM, s>>>(b.a3, b.w4, b4, out, nx, ny, nz);
    }
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
    const int nbt = thin_grid(nx, ny, 1024);  // partial sums of the thin weight gradients
    // layer 4: dW4, db4 and d3 = mask(a3) * W4^T d4
    k_dwlast_z<<<nbt, 128, 4 * PLANE_BYTES + TCELLS * 4, s>>>(b.a3, d4, b.part, nx, ny, nz);
    k_reduce_partials<<<(n4 + 255) / 256, 256, 0, s>>>(b.part, nbt, n4, gW4);
    k_chansum<1, true><<<nb, 256, 0, s>>>(d4, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 1, gb4);
    k_bwd_last<<<blocks_for(n), 256, 0, s>>>(d4, b.w4, b.a3, b.d1, nx, ny, nz);
    for (int q = 0; q < 5; ++q) note_launch();
    const size_t smem_dw = HALO_BYTES + TXC * TYC * 32;
    cudaFuncSetAttribute(k_dw16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dw);
    // layer 3: dW3 from (a2, d3); d2 = mask(a2) * conv(d3, W3 flipped)
    k_dw16<<<nb, 256, smem_dw, s>>>(b.a2, b.d1, b.part, nx, ny, nz);
    k_reduce_partials<<<(n2 + 255) / 256, 256, 0, s>>>(b.part, nb, n2, gW3);
    k_chansum<16, false><<<nb, 256, 0, s>>>(b.d1, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 16, gb3);
    conv16<EPI_MASK>(b, b.d1, b.w3b, nullptr, b.a2, b.d2, nx, ny, nz, s);
    // layer 2: dW2 from (a1, d2); d1 = mask(a1) * conv(d2, W2 flipped)
    k_dw16<<<nb, 256, smem_dw, s>>>(b.a1, b.d2, b.part, nx, ny, nz);
    k_reduce_partials<<<(n2 + 255) / 256, 256, 0, s>>>(b.part, nb, n2, gW2);
    k_chansum<16, false><<<nb, 256, 0, s>>>(b.d2, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 16, gb2);
    conv16<EPI_MASK>(b, b.d2, b.w2b, nullptr, b.a1, b.d1, nx, ny, nz, s);
    // layer 1: dW1 from (x, d1)
    if (cin == 1) k_dwfirst_z<1><<<nbt, 128, 0, s>>>(x, b.d1, b.part, nx, ny, nz);
    else k_dwfirst_z<2><<<nbt, 128, 0, s>>>(x, b.d1, b.part, nx, ny, nz);
    k_reduce_partials<<<(n1 + 255) / 256, 256, 0, s>>>(b.part, nbt, n1, gW1);
    k_chansum<16, false><<<nb, 256, 0, s>>>(b.d1, b.part, n, cpb);
    k_reduce_partials<<<1, 256, 0, s>>>(b.part, nb, 16, gb1);
    for (int q = 0; q < 12; ++q) note_launch();
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
