// FP32 denoiser on CUDA cores (the plain-precision path).
//
// D_eps = Id - G, G = T_K o ... o T_1, T_k(v) = ReLU(W_k v + b_k) (no ReLU on
// the last layer), W_k a 3x3 zero-padded multichannel cross-correlation
// (Sec. II-B, Eqs. 5-6, Example 1). Activations are NCHW FP32 planes of the
// whole image (or of every block-with-halo tile): a tile reads its
// neighbours' pixels straight from the previous layer's plane in HBM, so no
// halo is exchanged or duplicated. Every output is the same fixed-order sum
// (input channel, then tap dy, dx), independent of the tile or launch shape.
//
// Layer kernel: 256 threads compute a 32 x 8 pixel tile for all COUT output
// channels; each thread owns 4 consecutive pixels x COUT/4 channels. Input
// channels stream through shared memory in chunks of 8 with cp.async double
// buffering; weights are read as warp-wide broadcasts.
#include "pnp_internal.h"

namespace pnp {

constexpr int CV_TX = 32, CV_TY = 8, CV_THREADS = 256;
constexpr int CV_PITCH = 40;          // floats per smem row: 3 pad, x = -1 .. 32, pad
constexpr int CV_ROWS = CV_TY + 2;

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int sz = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(sz));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int CIN, int COUT>
struct ConvCfg {
    static constexpr int CHUNK = CIN < 8 ? CIN : 8;
    static constexpr int NCHUNK = CIN / CHUNK;
    static constexpr int CO_T = COUT / 4;
    static constexpr int IN_FLOATS = CHUNK * CV_ROWS * CV_PITCH;
    static constexpr int W_FLOATS = CHUNK * 9 * COUT;
    static constexpr int STAGE_FLOATS = IN_FLOATS + W_FLOATS;
    static constexpr size_t SMEM = sizeof(float) * 2 * STAGE_FLOATS;
};

// Stage chunk `ck` of the input planes (rows y0-1 .. y0+8, cols x0-1 .. x0+32,
// zero outside the image) and of the weights [ci][tap][co].
template <int CIN, int COUT>
__device__ __forceinline__ void stage_chunk(const float* __restrict__ in, const float* __restrict__ w,
                                            int ny, int nx, int y0, int x0, int ck, float* st) {
    using C = ConvCfg<CIN, COUT>;
    const int64_t plane = (int64_t)ny * nx;
    float* sin = st;
    float* sw = st + C::IN_FLOATS;
    constexpr int W_IN = CV_TX + 2;
    for (int e = threadIdx.x; e < C::CHUNK * CV_ROWS * W_IN; e += CV_THREADS) {
        const int c = e / (CV_ROWS * W_IN);
        const int rem = e - c * (CV_ROWS * W_IN);
        const int r = rem / W_IN, v = rem - r * W_IN;
        const int gy = y0 - 1 + r, gx = x0 - 1 + v;
        const bool ok = gy >= 0 && gy < ny && gx >= 0 && gx < nx;
        const float* src = in + (int64_t)(ck * C::CHUNK + c) * plane + (ok ? (int64_t)gy * nx + gx : 0);
        cp_async4(sin + (c * CV_ROWS + r) * CV_PITCH + 3 + v, src, ok);
    }
    const float* wsrc = w + (int64_t)ck * C::CHUNK * 9 * COUT;
    for (int e = threadIdx.x * 4; e < C::W_FLOATS; e += CV_THREADS * 4) cp_async16(sw + e, wsrc + e);
}

template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(CV_THREADS) k_conv3x3(const float* __restrict__ in,
                                                        const float* __restrict__ w,
                                                        const float* __restrict__ bias, int ny,
                                                        int nx, const Rect* __restrict__ rects,
                                                        float* __restrict__ out) {
    using C = ConvCfg<CIN, COUT>;
    extern __shared__ __align__(16) float smem[];
    const int img = blockIdx.z;
    const int64_t plane = (int64_t)ny * nx;
    const float* inb = in + (int64_t)img * CIN * plane;
    float* outb = out + (int64_t)img * COUT * plane;
    const int y0 = blockIdx.y * CV_TY, x0 = blockIdx.x * CV_TX;
    const int pxg = threadIdx.x % 64, cog = threadIdx.x / 64;
    const int ty = pxg / 8, tx4 = (pxg % 8) * 4;

    float acc[4][C::CO_T];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int c = 0; c < C::CO_T; ++c) acc[p][c] = 0.f;

    stage_chunk<CIN, COUT>(inb, w, ny, nx, y0, x0, 0, smem);
    cp_async_commit();
    for (int ck = 0; ck < C::NCHUNK; ++ck) {
        float* cur = smem + (ck & 1) * C::STAGE_FLOATS;
        if (ck + 1 < C::NCHUNK) {
            stage_chunk<CIN, COUT>(inb, w, ny, nx, y0, x0, ck + 1,
                                   smem + ((ck + 1) & 1) * C::STAGE_FLOATS);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float* sin = cur;
        const float* sw = cur + C::IN_FLOATS;
#pragma unroll 1
        for (int c = 0; c < C::CHUNK; ++c) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const float* row = sin + (c * CV_ROWS + ty + dy) * CV_PITCH + tx4 + 3;
                float r[6];
                r[0] = row[0];
                const float4 mid = *reinterpret_cast<const float4*>(row + 1);
                r[1] = mid.x; r[2] = mid.y; r[3] = mid.z; r[4] = mid.w;
                r[5] = row[5];
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float* wr = sw + (c * 9 + dy * 3 + dx) * COUT + cog * C::CO_T;
                    float wv[C::CO_T];
#pragma unroll
                    for (int q = 0; q < C::CO_T; q += 4) {
                        const float4 t = *reinterpret_cast<const float4*>(wr + q);
                        wv[q] = t.x; wv[q + 1] = t.y; wv[q + 2] = t.z; wv[q + 3] = t.w;
                    }
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < C::CO_T; ++q) acc[p][q] = fmaf(r[p + dx], wv[q], acc[p][q]);
                }
            }
        }
        __syncthreads();
    }
    const int y = y0 + ty;
    if (y >= ny) return;
    Rect R = rects ? rects[img] : Rect{0, ny, 0, nx};
    const bool row_ok = y >= R.y0 && y < R.y1;
#pragma unroll
    for (int q = 0; q < C::CO_T; ++q) {
        const int co = cog * C::CO_T + q;
        const float b = __ldg(bias + co);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int x = x0 + tx4 + p;
            if (x < nx) {
                float v = acc[p][q] + b;
                if (RELU) v = fmaxf(v, 0.f);
                if (!(row_ok && x >= R.x0 && x < R.x1)) v = 0.f;
                outb[(int64_t)co * plane + (int64_t)y * nx + x] = v;
            }
        }
    }
}

// Last layer (CIN -> 1, no ReLU) fused with the residual: d = x - (W_K a + b_K).
// One output pixel per thread, 32 x 8 tile, input channels staged in chunks.
template <int CIN>
__global__ void __launch_bounds__(CV_THREADS) k_conv3x3_last(const float* __restrict__ in,
                                                             const float* __restrict__ w,
                                                             const float* __restrict__ bias,
                                                             const float* __restrict__ xin,
                                                             int ny, int nx,
                                                             float* __restrict__ d) {
    constexpr int CHUNK = 16;
    __shared__ float sin[CHUNK][CV_ROWS][CV_TX + 2];
    __shared__ float sw[CIN * 9];
    const int img = blockIdx.z;
    const int64_t plane = (int64_t)ny * nx;
    const float* inb = in + (int64_t)img * CIN * plane;
    const int y0 = blockIdx.y * CV_TY, x0 = blockIdx.x * CV_TX;
    const int tx = threadIdx.x % CV_TX, ty = threadIdx.x / CV_TX;
    for (int e = threadIdx.x; e < CIN * 9; e += CV_THREADS) sw[e] = __ldg(w + e);
    float acc = 0.f;
    for (int ck = 0; ck < CIN; ck += CHUNK) {
        __syncthreads();
        for (int e = threadIdx.x; e < CHUNK * CV_ROWS * (CV_TX + 2); e += CV_THREADS) {
            const int c = e / (CV_ROWS * (CV_TX + 2));
            const int rem = e - c * (CV_ROWS * (CV_TX + 2));
            const int r = rem / (CV_TX + 2), v = rem - r * (CV_TX + 2);
            const int gy = y0 - 1 + r, gx = x0 - 1 + v;
            float val = 0.f;
            if (ck + c < CIN && gy >= 0 && gy < ny && gx >= 0 && gx < nx)
                val = __ldg(inb + (int64_t)(ck + c) * plane + (int64_t)gy * nx + gx);
            sin[c][r][v] = val;
        }
        __syncthreads();
        for (int c = 0; c < CHUNK && ck + c < CIN; ++c)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
                    acc = fmaf(sin[c][ty + dy][tx + dx], sw[(ck + c) * 9 + dy * 3 + dx], acc);
    }
    const int y = y0 + ty, x = x0 + tx;
    if (y < ny && x < nx) {
        const int64_t n = (int64_t)img * plane + (int64_t)y * nx + x;
        d[n] = xin[n] - (acc + __ldg(bias));
    }
}

template <int CIN, int COUT, bool RELU>
static cudaError_t launch_layer(const float* in, const float* w, const float* b, int ny, int nx,
                                int nimg, const Rect* rects, float* out, cudaStream_t s) {
    using C = ConvCfg<CIN, COUT>;
    auto kern = k_conv3x3<CIN, COUT, RELU>;
    static bool configured = false;   // per template instance
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid(ceil_div(nx, CV_TX), ceil_div(ny, CV_TY), nimg);
    const int tid = CIN == COUT ? T_CONV_FP32 : T_CONV_EDGE;
    timer_begin(tid, s);
    note_launch();
    kern<<<grid, CV_THREADS, C::SMEM, s>>>(in, w, b, ny, nx, rects, out);
    timer_end(tid, s);
    return cudaGetLastError();
}

template <int F>
static cudaError_t denoise_fp32_F(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                                  const Rect* rects, float* d, float* scratch, cudaStream_t s) {
    const size_t act = (size_t)nimg * F * ny * nx;
    float* A = scratch;
    float* B = scratch + act;
    cudaError_t e = launch_layer<1, F, true>(x, D.w32 + D.w32_off[0], D.b32 + D.b_off[0], ny, nx,
                                             nimg, rects, A, s);
    if (e != cudaSuccess) return e;
    for (int k = 1; k < D.K - 1; ++k) {
        e = launch_layer<F, F, true>(A, D.w32 + D.w32_off[k], D.b32 + D.b_off[k], ny, nx, nimg,
                                     rects, B, s);
        if (e != cudaSuccess) return e;
        float* t = A; A = B; B = t;
    }
    const int L = D.K - 1;
    dim3 grid(ceil_div(nx, CV_TX), ceil_div(ny, CV_TY), nimg);
    timer_begin(T_CONV_EDGE, s);
    note_launch();
    k_conv3x3_last<F><<<grid, CV_THREADS, 0, s>>>(A, D.w32 + D.w32_off[L], D.b32 + D.b_off[L], x,
                                                  ny, nx, d);
    timer_end(T_CONV_EDGE, s);
    return cudaGetLastError();
}

// Largest value of a non-negative array (post-ReLU activations): the float
// bit patterns of non-negative numbers order like unsigned integers.
__global__ void k_amax(const float* __restrict__ a, size_t n, unsigned* __restrict__ out) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

template <int F>
static cudaError_t denoise_fp32_amax_F(const DenoiserDev& D, const float* x, int ny, int nx,
                                       int nimg, float* d, float* scratch, unsigned* amax,
                                       cudaStream_t s) {
    const size_t act = (size_t)nimg * F * ny * nx;
    float* A = scratch;
    float* B = scratch + act;
    const int grid = 4 * num_sms();
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned) * D.K, s);
    if (e == cudaSuccess)
        e = launch_layer<1, F, true>(x, D.w32 + D.w32_off[0], D.b32 + D.b_off[0], ny, nx, nimg,
                                     nullptr, A, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_amax<<<grid, 256, 0, s>>>(A, act, amax + 0);
    for (int k = 1; k < D.K - 1; ++k) {
        e = launch_layer<F, F, true>(A, D.w32 + D.w32_off[k], D.b32 + D.b_off[k], ny, nx, nimg,
                                     nullptr, B, s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_amax<<<grid, 256, 0, s>>>(B, act, amax + k);
        float* t = A; A = B; B = t;
    }
    const int L = D.K - 1;
    dim3 g(ceil_div(nx, CV_TX), ceil_div(ny, CV_TY), nimg);
    note_launch();
    k_conv3x3_last<F><<<g, CV_THREADS, 0, s>>>(A, D.w32 + D.w32_off[L], D.b32 + D.b_off[L], x, ny,
                                               nx, d);
    return cudaGetLastError();
}

cudaError_t denoise_fp32_amax(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                              float* d, float* scratch, unsigned* amax, cudaStream_t s) {
    if (D.F != 64) return cudaErrorInvalidValue;
    return denoise_fp32_amax_F<64>(D, x, ny, nx, nimg, d, scratch, amax, s);
}

size_t denoise_fp32_scratch(const DenoiserDev& D, int ny, int nx, int nimg) {
    return sizeof(float) * 2 * (size_t)nimg * D.F * ny * nx;
}

cudaError_t denoise_fp32(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, float* scratch, cudaStream_t s) {
    if (D.ddfb) return ddfb_forward(D, x, ny, nx, nimg, rects, d, scratch, s);
    switch (D.F) {
        case 16: return denoise_fp32_F<16>(D, x, ny, nx, nimg, rects, d, scratch, s);
        case 32: return denoise_fp32_F<32>(D, x, ny, nx, nimg, rects, d, scratch, s);
        case 64: return denoise_fp32_F<64>(D, x, ny, nx, nimg, rects, d, scratch, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Block-with-halo gather / scatter (receptive-field variant of Sec. II-B2).
// Tile b holds rows r0-halo .. r1+halo-1 and cols c0-halo .. c1+halo-1 of its
// image at the top-left of a ty x tx plane; positions outside the image are
// zero and fall outside the tile's valid rect.
// ---------------------------------------------------------------------------
__global__ void k_gather(const float* __restrict__ x, int ny, int nx,
                         const BlockDesc* __restrict__ blocks, int halo, int ty, int tx,
                         float* __restrict__ tiles, Rect* __restrict__ rects) {
    const int b = blockIdx.z;
    const BlockDesc B = blocks[b];
    const int64_t plane = (int64_t)ny * nx;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && j == 0) {
        // valid rect: tile coordinates that map inside the image and inside the extended block
        const int h1 = B.r1 - B.r0 + 2 * halo, w1 = B.c1 - B.c0 + 2 * halo;
        Rect R;
        R.y0 = max(0, halo - B.r0);
        R.y1 = min(h1, ny - (B.r0 - halo));
        R.x0 = max(0, halo - B.c0);
        R.x1 = min(w1, nx - (B.c0 - halo));
        rects[b] = R;
    }
    if (i >= ty || j >= tx) return;
    const int gi = B.r0 - halo + i, gj = B.c0 - halo + j;
    const bool inside = i < B.r1 - B.r0 + 2 * halo && j < B.c1 - B.c0 + 2 * halo && gi >= 0 &&
                        gi < ny && gj >= 0 && gj < nx;
    tiles[(int64_t)b * ty * tx + (int64_t)i * tx + j] =
        inside ? x[(int64_t)B.img * plane + (int64_t)gi * nx + gj] : 0.f;
}

__global__ void k_scatter(const float* __restrict__ dt, int ny, int nx,
                          const BlockDesc* __restrict__ blocks, int halo, int ty, int tx,
                          float* __restrict__ d) {
    const int b = blockIdx.z;
    const BlockDesc B = blocks[b];
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.r1 - B.r0 || j >= B.c1 - B.c0) return;
    d[(int64_t)B.img * ny * nx + (int64_t)(B.r0 + i) * nx + (B.c0 + j)] =
        dt[(int64_t)b * ty * tx + (int64_t)(i + halo) * tx + (j + halo)];
}

cudaError_t launch_gather_blocks(const float* x, int ny, int nx, const BlockDesc* blocks,
                                 int nblocks, int halo, int ty, int tx, float* tiles, Rect* rects,
                                 cudaStream_t s) {
    dim3 blk(32, 8), grid(ceil_div(tx, 32), ceil_div(ty, 8), nblocks);
    note_launch();
    k_gather<<<grid, blk, 0, s>>>(x, ny, nx, blocks, halo, ty, tx, tiles, rects);
    return cudaGetLastError();
}

cudaError_t launch_scatter_blocks(const float* dtiles, int ny, int nx, const BlockDesc* blocks,
                                  int nblocks, int halo, int ty, int tx, float* d,
                                  cudaStream_t s) {
    dim3 blk(32, 8), grid(ceil_div(tx, 32), ceil_div(ty, 8), nblocks);
    note_launch();
    k_scatter<<<grid, blk, 0, s>>>(dtiles, ny, nx, blocks, halo, ty, tx, d);
    return cudaGetLastError();
}

}  // namespace pnp
