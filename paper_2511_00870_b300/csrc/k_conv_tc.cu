// BF16 denoiser: the F -> F 3x3 layers as an implicit GEMM on tcgen05 tensor
// cores, the 1 -> F and F -> 1 layers on CUDA cores (Sec. II-B, Eqs. 5-6,
// Example 1: D = Id - G, ReLU on all layers but the last).
//
// Activation layout ("channel-group planar"): act[img][y][cg][xp][8] BF16,
// cg = channel / 8, xp over the width padded to a multiple of 8 (padding
// columns hold zeros). One TMA box per input row - 8 channel groups x 144
// pixels (the 128-pixel output segment plus 8 on each side) - lands in shared
// memory exactly in the UMMA no-swizzle K-major layout: a core matrix is 8
// consecutive pixels x 8 channels = 128 contiguous bytes, consecutive pixel
// octets are 128 B apart (SBO) and consecutive channel groups 2304 B apart
// (LBO). A tap shift dx is then a 16-byte offset of the descriptor start
// address and a tap shift dy selects another row slot, so each input row is
// fetched from HBM/L2 once per 128-pixel column strip.
//
// GEMM per output row segment: M = 128 pixels, N = 64 output channels,
// K = 9 taps x 64 input channels, accumulated in TMEM (FP32) as 36 MMAs of
// 128 x 64 x 16. Warp roles: warp 0 = TMA producer, warp 1 = MMA issuer,
// warps 2-5 = epilogue (TMEM -> registers, bias, ReLU, zero outside the valid
// rect, BF16, global store). Input rows circulate through a 6-slot ring;
// accumulators are double-buffered in TMEM so the epilogue of one row overlaps
// the MMAs of the next. Every CTA walks a contiguous range of the
// (image, strip, row) stream, so work is balanced to within one row.
#include <cuda.h>

#include <algorithm>

#include "pnp_internal.h"
#include "tc_ptx.cuh"

namespace pnp {

namespace tc {
constexpr int F = 64;
constexpr int SEG = 128;                 // output pixels per row segment (UMMA M)
constexpr int HALO_PX = 8;               // smem row starts 8 px left of the segment
constexpr int ROW_PX = SEG + 2 * HALO_PX;   // 144
constexpr int CG_BYTES = ROW_PX * 16;       // 2304: one channel-group plane of a row
constexpr int ROW_BYTES = 8 * CG_BYTES;     // 18432
constexpr int NS = 6;                       // input-row ring slots
constexpr int TAP_W_BYTES = 8 * F * 16;     // 8192: [cg][co][8 ci] of one tap
constexpr int W_BYTES = 9 * TAP_W_BYTES;    // 73728
constexpr int THREADS = 192;
constexpr int OFF_RING = 0;
constexpr int OFF_W = OFF_RING + NS * ROW_BYTES;
constexpr int OFF_BIAS = OFF_W + W_BYTES;
constexpr int OFF_BAR = OFF_BIAS + F * 4;
constexpr int NBAR = 2 * NS + 1 + 2 + 2 + 1;   // full, empty, weights, tfull, tempty, drain
constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
constexpr int SMEM = OFF_MISC + 16 + 1024;     // + alignment slack
constexpr uint32_t IDESC = ptx::idesc_bf16_f32(SEG, F);
constexpr long long BUDGET = 4000000000LL;     // ~2 s of SM clock per wait
}  // namespace tc

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

struct TcConvArgs {
    const __nv_bfloat16* wblob;   // [9 taps][8 cg][64 co][8 ci]
    const float* bias;            // [64]
    __nv_bfloat16* out;
    const Rect* rects;
    int* err;
    int ny, nx, nxp, nimg, strips;
    int64_t total_rows;
};

__global__ void __launch_bounds__(tc::THREADS, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tin, const TcConvArgs a) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* ring = smem + OFF_RING;
    uint8_t* wsm = smem + OFF_W;
    float* bias_s = (float*)(smem + OFF_BIAS);
    uint64_t* bars = (uint64_t*)(smem + OFF_BAR);
    uint64_t* full = bars;
    uint64_t* empty = bars + NS;
    uint64_t* wbar = bars + 2 * NS;
    uint64_t* tfull = bars + 2 * NS + 1;
    uint64_t* tempty = bars + 2 * NS + 3;
    uint64_t* drain = bars + 2 * NS + 5;
    uint32_t* tmem_slot = (uint32_t*)(smem + OFF_MISC);
    volatile int* abort_flag = (volatile int*)(smem + OFF_MISC + 4);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        ptx::mbar_init(wbar, 1);
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&tfull[i], 1);
            ptx::mbar_init(&tempty[i], 4);
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) ptx::prefetch_tensormap(&tin);
    if (warp == 2) {
        ptx::tmem_alloc(tmem_slot, 128);
        ptx::tmem_relinquish();
    }
    if (threadIdx.x >= 64 && threadIdx.x < 64 + F) bias_s[threadIdx.x - 64] = a.bias[threadIdx.x - 64];
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    // this CTA's share of the (image, strip, row) stream
    const int64_t g_begin = a.total_rows * blockIdx.x / gridDim.x;
    const int64_t g_end = a.total_rows * (blockIdx.x + 1) / gridDim.x;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            ptx::mbar_arrive_expect_tx(wbar, W_BYTES);
            for (int t = 0; t < 9; ++t)
                ptx::bulk_load(wsm + t * TAP_W_BYTES, (const uint8_t*)a.wblob + t * TAP_W_BYTES,
                               TAP_W_BYTES, wbar);
            uint32_t L = 0;
            bool ok = true;
            for (int64_t g = g_begin; g < g_end && ok;) {
                const int64_t q = g / a.ny;
                const int y = (int)(g - q * a.ny);
                const int s = (int)(q % a.strips), img = (int)(q / a.strips);
                const int len = (int)imin64(g_end - g, (int64_t)a.ny - y);
                for (int r = y - 1; r <= y + len && ok; ++r, ++L) {
                    const uint32_t slot = L % NS, u = L / NS;
                    if (!ptx::mbar_wait(&empty[slot], (u & 1) ^ 1, abort_flag, BUDGET)) { ok = false; break; }
                    ptx::mbar_arrive_expect_tx(&full[slot], ROW_BYTES);
                    ptx::tma_load_5d(ring + slot * ROW_BYTES, &tin, &full[slot], 0,
                                     s * (SEG / 8) - HALO_PX / 8, 0, r, img);
                }
                g += len;
            }
            // wait for this thread's copies still in flight (only after an abort)
            if (!ok) {
                for (uint32_t k = (L > NS ? L - NS : 0); k < L; ++k)
                    ptx::mbar_wait(&full[k % NS], (k / NS) & 1, abort_flag, BUDGET / 8);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            bool ok = ptx::mbar_wait(wbar, 0, abort_flag, BUDGET);
            const uint32_t ring_a = ptx::smem_u32(ring), w_a = ptx::smem_u32(wsm);
            uint32_t L = 0, R = 0;
            bool issued = false;
            for (int64_t g = g_begin; g < g_end && ok;) {
                const int64_t q = g / a.ny;
                const int y = (int)(g - q * a.ny);
                const int len = (int)imin64(g_end - g, (int64_t)a.ny - y);
                (void)y;
                const uint32_t base = L;
                for (uint32_t k = 0; k < 2 && ok; ++k)
                    ok = ptx::mbar_wait(&full[(base + k) % NS], ((base + k) / NS) & 1, abort_flag, BUDGET);
                for (int k = 0; k < len && ok; ++k) {
                    const uint32_t Ln = base + k + 2;
                    ok = ptx::mbar_wait(&full[Ln % NS], (Ln / NS) & 1, abort_flag, BUDGET);
                    const uint32_t acc = R & 1, v = R >> 1;
                    if (ok) ok = ptx::mbar_wait(&tempty[acc], (v & 1) ^ 1, abort_flag, BUDGET);
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t d_tmem = tmem_base + acc * F;
#pragma unroll 1
                    for (int dy = 0; dy < 3; ++dy) {
                        const uint32_t slot_addr = ring_a + ((base + k + dy) % NS) * ROW_BYTES;
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = ptx::smem_desc_noswizzle(
                                    slot_addr + kk * 2 * CG_BYTES + (HALO_PX - 1 + dx) * 16, CG_BYTES, 128);
                                const uint64_t bd = ptx::smem_desc_noswizzle(
                                    w_a + (dy * 3 + dx) * TAP_W_BYTES + kk * 2 * (F * 16), F * 16, 128);
                                ptx::mma_bf16(d_tmem, ad, bd, IDESC, (dy | dx | kk) != 0);
                            }
                        }
                    }
                    issued = true;
                    ptx::mma_commit(&empty[(base + k) % NS]);   // row y+k-1 is no longer needed
                    ptx::mma_commit(&tfull[acc]);
                    ++R;
                }
                if (ok) {
                    ptx::mma_commit(&empty[(base + len) % NS]);
                    ptx::mma_commit(&empty[(base + len + 1) % NS]);
                }
                L = base + len + 2;
                g += len;
            }
            if (issued) {
                ptx::mma_commit(drain);
                ptx::mbar_wait(drain, 0, abort_flag, BUDGET);
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5 own TMEM lane quadrants 2,3,0,1
        const int quad = warp & 3;
        const int j = quad * 32 + lane;
        uint32_t R = 0;
        bool ok = true;
        for (int64_t g = g_begin; g < g_end && ok;) {
            const int64_t q = g / a.ny;
            const int y = (int)(g - q * a.ny);
            const int s = (int)(q % a.strips), img = (int)(q / a.strips);
            const int len = (int)imin64(g_end - g, (int64_t)a.ny - y);
            const Rect rc = a.rects ? a.rects[img] : Rect{0, a.ny, 0, a.nx};
            const int x = s * SEG + j;
            for (int k = 0; k < len; ++k, ++R) {
                const uint32_t acc = R & 1, v = R >> 1;
                if (!ptx::mbar_wait(&tfull[acc], v & 1, abort_flag, BUDGET)) { ok = false; break; }
                ptx::tc_fence_after();
                uint32_t r[64];
                ptx::tmem_ld_32x32b_x64(tmem_base + ((uint32_t)(quad * 32) << 16) + acc * F, r);
                ptx::tmem_ld_wait();
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
                const int yy = y + k;
                if (x < a.nxp) {
                    const bool valid = x < a.nx && yy >= rc.y0 && yy < rc.y1 && x >= rc.x0 && x < rc.x1;
                    __nv_bfloat16* o = a.out + ((((int64_t)img * a.ny + yy) * 8) * a.nxp + x) * 8;
#pragma unroll
                    for (int cg = 0; cg < 8; ++cg) {
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c0 = cg * 8 + 2 * e;
                            float v0 = fmaxf(__uint_as_float(r[c0]) + bias_s[c0], 0.f);
                            float v1 = fmaxf(__uint_as_float(r[c0 + 1]) + bias_s[c0 + 1], 0.f);
                            if (!valid) v0 = v1 = 0.f;
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                            pk[e] = *reinterpret_cast<uint32_t*>(&h2);
                        }
                        *reinterpret_cast<uint4*>(o + (int64_t)cg * a.nxp * 8) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                }
            }
            g += len;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 128);
    }
    if (threadIdx.x == 0 && *abort_flag && a.err) atomicExch(a.err, (int)PNP_ETIMEOUT);
}

// ---------------------------------------------------------------------------
// First layer 1 -> 64 (+bias, ReLU) from the FP32 image into the BF16
// channel-group-planar layout; padding columns are written as zeros.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_first_bf16(const float* __restrict__ x,
                                                    const float* __restrict__ w,   // [9][64]
                                                    const float* __restrict__ bias, int ny,
                                                    int nx, int nxp,
                                                    const Rect* __restrict__ rects,
                                                    __nv_bfloat16* __restrict__ out) {
    __shared__ float ws[9 * 64 + 64];
    for (int e = threadIdx.x; e < 9 * 64; e += blockDim.x) ws[e] = w[e];
    for (int e = threadIdx.x; e < 64; e += blockDim.x) ws[9 * 64 + e] = bias[e];
    __syncthreads();
    const int xx = blockIdx.x * blockDim.x + threadIdx.x;
    const int yy = blockIdx.y, img = blockIdx.z;
    if (xx >= nxp) return;
    const int64_t plane = (int64_t)ny * nx;
    const Rect rc = rects ? rects[img] : Rect{0, ny, 0, nx};
    const bool valid = xx < nx && yy >= rc.y0 && yy < rc.y1 && xx >= rc.x0 && xx < rc.x1;
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int sy = yy + t / 3 - 1, sx = xx + t % 3 - 1;
        v[t] = (valid && sy >= 0 && sy < ny && sx >= 0 && sx < nx)
                   ? __ldg(x + img * plane + (int64_t)sy * nx + sx)
                   : 0.f;
    }
    __nv_bfloat16* o = out + ((((int64_t)img * ny + yy) * 8) * nxp + xx) * 8;
#pragma unroll
    for (int cg = 0; cg < 8; ++cg) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float r2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = cg * 8 + 2 * e + h;
                float s = ws[9 * 64 + co];
#pragma unroll
                for (int t = 0; t < 9; ++t) s = fmaf(ws[t * 64 + co], v[t], s);
                r2[h] = valid ? fmaxf(s, 0.f) : 0.f;
            }
            __nv_bfloat162 h2 = __floats2bfloat162_rn(r2[0], r2[1]);
            pk[e] = *reinterpret_cast<uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// ---------------------------------------------------------------------------
// Last layer 64 -> 1 (no ReLU) fused with the residual d = x - G(x).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_last_bf16(const __nv_bfloat16* __restrict__ act,
                                                   const float* __restrict__ w,   // [9][64]
                                                   const float* __restrict__ bias,
                                                   const float* __restrict__ x, int ny, int nx,
                                                   int nxp, float* __restrict__ d) {
    __shared__ float ws[9 * 64];
    for (int e = threadIdx.x; e < 9 * 64; e += blockDim.x) ws[e] = w[e];
    __syncthreads();
    const int xx = blockIdx.x * blockDim.x + threadIdx.x;
    const int yy = blockIdx.y, img = blockIdx.z;
    if (xx >= nx) return;
    float acc = 0.f;
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
        const int sy = yy + t / 3 - 1, sx = xx + t % 3 - 1;
        if (sy < 0 || sy >= ny || sx < 0 || sx >= nx) continue;
        const __nv_bfloat16* p = act + ((((int64_t)img * ny + sy) * 8) * nxp + sx) * 8;
#pragma unroll
        for (int cg = 0; cg < 8; ++cg) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(p + (int64_t)cg * nxp * 8));
            const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&wd[e]);
                const float2 f = __bfloat1622float2(h2);
                acc = fmaf(ws[t * 64 + cg * 8 + 2 * e], f.x, acc);
                acc = fmaf(ws[t * 64 + cg * 8 + 2 * e + 1], f.y, acc);
            }
        }
    }
    const int64_t n = (int64_t)img * ny * nx + (int64_t)yy * nx + xx;
    d[n] = x[n] - (acc + __ldg(bias));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

static inline int pad8(int n) { return (n + 7) & ~7; }

size_t denoise_bf16_scratch(const DenoiserDev& D, int ny, int nx, int nimg) {
    (void)D;
    return 2 * (size_t)nimg * ny * pad8(nx) * 64 * sizeof(__nv_bfloat16) + 256;
}

static cudaError_t make_act_map(CUtensorMap* m, void* base, int ny, int nxp, int nimg) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {64, (cuuint64_t)nxp / 8, 8, (cuuint64_t)ny, (cuuint64_t)nimg};
    const cuuint64_t strides[4] = {128, (cuuint64_t)nxp * 16, (cuuint64_t)nxp * 128,
                                   (cuuint64_t)nxp * 128 * ny};
    const cuuint32_t box[5] = {64, tc::ROW_PX / 8, 8, 1, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t conv_tc_layer(const __nv_bfloat16* in, const __nv_bfloat16* wblob, const float* bias,
                          int ny, int nx, int nimg, const Rect* rects, __nv_bfloat16* out,
                          int* err, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int nxp = pad8(nx);
    CUtensorMap m;
    cudaError_t e = make_act_map(&m, (void*)in, ny, nxp, nimg);
    if (e != cudaSuccess) return e;
    TcConvArgs a;
    a.wblob = wblob;
    a.bias = bias;
    a.out = out;
    a.rects = rects;
    a.err = err;
    a.ny = ny;
    a.nx = nx;
    a.nxp = nxp;
    a.nimg = nimg;
    a.strips = ceil_div(nx, tc::SEG);
    a.total_rows = (int64_t)nimg * a.strips * ny;
    const int grid = (int)std::min<int64_t>(num_sms(), a.total_rows);
    timer_begin(T_CONV_TC, s);
    k_conv_tc<<<grid, tc::THREADS, tc::SMEM, s>>>(m, a);
    timer_end(T_CONV_TC, s);
    return cudaGetLastError();
}

cudaError_t denoise_bf16(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, void* scratch, cudaStream_t s) {
    if (D.F != 64 || !D.wtc) return cudaErrorInvalidValue;
    const int nxp = pad8(nx);
    const size_t act = (size_t)nimg * ny * nxp * 64;
    __nv_bfloat16* A = (__nv_bfloat16*)scratch;
    __nv_bfloat16* B = A + act;
    int* err = (int*)(B + act);
    dim3 g1(ceil_div(nxp, 128), ny, nimg);
    timer_begin(T_CONV_EDGE, s);
    k_first_bf16<<<g1, 128, 0, s>>>(x, D.wfirst, D.b32 + D.b_off[0], ny, nx, nxp, rects, A);
    timer_end(T_CONV_EDGE, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int k = 1; k < D.K - 1; ++k) {
        e = conv_tc_layer(A, D.wtc + (size_t)(k - 1) * (tc::W_BYTES / 2), D.b32 + D.b_off[k], ny,
                          nx, nimg, rects, B, err, s);
        if (e != cudaSuccess) return e;
        __nv_bfloat16* t = A; A = B; B = t;
    }
    dim3 g2(ceil_div(nx, 128), ny, nimg);
    timer_begin(T_CONV_EDGE, s);
    k_last_bf16<<<g2, 128, 0, s>>>(A, D.wlast, D.b32 + D.b_off[D.K - 1], x, ny, nx, nxp, d);
    timer_end(T_CONV_EDGE, s);
    return cudaGetLastError();
}

}  // namespace pnp
