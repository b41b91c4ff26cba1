// Blur operator H, its adjoint, the fused PnP-ULA update and the final moments.
//
// H is the circular 2-D convolution of the Gaussian-deconvolution likelihood
// (Sec. III-A2): (h * x)[i,j] = sum_{a,b} h[a,b] x[i-a+ry, j-b+rx] (indices mod
// the image size). H^T is the correlation sum_{a,b} h[a,b] r[i+a-ry, j+b-rx].
// Both are evaluated as a correlation over a shared-memory window that holds the
// output tile plus a (kh-1) x (kw-1) circular halo; the forward operator just
// uses the flipped kernel.
//
// A tile is 64 outputs wide and R * BY rows high: a block of 16 x BY threads,
// each thread owning R rows of 4 consecutive outputs. The kernel width kw is a
// template parameter (the tap loop is unrolled; taps and window rows come out of
// shared memory as 128-bit loads, the window row slides through registers), the
// kernel height is a run-time loop. Every output is the fixed-order sum
// acc = fma(h[a][b], w, acc) over a = 0..kh-1, then b = 0..kw-1, starting from 0,
// so results are bitwise the same for every tile shape, which is what lets the
// tile be picked by timing (stencil_autotune) without changing any result.
//
// Rank-one kernels h = u v^T (Gaussian, uniform; detected on the host) take a
// separable path: a vertical pass over every window column into a
// shared-memory strip V = u * window, then a horizontal pass
// out = sum_b v[b] V[., j + b] - kh + kw instead of kh kw FMAs per output,
// again in a fixed order.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "pdl.cuh"
#include "philox.cuh"
#include "pnp_internal.h"
#include "stencil_dev.cuh"

namespace pnp {

// Candidate tile shapes: R output rows per thread, BY thread rows per block.
struct TileShape {
    int R, BY;
};
constexpr TileShape kTiles[] = {{1, 16}, {2, 8}, {2, 16}, {4, 8}, {1, 8}, {4, 16}};
constexpr int kNumTiles = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
static std::atomic<int> g_forced_tile{-1};

// Window rows [0, rows + kh - 1) x cols [0, WXA) of image `img` starting at
// image coordinate (i0 - ry, j0 - AL), wrapped circularly, copied
// asynchronously (the caller waits with cp_async_wait_all before its
// barrier). Interior tiles of images whose rows are whole 16-byte units copy
// 16 bytes per access; others one float at a time.
template <int KW>
__device__ __forceinline__ void fill_window(const float* __restrict__ img, int ny, int nx, int i0,
                                            int j0, int kh, int rows, float* win) {
    using G = Geom<KW>;
    const int ry = kh / 2;
    const int wy = rows + kh - 1;
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const bool interior = i0 - ry >= 0 && i0 + rows - 1 + ry < ny && j0 - G::AL >= 0 &&
                          j0 + ST_TX - 1 + G::AL < nx;
    const bool vec = (nx & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
    if (interior && vec) {
        constexpr int NV = G::WXA / 4;
        const float* base = img + (int64_t)(i0 - ry) * nx + (j0 - G::AL);
        for (int e = tid; e < wy * NV; e += nt) {
            const int u = e / NV, c4 = e - u * NV;
            cp_async16(win + u * G::WP + 4 * c4, base + (int64_t)u * nx + 4 * c4);
        }
    } else if (interior) {
        const float* base = img + (int64_t)(i0 - ry) * nx + (j0 - G::AL);
        for (int e = tid; e < wy * G::WXA; e += nt) {
            const int u = e / G::WXA, v = e - u * G::WXA;
            cp_async4(win + u * G::WP + v, base + (int64_t)u * nx + v);
        }
    } else {
        for (int e = tid; e < wy * G::WXA; e += nt) {
            const int u = e / G::WXA, v = e - u * G::WXA;
            const int gi = wrap(i0 - ry + u, ny), gj = wrap(j0 - G::AL + v, nx);
            cp_async4(win + u * G::WP + v, img + (int64_t)gi * nx + gj);
        }
    }
}

// 2-D taps (flipped if `flip`), zero-padded to KWP per row.
template <int KW>
__device__ __forceinline__ void load_taps2d(const float* __restrict__ h, int kh, bool flip,
                                            float* hs) {
    using G = Geom<KW>;
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int kk = kh * KW;
    for (int e = tid; e < kh * G::KWP; e += nt) {
        const int a = e / G::KWP, b = e - a * G::KWP;
        float v = 0.f;
        if (b < KW) {
            const int k = a * KW + b;
            v = __ldg(h + (flip ? kk - 1 - k : k));
        }
        hs[e] = v;
    }
}

// acc[o][q] = sum_{a,b} hs[a][b] win[ty R + o + a][4 tx + SHIFT + q + b]
template <int KW, int R>
__device__ __forceinline__ void correlate(const float* win, const float* hs, int kh, int ty, int tx,
                                          float acc[R][4]) {
    using G = Geom<KW>;
#pragma unroll
    for (int o = 0; o < R; ++o)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[o][q] = 0.f;
#pragma unroll 1
    for (int u = 0; u < R + kh - 1; ++u) {
        float w[4 * G::NW4];
        const float4* src = reinterpret_cast<const float4*>(win + (ty * R + u) * G::WP + 4 * tx);
#pragma unroll
        for (int k = 0; k < G::NW4; ++k) {
            const float4 v = src[k];
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int o = 0; o < R; ++o) {
            const int a = u - o;
            if (a < 0 || a >= kh) continue;
            const float4* hp = reinterpret_cast<const float4*>(hs + a * G::KWP);
#pragma unroll
            for (int b4 = 0; b4 < G::KWP / 4; ++b4) {
                const float4 hv = hp[b4];
                const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const int b = 4 * b4 + bb;
                    if (b < KW) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            acc[o][q] = fmaf(hh[bb], w[G::SHIFT + q + b], acc[o][q]);
                    }
                }
            }
        }
    }
}

// Shared-memory floats of one tile: window, then the 2-D taps or the strip T
// and the separable taps.
static int window_pitch(int kw) {
    const int rx = kw / 2, al = (rx + 3) & ~3, shift = al - rx;
    const int nw4 = (kw + 6) / 4 + (shift > 0 ? 1 : 0);
    const int wxa = ST_TX + 2 * al;
    return wxa > ST_TX + 4 * nw4 ? wxa : ST_TX + 4 * nw4;
}

static size_t tile_smem(int kw, int kh, int rows, bool sep) {
    const int wp = window_pitch(kw), kwp = (kw + 3) & ~3;
    const size_t wy = (size_t)rows + kh - 1;
    if (!sep) return sizeof(float) * (wy * wp + (size_t)kh * kwp);
    return sizeof(float) * (wy * wp + (size_t)rows * wp + kwp + ((kh + 3) & ~3));
}

// The R x 4 outputs of thread (threadIdx.x, threadIdx.y) of the tile at
// (i0, j0): the correlation of `img` with the taps (flipped if `flip`). Every
// thread of the block must call it (it synchronises); `active` threads get acc.
template <int KW, int R, bool SEP>
__device__ __forceinline__ void stencil_tile(const float* img, int ny, int nx, int i0, int j0,
                                             int kh, int rows, const float* h, bool flip,
                                             float* sm, bool active, float acc[R][4]) {
    using G = Geom<KW>;
    const int wy = rows + kh - 1;
    float* win = sm;
    fill_window<KW>(img, ny, nx, i0, j0, kh, rows, win);
    if constexpr (SEP) {
        float* V = win + wy * G::WP;      // rows x WP
        float* vs = V + rows * G::WP;
        float* us = vs + G::KWP;
        load_taps_sep<KW>(h, kh, flip, vs, us);
        cp_async_wait_all();
        __syncthreads();
        sep_vert<KW, SEP_VR>(win, us, kh, rows, V);
        __syncthreads();
        if (active) sep_horz<KW, R>(V, vs, threadIdx.y, threadIdx.x, acc);
    } else {
        float* hs = win + wy * G::WP;
        load_taps2d<KW>(h, kh, flip, hs);
        cp_async_wait_all();
        __syncthreads();
        if (active) correlate<KW, R>(win, hs, kh, threadIdx.y, threadIdx.x, acc);
    }
}

// out = (a (h * x) - y) scale; y is shared by the images (y_img_stride 0) or
// one plane per image (the Poisson sampler's z1).
template <int KW, int R, bool SEP>
__device__ __forceinline__ void blur_body(const BlurArgs& A, int bx, int by, int img) {
    extern __shared__ float4 sm4[];
    const float* __restrict__ x = A.x;
    const float* __restrict__ y = A.y;
    const float* __restrict__ h = A.h;
    const int kh = A.kh, ny = A.ny, nx = A.nx, adjoint = A.adjoint;
    const float scale = A.scale, a = A.a;
    float* __restrict__ out = A.out;
    const int64_t y_img_stride = A.y_img_stride;
    const int rows = R * blockDim.y;
    const int64_t plane = (int64_t)ny * nx;
    const int i0 = by * rows, j0 = bx * ST_TX;
    pdl_wait();
    pdl_launch_dependents();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = j0 + 4 * tx;
    const bool active = j < nx && i0 + ty * R < ny;
    float acc[R][4];
    // forward H: correlation with the flipped kernel; adjoint: with h itself
    stencil_tile<KW, R, SEP>(x + img * plane, ny, nx, i0, j0, kh, rows, h, !adjoint,
                             reinterpret_cast<float*>(sm4), active, acc);
    if (!active) return;
    if (y) y += img * y_img_stride;
    // 128-bit accesses when rows are whole float4s (then j + 3 < nx) and aligned
    const bool vec = (nx & 3) == 0 && ((reinterpret_cast<uintptr_t>(out) |
                                        reinterpret_cast<uintptr_t>(y)) & 15) == 0;
#pragma unroll
    for (int o = 0; o < R; ++o) {
        const int i = i0 + ty * R + o;
        if (i >= ny) break;
        const int64_t n = (int64_t)i * nx + j;
        if (vec) {
            // a (h * x) rounded before y is subtracted (no fused multiply-add),
            // so the per-job and the grouped launches give the same r
            float4 v = make_float4(__fmul_rn(a, acc[o][0]), __fmul_rn(a, acc[o][1]),
                                   __fmul_rn(a, acc[o][2]), __fmul_rn(a, acc[o][3]));
            if (y) {
                const float4 yv = __ldg(reinterpret_cast<const float4*>(y + n));
                v.x -= yv.x; v.y -= yv.y; v.z -= yv.z; v.w -= yv.w;
            }
            v.x *= scale; v.y *= scale; v.z *= scale; v.w *= scale;
            *reinterpret_cast<float4*>(out + img * plane + n) = v;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (j + q < nx) {
                    float v = __fmul_rn(a, acc[o][q]);
                    if (y) v -= __ldg(y + n + q);
                    out[img * plane + n + q] = v * scale;
                }
            }
        }
    }
}

template <int KW, int R, bool SEP>
__global__ void __launch_bounds__(256) k_blur(const BlurArgs A) {
    blur_body<KW, R, SEP>(A, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Fused x-update (Eq. 8): g = H^T r / sigma^2 from the shared-memory window
// of r, then x+ = x - gamma g + c_prior (d - x) + c_proj (clamp(x) - x)
// + c_noise xi and, when sampling, the FP32 Welford step
// delta = x+ - mean; mean += delta / n; m2 += delta (x+ - mean).
// With `arrive` set, the last block to finish advances the device step counter
// (every block has read t by then).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void normals4(uint32_t key0, uint32_t key1, int64_t n0, uint32_t t,
                                         uint32_t chain, float z[4], uint32_t stream = 0) {
    // normals of the 4 pixels n0..n0+3 (flat row-major index): 1 or 2 Philox groups
    const uint32_t m0 = (uint32_t)(n0 >> 2);
    float za[4];
    normals_group(m0, t, chain, key0, key1, za, stream);
    const int off = (int)(n0 & 3);
    if (off == 0) {
        z[0] = za[0]; z[1] = za[1]; z[2] = za[2]; z[3] = za[3];
    } else {
        float zb[4];
        normals_group(m0 + 1, t, chain, key0, key1, zb, stream);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = off + q;
            const float a = k == 0 ? za[0] : k == 1 ? za[1] : k == 2 ? za[2] : za[3];
            const float b = k == 4 ? zb[0] : k == 5 ? zb[1] : zb[2];
            z[q] = k < 4 ? a : b;
        }
    }
}

template <int KW, int R, bool SEP>
__device__ __forceinline__ void update_body(const UpdateParams& p, int bx, int by, int chain,
                                            unsigned nblk) {
    extern __shared__ float4 sm4[];
    const int kh = p.kh, ny = p.ny, nx = p.nx;
    const int rows = R * blockDim.y;
    const int64_t plane = (int64_t)ny * nx;
    const int i0 = by * rows, j0 = bx * ST_TX;
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = j0 + 4 * tx;
    const bool active = j < nx && i0 + ty * R < ny;
    if (active && (tx & 7) == 0) {
        // the operands of this thread's outputs head for L2 while the window is
        // copied and the stencil runs (one 128-byte line per 8 threads of a row)
#pragma unroll
        for (int o = 0; o < R; ++o) {
            const int i = i0 + ty * R + o;
            if (i >= ny) break;
            const int64_t n0 = (int64_t)chain * plane + (int64_t)i * nx + j;
            if (p.d) prefetch_l2(p.d + n0);
            if (p.qb) prefetch_l2(p.qb + (int64_t)i * nx + j);
            if (p.mean) {
                prefetch_l2(p.mean + n0);
                prefetch_l2(p.m2 + n0);
            }
            if (!p.qb) prefetch_l2(p.x + n0);
        }
    }
    float g[R][4];
    stencil_tile<KW, R, SEP>(p.r + chain * plane, ny, nx, i0, j0, kh, rows,
                             SEP ? p.hsep : p.h, false, reinterpret_cast<float*>(sm4), active, g);
    if (active) {
        float inv_n = p.inv_n;
        if (p.burn_dev) {
            const int64_t n = (int64_t)t + 1 - *p.burn_dev;
            inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
        }
        // one-pass gradient: the stencil ran over the current state x itself,
        // so x at this thread's outputs is in the window (rows from i0 - kh/2,
        // columns from j0 - AL), and x+ goes to the other state buffer
        const bool fused = p.qb != nullptr;
        const float* xwin = reinterpret_cast<const float*>(sm4) +
                            (ty * R + kh / 2) * Geom<KW>::WP + 4 * tx + Geom<KW>::AL;
        float* xc = p.x + chain * plane;
        float* xo = fused ? p.x_out + chain * plane : xc;
        const float* dc = p.d ? p.d + chain * plane : nullptr;
        float* mc = p.mean ? p.mean + chain * plane : nullptr;
        float* qc = p.m2 ? p.m2 + chain * plane : nullptr;
        const bool vec = (nx & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(p.x) | reinterpret_cast<uintptr_t>(p.d) |
                           reinterpret_cast<uintptr_t>(p.mean) | reinterpret_cast<uintptr_t>(p.m2) |
                           reinterpret_cast<uintptr_t>(p.z2) | reinterpret_cast<uintptr_t>(p.qb) |
                           reinterpret_cast<uintptr_t>(p.x_out)) & 15) == 0;
#pragma unroll
        for (int o = 0; o < R; ++o) {
            const int i = i0 + ty * R + o;
            if (i >= ny) break;
            const int64_t n0 = (int64_t)i * nx + j;
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (vec) {
                // this row's operands (prefetched to L2 above) are loaded before
                // the noise is drawn, so their latency overlaps the Philox
                // rounds; mean and m2 are read before x+ is stored
                const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 bv = fused ? __ldg(reinterpret_cast<const float4*>(p.qb + n0)) : zero4;
                const float4 dv = dc ? __ldg(reinterpret_cast<const float4*>(dc + n0)) : zero4;
                const float4 z2v =
                    p.z2 ? __ldg(reinterpret_cast<const float4*>(p.z2 + chain * plane + n0)) : zero4;
                float4 mo = zero4, qo = zero4;
                if (inv_n > 0.f) {
                    mo = *reinterpret_cast<const float4*>(mc + n0);
                    qo = *reinterpret_cast<const float4*>(qc + n0);
                }
                const float4 xv = fused ? *reinterpret_cast<const float4*>(xwin + o * Geom<KW>::WP)
                                        : *reinterpret_cast<const float4*>(xc + n0);
                // n0 is a multiple of 4 here (nx and j are): one Philox group
                if (p.c_noise != 0.f)
                    normals_group((uint32_t)(n0 >> 2), t, (uint32_t)chain, p.key0, p.key1, z);
                if (fused) {
                    // g = (H^T H) x - H^T y
                    g[o][0] -= bv.x;
                    g[o][1] -= bv.y;
                    g[o][2] -= bv.z;
                    g[o][3] -= bv.w;
                }
                float4 v;
                v.x = update1(p, xv.x, g[o][0], dv.x, z[0], z2v.x);
                v.y = update1(p, xv.y, g[o][1], dv.y, z[1], z2v.y);
                v.z = update1(p, xv.z, g[o][2], dv.z, z[2], z2v.z);
                v.w = update1(p, xv.w, g[o][3], dv.w, z[3], z2v.w);
                *reinterpret_cast<float4*>(xo + n0) = v;
                if (inv_n > 0.f) {
                    welford1(v.x, inv_n, mo.x, qo.x);
                    welford1(v.y, inv_n, mo.y, qo.y);
                    welford1(v.z, inv_n, mo.z, qo.z);
                    welford1(v.w, inv_n, mo.w, qo.w);
                    *reinterpret_cast<float4*>(mc + n0) = mo;
                    *reinterpret_cast<float4*>(qc + n0) = qo;
                }
            } else {
                if (p.c_noise != 0.f) normals4(p.key0, p.key1, n0, t, (uint32_t)chain, z);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (j + q >= nx) break;
                    const int64_t n = n0 + q;
                    if (fused) g[o][q] -= __ldg(p.qb + n);   // g = (H^T H) x - H^T y
                    const float xv = fused ? xwin[o * Geom<KW>::WP + q] : xc[n];
                    const float v = update1(p, xv, g[o][q], dc ? __ldg(dc + n) : 0.f, z[q],
                                            p.z2 ? __ldg(p.z2 + chain * plane + n) : 0.f);
                    xo[n] = v;
                    if (inv_n > 0.f) {
                        float mo = mc[n], qo = qc[n];
                        welford1(v, inv_n, mo, qo);
                        mc[n] = mo;
                        qc[n] = qo;
                    }
                }
            }
        }
    }
    if (p.arrive) {
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            if (atomicAdd(p.arrive, 1u) == nblk - 1) {
                *p.arrive = 0u;
                *const_cast<uint32_t*>(p.t_dev) = t + 1u;
            }
        }
    }
}

template <int KW, int R, bool SEP>
__global__ void __launch_bounds__(256) k_update(const UpdateParams p) {
    update_body<KW, R, SEP>(p, blockIdx.x, blockIdx.y, blockIdx.z,
                            gridDim.x * gridDim.y * gridDim.z);
}

// ---------------------------------------------------------------------------
// Poisson sampler, auxiliary variables (Eq. 14, PSGLA transition of z from the
// new x, Algorithm 1's z-update): w = eta (h * x+) from the shared-memory
// window of x+ (the forward operator: correlation with the flipped taps), then
//   z1+ = prox_{kappa1 KL(y || .)}( z1 - (kappa1 / rho1)(z1 - w) + sqrt(2 kappa1) zeta1 )
//   z2+ = max( z2 - (kappa2 / rho2)(z2 - x+) + sqrt(2 kappa2) zeta2, 0 )
// with zeta1, zeta2 from Philox streams 1 and 2. The KL prox is the positive
// root of u^2 + (kappa - v) u - kappa y = 0, evaluated as (a + s) / 2 for
// a = v - kappa >= 0 and as 2 kappa y / (s - a) otherwise (s = sqrt(a^2 + 4
// kappa y)), which avoids the cancellation of the first form for a < 0. With
// r_out set it also writes the next iteration's residual eta H x+ - z1+ (the
// iteration then needs no blur launch). With `arrive` set, the last block
// advances the step counter (this is the last kernel of a Poisson iteration).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kl_prox(float v, float y, float kappa) {
    const float a = v - kappa;
    const float s = sqrtf(fmaf(a, a, 4.0f * kappa * y));
    return a >= 0.f ? 0.5f * (a + s) : (2.0f * kappa * y) / (s - a);
}

template <int KW, int R, bool SEP>
__device__ __forceinline__ void zupdate_body(const ZParams& p, int bx, int by, int chain,
                                             unsigned nblk) {
    extern __shared__ float4 sm4[];
    const int kh = p.kh, ny = p.ny, nx = p.nx;
    const int rows = R * blockDim.y;
    const int64_t plane = (int64_t)ny * nx;
    const int i0 = by * rows, j0 = bx * ST_TX;
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = j0 + 4 * tx;
    const bool active = j < nx && i0 + ty * R < ny;
    float hx[R][4];
    // forward operator on x+: correlation with the flipped kernel
    stencil_tile<KW, R, SEP>(p.x + chain * plane, ny, nx, i0, j0, kh, rows, SEP ? p.hsep : p.h,
                             true, reinterpret_cast<float*>(sm4), active, hx);
    if (active) {
        const float* xc = p.x + chain * plane;
        float* z1c = p.z1 + chain * plane;
        float* z2c = p.z2 + chain * plane;
#pragma unroll
        for (int o = 0; o < R; ++o) {
            const int i = i0 + ty * R + o;
            if (i >= ny) break;
            const int64_t n0 = (int64_t)i * nx + j;
            float e1[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
            if (p.noise && (nx & 3) == 0) {
                // n0 is a multiple of 4: one Philox group per stream
                normals_group((uint32_t)(n0 >> 2), t, (uint32_t)chain, p.key0, p.key1, e1, 1u);
                normals_group((uint32_t)(n0 >> 2), t, (uint32_t)chain, p.key0, p.key1, e2, 2u);
            } else if (p.noise) {
                normals4(p.key0, p.key1, n0, t, (uint32_t)chain, e1, 1u);
                normals4(p.key0, p.key1, n0, t, (uint32_t)chain, e2, 2u);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (j + q >= nx) break;
                const int64_t n = n0 + q;
                // eta H x+ rounded once: every kernel that inlines this body
                // (per job or grouped) then forms z1+ and r from the same w,
                // whatever multiply-add fusion the compiler picks around it
                const float w = __fmul_rn(p.eta, hx[o][q]);
                const float z1 = z1c[n];
                const float v1 = z1 - p.a1 * (z1 - w) + p.s1 * e1[q];
                const float z1n = kl_prox(v1, __ldg(p.y + n), p.kappa1);
                z1c[n] = z1n;
                if (p.r_out) p.r_out[chain * plane + n] = w - z1n;
                const float z2 = z2c[n];
                const float v2 = z2 - p.a2 * (z2 - __ldg(xc + n)) + p.s2 * e2[q];
                z2c[n] = fmaxf(v2, 0.f);
            }
        }
    }
    if (p.arrive) {
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            if (atomicAdd(p.arrive, 1u) == nblk - 1) {
                *p.arrive = 0u;
                *const_cast<uint32_t*>(p.t_dev) = t + 1u;
            }
        }
    }
}

template <int KW, int R, bool SEP>
__global__ void __launch_bounds__(256) k_zupdate(const ZParams p) {
    zupdate_body<KW, R, SEP>(p, blockIdx.x, blockIdx.y, blockIdx.z,
                             gridDim.x * gridDim.y * gridDim.z);
}

// ---------------------------------------------------------------------------
// Grouped launches (batches of jobs): one launch runs the tiles of several jobs
// that share a kernel width, form and tile shape. The arguments of every job
// travel by value; block b works on the last job j with tile_begin[j] <= b,
// whose tiles are ordered (image, tile row, tile column) as in a per-job
// launch, so every output is the same sum as when the job runs alone.
// ---------------------------------------------------------------------------
template <typename A>
struct StencilTable {
    A a[STENCIL_TABLE_MAXJ];
    uint32_t tile_begin[STENCIL_TABLE_MAXJ];
    int n;
};
constexpr int GRP_R = 4, GRP_BY = 16;   // the grouped launches' tile: 64 x 64 outputs

__device__ __forceinline__ int table_job(const uint32_t* begin, int n, uint32_t b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// (tile column, tile row, image, tiles of the job) of block b of job j
struct TilePos {
    int bx, by, img;
    unsigned nblk;
};
__device__ __forceinline__ TilePos table_tile(uint32_t local, int ny, int nx, int nimg) {
    const uint32_t tx = (uint32_t)(nx + ST_TX - 1) / ST_TX;
    const uint32_t ty = (uint32_t)(ny + GRP_R * GRP_BY - 1) / (GRP_R * GRP_BY);
    const uint32_t per = tx * ty;
    const uint32_t img = local / per, rem = local - img * per;
    TilePos t;
    t.by = (int)(rem / tx);
    t.bx = (int)(rem - (uint32_t)t.by * tx);
    t.img = (int)img;
    t.nblk = per * (uint32_t)nimg;
    return t;
}

template <int KW, bool SEP>
__global__ void __launch_bounds__(256) k_blur_jobs(const __grid_constant__ StencilTable<BlurArgs> T) {
    const int j = table_job(T.tile_begin, T.n, blockIdx.x);
    const BlurArgs& A = T.a[j];
    const TilePos q = table_tile(blockIdx.x - T.tile_begin[j], A.ny, A.nx, A.nimg);
    blur_body<KW, GRP_R, SEP>(A, q.bx, q.by, q.img);
}

template <int KW, bool SEP>
__global__ void __launch_bounds__(256) k_update_jobs(const __grid_constant__ StencilTable<UpdateParams> T) {
    const int j = table_job(T.tile_begin, T.n, blockIdx.x);
    const UpdateParams& p = T.a[j];
    const TilePos q = table_tile(blockIdx.x - T.tile_begin[j], p.ny, p.nx, p.nchain);
    update_body<KW, GRP_R, SEP>(p, q.bx, q.by, q.img, q.nblk);
}

template <int KW, bool SEP>
__global__ void __launch_bounds__(256) k_zupdate_jobs(const __grid_constant__ StencilTable<ZParams> T) {
    const int j = table_job(T.tile_begin, T.n, blockIdx.x);
    const ZParams& p = T.a[j];
    const TilePos q = table_tile(blockIdx.x - T.tile_begin[j], p.ny, p.nx, p.nchain);
    zupdate_body<KW, GRP_R, SEP>(p, q.bx, q.by, q.img, q.nblk);
}

// ---------------------------------------------------------------------------
// Inpainting x-update (Eq. 8 with H = diag(mask), Sec. IV-A): H^T (H x - y) is
// x - y at an observed pixel and 0 at a missing one, so there is no stencil
// and no residual plane. y holds NaN at missing pixels (the mask costs no
// extra bytes). Each thread updates 4 consecutive pixels of one chain:
// 16 B (x, y, d read; x written) during burn-in, 32 B while sampling.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_update_mask(UpdateParams p) {
    const int64_t plane = (int64_t)p.ny * p.nx;
    const int chain = blockIdx.y;
    const int64_t n0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    if (n0 < plane) {
        float inv_n = p.inv_n;
        if (p.burn_dev) {
            const int64_t n = (int64_t)t + 1 - *p.burn_dev;
            inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
        }
        float* xc = p.x + chain * plane;
        const float* dc = p.d ? p.d + chain * plane : nullptr;
        float* mc = p.mean ? p.mean + chain * plane : nullptr;
        float* qc = p.m2 ? p.m2 + chain * plane : nullptr;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        // n0 is a multiple of 4: one Philox group
        if (p.c_noise != 0.f)
            normals_group((uint32_t)(n0 >> 2), t, (uint32_t)chain, p.key0, p.key1, z);
        const bool vec = (plane & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(p.x) | reinterpret_cast<uintptr_t>(p.d) |
                           reinterpret_cast<uintptr_t>(p.r) | reinterpret_cast<uintptr_t>(p.mean) |
                           reinterpret_cast<uintptr_t>(p.m2)) & 15) == 0;
        if (vec) {
            const float4 xv = *reinterpret_cast<const float4*>(xc + n0);
            const float4 yv = __ldg(reinterpret_cast<const float4*>(p.r + n0));
            float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (dc) dv = __ldg(reinterpret_cast<const float4*>(dc + n0));
            float4 v;
            v.x = update1(p, xv.x, isnan(yv.x) ? 0.f : xv.x - yv.x, dv.x, z[0], 0.f);
            v.y = update1(p, xv.y, isnan(yv.y) ? 0.f : xv.y - yv.y, dv.y, z[1], 0.f);
            v.z = update1(p, xv.z, isnan(yv.z) ? 0.f : xv.z - yv.z, dv.z, z[2], 0.f);
            v.w = update1(p, xv.w, isnan(yv.w) ? 0.f : xv.w - yv.w, dv.w, z[3], 0.f);
            *reinterpret_cast<float4*>(xc + n0) = v;
            if (inv_n > 0.f) {
                float4 mo = *reinterpret_cast<const float4*>(mc + n0);
                float4 qo = *reinterpret_cast<const float4*>(qc + n0);
                welford1(v.x, inv_n, mo.x, qo.x);
                welford1(v.y, inv_n, mo.y, qo.y);
                welford1(v.z, inv_n, mo.z, qo.z);
                welford1(v.w, inv_n, mo.w, qo.w);
                *reinterpret_cast<float4*>(mc + n0) = mo;
                *reinterpret_cast<float4*>(qc + n0) = qo;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t n = n0 + q;
                if (n >= plane) break;
                const float xv = xc[n], yv = __ldg(p.r + n);
                const float v = update1(p, xv, isnan(yv) ? 0.f : xv - yv, dc ? __ldg(dc + n) : 0.f,
                                        z[q], 0.f);
                xc[n] = v;
                if (inv_n > 0.f) {
                    float mo = mc[n], qo = qc[n];
                    welford1(v, inv_n, mo, qo);
                    mc[n] = mo;
                    qc[n] = qo;
                }
            }
        }
    }
    if (p.arrive) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
            if (atomicAdd(p.arrive, 1u) == nblk - 1) {
                *p.arrive = 0u;
                *const_cast<uint32_t*>(p.t_dev) = t + 1u;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Wide stencil for large kernels (up to 129 x 129). A block of 32 x 16 threads
// owns a 64-row x 128-column output tile; the window (64 + kh + 2) x (128 +
// kw - 1) is filled once with circular wrap (195 KB at 129 x 129, so one block
// per SM there: 16 warps to hide the shared-memory latency). Thread (tx, ty)
// accumulates rows 4 ty .. 4 ty + 3 at columns tx + 32 q (q = 0..3): for a
// fixed offset the 32 lanes of a warp read 32 consecutive window words, so the
// loads are free of bank conflicts for any pitch. Taps come in groups of four
// on consecutive rows of one window column: a thread loads the 4 + 3 window
// values of a column once and applies all four taps to its 4 rows (16
// multiply-adds per 7 shared-memory loads instead of one per load). Only
// groups holding a nonzero tap are visited (a motion blur of length L has O(L)
// of its L^2 entries). Sums run over window columns in order, rows ascending;
// the operator entry points pass no group list and the kernel walks h in
// groups of four rows itself, in the same order (zero taps add exactly
// nothing), so both give the same sums.
// ---------------------------------------------------------------------------
constexpr int WD_TW = 128, WD_R = 4, WD_BY = 16, WD_TR = WD_R * WD_BY;

static size_t wide_smem(int kh, int kw) {
    return sizeof(float) * (size_t)(WD_TR + kh + 2) * (WD_TW + kw - 1);
}

__device__ __forceinline__ void wide_tile(const float* __restrict__ img, int ny, int nx, int i0,
                                          int j0, int kh, int kw, const WTap* __restrict__ taps,
                                          int ntaps, const float* __restrict__ h, bool adjoint,
                                          float* win, float acc[WD_R][4]) {
    const int ay = kh >> 1, ax = kw >> 1;
    const int wy = WD_TR + kh + 2, wp = WD_TW + kw - 1;   // + 3 rows read by the last group
    // window fill: each row of threads copies whole window rows (circular
    // wrap of the row once per row; columns wrap only on border tiles), all
    // copies asynchronous
    const int c0 = j0 - ax;
    const bool col_interior = c0 >= 0 && c0 + wp <= nx;
    for (int r = threadIdx.y; r < wy; r += WD_BY) {
        int gi = (i0 - ay + r) % ny;
        if (gi < 0) gi += ny;
        const float* src = img + (int64_t)gi * nx;
        float* dst = win + r * wp;
        if (col_interior) {
            for (int c = threadIdx.x; c < wp; c += 32) cp_async4(dst + c, src + c0 + c);
        } else {
            for (int c = threadIdx.x; c < wp; c += 32) {
                int gj = (c0 + c) % nx;
                if (gj < 0) gj += nx;
                cp_async4(dst + c, src + gj);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // accumulators of the column pairs (q, q + 1) = (2 p, 2 p + 1): packed FP32
    // FMAs, each component rounded exactly as fmaf, in the same order
    float2 acc2[WD_R][2];
#pragma unroll
    for (int o = 0; o < WD_R; ++o) acc2[o][0] = acc2[o][1] = make_float2(0.f, 0.f);
    const float* base = win + threadIdx.y * WD_R * wp + threadIdx.x;
    auto group = [&](int off, float w0, float w1, float w2, float w3) {
        const float* b = base + off;
        const float2 t0 = make_float2(w0, w0), t1 = make_float2(w1, w1);
        const float2 t2 = make_float2(w2, w2), t3 = make_float2(w3, w3);
#pragma unroll
        for (int pq = 0; pq < 2; ++pq) {
            float2 v[WD_R + 3];
#pragma unroll
            for (int o = 0; o < WD_R + 3; ++o)
                v[o] = make_float2(b[o * wp + 64 * pq], b[o * wp + 64 * pq + 32]);
#pragma unroll
            for (int o = 0; o < WD_R; ++o) {
                float2 sacc = acc2[o][pq];
                sacc = __ffma2_rn(t0, v[o], sacc);
                sacc = __ffma2_rn(t1, v[o + 1], sacc);
                sacc = __ffma2_rn(t2, v[o + 2], sacc);
                sacc = __ffma2_rn(t3, v[o + 3], sacc);
                acc2[o][pq] = sacc;
            }
        }
    };
    if (taps) {
#pragma unroll 2
        for (int k = 0; k < ntaps; ++k) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(taps[k].w));
            group(__ldg(&taps[k].off), w.x, w.y, w.z, w.w);
        }
    } else {
        // window row wr, column wc hold tap (wr, wc) of the adjoint and tap
        // (2 ay - wr, 2 ax - wc) of the forward operator
        for (int wc = 0; wc < kw; ++wc)
            for (int r0 = 0; r0 < kh; r0 += 4) {
                float w[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int wr = r0 + t;
                    const int a = adjoint ? wr : 2 * ay - wr, b = adjoint ? wc : 2 * ax - wc;
                    w[t] = wr < kh ? __ldg(h + a * kw + b) : 0.f;
                }
                if (w[0] == 0.f && w[1] == 0.f && w[2] == 0.f && w[3] == 0.f) continue;
                group(r0 * wp + wc, w[0], w[1], w[2], w[3]);
            }
    }
#pragma unroll
    for (int o = 0; o < WD_R; ++o) {
        acc[o][0] = acc2[o][0].x;
        acc[o][1] = acc2[o][0].y;
        acc[o][2] = acc2[o][1].x;
        acc[o][3] = acc2[o][1].y;
    }
}

// out = (a (h * x) - y) scale (forward) or scale (h^T x) (adjoint).
__global__ void __launch_bounds__(32 * WD_BY) k_blur_wide(const float* __restrict__ x,
                                                   const float* __restrict__ y,
                                                   const float* __restrict__ h,
                                                   const WTap* __restrict__ taps, int ntaps,
                                                   int kh, int kw, int ny, int nx, float scale,
                                                   int adjoint, float* __restrict__ out, float a,
                                                   int64_t y_img_stride) {
    extern __shared__ float4 sm4[];
    const int64_t plane = (int64_t)ny * nx;
    const int img = blockIdx.z;
    const int i0 = blockIdx.y * WD_TR, j0 = blockIdx.x * WD_TW;
    pdl_wait();
    pdl_launch_dependents();
    float acc[WD_R][4];
    wide_tile(x + img * plane, ny, nx, i0, j0, kh, kw, taps, ntaps, h, adjoint != 0,
              reinterpret_cast<float*>(sm4), acc);
    if (y) y += img * y_img_stride;
#pragma unroll
    for (int o = 0; o < WD_R; ++o) {
        const int i = i0 + threadIdx.y * WD_R + o;
        if (i >= ny) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + threadIdx.x + 32 * q;
            if (j >= nx) continue;
            const int64_t n = (int64_t)i * nx + j;
            float v = a * acc[o][q];
            if (y) v -= __ldg(y + n);
            out[img * plane + n] = v * scale;
        }
    }
}

// Fused x-update with g = H^T r from the wide stencil: the tile's gradient is
// staged in shared memory, then each thread updates 4 consecutive pixels of a
// row (the Philox group layout and 16-byte accesses of k_update).
__global__ void __launch_bounds__(32 * WD_BY) k_update_wide(UpdateParams p) {
    extern __shared__ float4 sm4[];
    float* win = reinterpret_cast<float*>(sm4);
    const int ny = p.ny, nx = p.nx;
    const int64_t plane = (int64_t)ny * nx;
    const int chain = blockIdx.z;
    const int i0 = blockIdx.y * WD_TR, j0 = blockIdx.x * WD_TW;
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    float acc[WD_R][4];
    wide_tile(p.r + chain * plane, ny, nx, i0, j0, p.kh, p.kw, p.wtaps, p.nwtaps, p.h, true, win,
              acc);
    __syncthreads();   // every warp is done with the window: reuse it for the gradient
    float* G = win;    // [WD_TR][WD_TW]
#pragma unroll
    for (int o = 0; o < WD_R; ++o)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            G[(threadIdx.y * WD_R + o) * WD_TW + threadIdx.x + 32 * q] = acc[o][q];
    __syncthreads();
    float inv_n = p.inv_n;
    if (p.burn_dev) {
        const int64_t n = (int64_t)t + 1 - *p.burn_dev;
        inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
    }
    float* xc = p.x + chain * plane;
    const float* dc = p.d ? p.d + chain * plane : nullptr;
    float* mc = p.mean ? p.mean + chain * plane : nullptr;
    float* qc = p.m2 ? p.m2 + chain * plane : nullptr;
    const float* z2c = p.z2 ? p.z2 + chain * plane : nullptr;
    const bool vec = (nx & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(p.x) | reinterpret_cast<uintptr_t>(p.d) |
                       reinterpret_cast<uintptr_t>(p.mean) | reinterpret_cast<uintptr_t>(p.m2) |
                       reinterpret_cast<uintptr_t>(p.z2)) & 15) == 0;
    const int j = j0 + 4 * threadIdx.x;
    for (int o = 0; o < WD_R; ++o) {
        const int li = threadIdx.y * WD_R + o, i = i0 + li;
        if (i >= ny || j >= nx) break;
        const float4 g4 = *reinterpret_cast<const float4*>(G + li * WD_TW + 4 * threadIdx.x);
        const float g[4] = {g4.x, g4.y, g4.z, g4.w};
        const int64_t n0 = (int64_t)i * nx + j;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (p.c_noise != 0.f) normals4(p.key0, p.key1, n0, t, (uint32_t)chain, z);
        if (vec) {
            const float4 xv = *reinterpret_cast<const float4*>(xc + n0);
            float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (dc) dv = __ldg(reinterpret_cast<const float4*>(dc + n0));
            float4 z2v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (z2c) z2v = __ldg(reinterpret_cast<const float4*>(z2c + n0));
            float4 v;
            v.x = update1(p, xv.x, g[0], dv.x, z[0], z2v.x);
            v.y = update1(p, xv.y, g[1], dv.y, z[1], z2v.y);
            v.z = update1(p, xv.z, g[2], dv.z, z[2], z2v.z);
            v.w = update1(p, xv.w, g[3], dv.w, z[3], z2v.w);
            *reinterpret_cast<float4*>(xc + n0) = v;
            if (inv_n > 0.f) {
                float4 mo = *reinterpret_cast<const float4*>(mc + n0);
                float4 qo = *reinterpret_cast<const float4*>(qc + n0);
                welford1(v.x, inv_n, mo.x, qo.x);
                welford1(v.y, inv_n, mo.y, qo.y);
                welford1(v.z, inv_n, mo.z, qo.z);
                welford1(v.w, inv_n, mo.w, qo.w);
                *reinterpret_cast<float4*>(mc + n0) = mo;
                *reinterpret_cast<float4*>(qc + n0) = qo;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (j + q >= nx) break;
                const int64_t n = n0 + q;
                const float v = update1(p, xc[n], g[q], dc ? __ldg(dc + n) : 0.f, z[q],
                                        z2c ? __ldg(z2c + n) : 0.f);
                xc[n] = v;
                if (inv_n > 0.f) {
                    float mo = mc[n], qo = qc[n];
                    welford1(v, inv_n, mo, qo);
                    mc[n] = mo;
                    qc[n] = qo;
                }
            }
        }
    }
    if (p.arrive) {
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
            if (atomicAdd(p.arrive, 1u) == nblk - 1) {
                *p.arrive = 0u;
                *const_cast<uint32_t*>(p.t_dev) = t + 1u;
            }
        }
    }
}

std::vector<WTap> wide_taps(const float* h, int kh, int kw, bool adjoint) {
    const int wp = WD_TW + kw - 1, ay = kh / 2, ax = kw / 2;
    auto tap = [&](int wr, int wc) {
        if (wr >= kh) return 0.f;
        const int a = adjoint ? wr : 2 * ay - wr, b = adjoint ? wc : 2 * ax - wc;
        return h[a * kw + b];
    };
    std::vector<WTap> t;
    for (int wc = 0; wc < kw; ++wc)
        for (int wr = 0; wr < kh;) {
            if (tap(wr, wc) == 0.f) {
                ++wr;
                continue;
            }
            WTap g = {};
            for (int q = 0; q < 4; ++q) g.w[q] = tap(wr + q, wc);
            g.off = wr * wp + wc;
            t.push_back(g);
            wr += 4;
        }
    return t;
}

// ------------------------------------------------------------ dispatch

using BlurFn = void (*)(BlurArgs);
using UpdFn = void (*)(UpdateParams);
using ZFn = void (*)(ZParams);

template <int KW>
static BlurFn blur_fn_r(int R, bool sep) {
    if (sep) return R == 1 ? k_blur<KW, 1, true> : R == 2 ? k_blur<KW, 2, true> : k_blur<KW, 4, true>;
    return R == 1 ? k_blur<KW, 1, false> : R == 2 ? k_blur<KW, 2, false> : k_blur<KW, 4, false>;
}
template <int KW>
static ZFn z_fn_r(int R, bool sep) {
    if (sep) return R == 1 ? k_zupdate<KW, 1, true> : R == 2 ? k_zupdate<KW, 2, true> : k_zupdate<KW, 4, true>;
    return R == 1 ? k_zupdate<KW, 1, false> : R == 2 ? k_zupdate<KW, 2, false> : k_zupdate<KW, 4, false>;
}
template <int KW>
static UpdFn upd_fn_r(int R, bool sep) {
    if (sep) return R == 1 ? k_update<KW, 1, true> : R == 2 ? k_update<KW, 2, true> : k_update<KW, 4, true>;
    return R == 1 ? k_update<KW, 1, false> : R == 2 ? k_update<KW, 2, false> : k_update<KW, 4, false>;
}

#define PNP_KW_CASES(F)                                                                        \
    switch (kw) {                                                                              \
    case 1: return F<1>(R, sep);   case 3: return F<3>(R, sep);   case 5: return F<5>(R, sep); \
    case 7: return F<7>(R, sep);   case 9: return F<9>(R, sep);   case 11: return F<11>(R, sep); \
    case 13: return F<13>(R, sep); case 15: return F<15>(R, sep); case 17: return F<17>(R, sep); \
    case 19: return F<19>(R, sep); case 21: return F<21>(R, sep); case 23: return F<23>(R, sep); \
    case 25: return F<25>(R, sep); case 27: return F<27>(R, sep); case 29: return F<29>(R, sep); \
    case 31: return F<31>(R, sep);                                                             \
    default: return nullptr;                                                                   \
    }

static BlurFn blur_fn(int kw, int R, bool sep) { PNP_KW_CASES(blur_fn_r) }
static UpdFn upd_fn(int kw, int R, bool sep) { PNP_KW_CASES(upd_fn_r) }
static ZFn z_fn(int kw, int R, bool sep) { PNP_KW_CASES(z_fn_r) }

using BlurJFn = void (*)(StencilTable<BlurArgs>);
using UpdJFn = void (*)(StencilTable<UpdateParams>);
using ZJFn = void (*)(StencilTable<ZParams>);
template <int KW>
static BlurJFn blurj_fn_r(int, bool sep) { return sep ? k_blur_jobs<KW, true> : k_blur_jobs<KW, false>; }
template <int KW>
static UpdJFn updj_fn_r(int, bool sep) { return sep ? k_update_jobs<KW, true> : k_update_jobs<KW, false>; }
template <int KW>
static ZJFn zj_fn_r(int, bool sep) { return sep ? k_zupdate_jobs<KW, true> : k_zupdate_jobs<KW, false>; }
static BlurJFn blurj_fn(int kw, bool sep) { const int R = 0; PNP_KW_CASES(blurj_fn_r) }
static UpdJFn updj_fn(int kw, bool sep) { const int R = 0; PNP_KW_CASES(updj_fn_r) }
static ZJFn zj_fn(int kw, bool sep) { const int R = 0; PNP_KW_CASES(zj_fn_r) }
#undef PNP_KW_CASES

// Tiles whose shared memory exceeds the 48 KB default need the opt-in, once
// per kernel.
template <typename Fn>
static cudaError_t allow_smem(Fn fn, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<const void*, size_t> done;
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = done[reinterpret_cast<const void*>(fn)];
    if (smem <= have) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) have = smem;
    return e;
}

// the tile a launch uses: the forced one if set, else the caller's choice
static int resolve_tile(int tile) {
    const int f = g_forced_tile.load();
    if (f >= 0) return f;
    return (tile >= 0 && tile < kNumTiles) ? tile : 0;
}

static cudaError_t blur_raw(const float* x, const float* y, const float* h, const float* hsep,
                            int kh, int kw, int ny, int nx, int nimg, float scale, bool adjoint,
                            float* out, int tile, cudaStream_t s, float a = 1.0f,
                            int64_t y_img_stride = 0) {
    const TileShape ts = kTiles[tile];
    const int rows = ts.R * ts.BY;
    const bool sep = hsep != nullptr;
    BlurFn fn = blur_fn(kw, ts.R, sep);
    if (!fn || kh > ST_MAXK) return cudaErrorInvalidValue;
    const size_t smem = tile_smem(kw, kh, rows, sep);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(nx, ST_TX), ceil_div(ny, rows), nimg);
    BlurArgs A{x, y, sep ? hsep : h, kh, ny, nx, nimg, scale, adjoint ? 1 : 0, out, a, y_img_stride};
    return launch_pdl(fn, grid, dim3(16, ts.BY), smem, s, A);
}

static cudaError_t zupdate_raw(const ZParams& p, int tile, cudaStream_t s) {
    const TileShape ts = kTiles[tile];
    const int rows = ts.R * ts.BY;
    const bool sep = p.hsep != nullptr;
    ZFn fn = z_fn(p.kw, ts.R, sep);
    if (!fn || p.kh > ST_MAXK) return cudaErrorInvalidValue;
    const size_t smem = tile_smem(p.kw, p.kh, rows, sep);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(p.nx, ST_TX), ceil_div(p.ny, rows), p.nchain);
    return launch_pdl(fn, grid, dim3(16, ts.BY), smem, s, p);
}

static cudaError_t update_raw(const UpdateParams& p, int tile, cudaStream_t s) {
    const TileShape ts = kTiles[tile];
    const int rows = ts.R * ts.BY;
    const bool sep = p.hsep != nullptr;
    if (p.os && sep) {
        // one-pass form: the pipelined kernel when the form fits it
        const cudaError_t e = launch_update_os(p, tile, s);
        if (e != cudaErrorNotSupported) return e;
    }
    UpdFn fn = upd_fn(p.kw, ts.R, sep);
    if (!fn || p.kh > ST_MAXK) return cudaErrorInvalidValue;
    const size_t smem = tile_smem(p.kw, p.kh, rows, sep);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(p.nx, ST_TX), ceil_div(p.ny, rows), p.nchain);
    return launch_pdl(fn, grid, dim3(16, ts.BY), smem, s, p);
}

static cudaError_t blur_wide(const float* x, const float* y, const float* h, const WTap* wt,
                             int nwt, int kh, int kw, int ny, int nx, int nimg, float scale,
                             bool adjoint, float* out, cudaStream_t s, float a,
                             int64_t y_img_stride) {
    if (kh > WIDE_MAXK || kw > WIDE_MAXK) return cudaErrorInvalidValue;
    const size_t smem = wide_smem(kh, kw);
    cudaError_t e = allow_smem(k_blur_wide, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(nx, WD_TW), ceil_div(ny, WD_TR), nimg);
    return launch_pdl(k_blur_wide, grid, dim3(32, WD_BY), smem, s, x, y, h, wt, nwt, kh, kw, ny,
                      nx, scale, adjoint ? 1 : 0, out, a, y_img_stride);
}

cudaError_t launch_blur(const float* x, const float* y, const float* h, int kh, int kw, int ny,
                        int nx, int nimg, float* r, cudaStream_t s, int tile, const float* hsep,
                        float a, int64_t y_img_stride, const WTap* wt, int nwt) {
    timer_begin(T_BLUR, s);
    cudaError_t e = is_wide(kh, kw)
        ? blur_wide(x, y, h, wt, nwt, kh, kw, ny, nx, nimg, 1.0f, false, r, s, a, y_img_stride)
        : blur_raw(x, y, h, hsep, kh, kw, ny, nx, nimg, 1.0f, false, r, resolve_tile(tile), s, a,
                   y_img_stride);
    timer_end(T_BLUR, s);
    return e;
}

cudaError_t launch_blur_adjoint(const float* r, const float* h, int kh, int kw, int ny, int nx,
                                int nimg, float scale, float* g, cudaStream_t s, int tile) {
    if (is_wide(kh, kw))
        return blur_wide(r, nullptr, h, nullptr, 0, kh, kw, ny, nx, nimg, scale, true, g, s, 1.0f, 0);
    return blur_raw(r, nullptr, h, nullptr, kh, kw, ny, nx, nimg, scale, true, g,
                    resolve_tile(tile), s);
}

static cudaError_t update_wide(const UpdateParams& p, cudaStream_t s) {
    if (p.kh > WIDE_MAXK || p.kw > WIDE_MAXK) return cudaErrorInvalidValue;
    const size_t smem = wide_smem(p.kh, p.kw);
    cudaError_t e = allow_smem(k_update_wide, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(p.nx, WD_TW), ceil_div(p.ny, WD_TR), p.nchain);
    return launch_pdl(k_update_wide, grid, dim3(32, WD_BY), smem, s, p);
}

cudaError_t launch_langevin_update(const UpdateParams& p, cudaStream_t s) {
    timer_begin(T_UPDATE, s);
    cudaError_t e = is_wide(p.kh, p.kw) ? update_wide(p, s) : update_raw(p, resolve_tile(p.tile), s);
    timer_end(T_UPDATE, s);
    return e;
}

cudaError_t launch_update_mask(const UpdateParams& p, cudaStream_t s) {
    timer_begin(T_UPDATE, s);
    const int64_t plane = (int64_t)p.ny * p.nx;
    const int64_t groups = (plane + 3) / 4;
    dim3 grid((unsigned)((groups + 255) / 256), p.nchain, 1);
    cudaError_t e = launch_pdl(k_update_mask, grid, dim3(256), 0, s, p);
    timer_end(T_UPDATE, s);
    return e;
}

cudaError_t launch_zupdate(const ZParams& p, cudaStream_t s) {
    timer_begin(T_ZUPDATE, s);
    cudaError_t e = zupdate_raw(p, resolve_tile(p.tile), s);
    timer_end(T_ZUPDATE, s);
    return e;
}

// Grouped launch of jobs sharing kernel width kw and form (sep); chunks of
// STENCIL_TABLE_MAXJ jobs per launch. tiles(a) = a job's tile count, kh(a) its
// kernel height (the shared memory is sized for the tallest).
template <typename A, typename Fn, typename Tiles, typename Kh>
static cudaError_t launch_group(Fn fn, const A* jobs, int n, int kw, bool sep, cudaStream_t s,
                                Tiles tiles, Kh kh_of) {
    if (!fn) return cudaErrorInvalidValue;
    for (int c0 = 0; c0 < n; c0 += STENCIL_TABLE_MAXJ) {
        StencilTable<A> T;
        memset(&T, 0, sizeof(T));
        uint64_t total = 0;
        int khmax = 1;
        for (int k = c0; k < std::min(n, c0 + STENCIL_TABLE_MAXJ); ++k) {
            T.a[T.n] = jobs[k];
            T.tile_begin[T.n] = (uint32_t)total;
            total += tiles(jobs[k]);
            khmax = std::max(khmax, kh_of(jobs[k]));
            ++T.n;
        }
        if (total == 0) continue;
        if (total >= (1ull << 31) || khmax > ST_MAXK) return cudaErrorInvalidValue;
        const size_t smem = tile_smem(kw, khmax, GRP_R * GRP_BY, sep);
        cudaError_t e = allow_smem(fn, smem);
        if (e != cudaSuccess) return e;
        e = launch_pdl(fn, dim3((unsigned)total), dim3(16, GRP_BY), smem, s, T);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static uint64_t group_tiles(int ny, int nx, int nimg) {
    return (uint64_t)ceil_div(nx, ST_TX) * ceil_div(ny, GRP_R * GRP_BY) * (uint64_t)nimg;
}

cudaError_t launch_blur_group(const BlurArgs* jobs, int n, int kw, bool sep, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    timer_begin(T_BLUR, s);
    cudaError_t e = launch_group(blurj_fn(kw, sep), jobs, n, kw, sep, s,
                                 [](const BlurArgs& a) { return group_tiles(a.ny, a.nx, a.nimg); },
                                 [](const BlurArgs& a) { return a.kh; });
    timer_end(T_BLUR, s);
    return e;
}

cudaError_t launch_update_group(const UpdateParams* jobs, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const bool sep = jobs[0].hsep != nullptr;
    timer_begin(T_UPDATE, s);
    cudaError_t e = launch_group(updj_fn(jobs[0].kw, sep), jobs, n, jobs[0].kw, sep, s,
                                 [](const UpdateParams& p) { return group_tiles(p.ny, p.nx, p.nchain); },
                                 [](const UpdateParams& p) { return p.kh; });
    timer_end(T_UPDATE, s);
    return e;
}

cudaError_t launch_zupdate_group(const ZParams* jobs, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const bool sep = jobs[0].hsep != nullptr;
    timer_begin(T_ZUPDATE, s);
    cudaError_t e = launch_group(zj_fn(jobs[0].kw, sep), jobs, n, jobs[0].kw, sep, s,
                                 [](const ZParams& p) { return group_tiles(p.ny, p.nx, p.nchain); },
                                 [](const ZParams& p) { return p.kh; });
    timer_end(T_ZUPDATE, s);
    return e;
}

int stencil_tile_count() { return kNumTiles; }

bool set_forced_stencil_tile(int tile) {
    if (tile < -1 || tile >= kNumTiles) return false;
    g_forced_tile = tile;
    return true;
}

// ------------------------------------------------------------ autotuner

// Times every tile shape for r = Hx - y and for the update on the problem's own
// buffers and returns the fastest of each. The update candidates overwrite x,
// mean and m2 (callers initialise them afterwards). Choices are cached per
// (ny, nx, kh, kw, nimg, separable): every shape gives bitwise the same
// results, so the cache only saves the timing.
cudaError_t stencil_autotune(const float* x, const float* y, const float* h, const float* hsep,
                             int kh, int kw, int ny, int nx, int nimg, float* r,
                             const UpdateParams& u, cudaStream_t s, int* blur_tile,
                             int* update_tile) {
    using Key = std::tuple<int, int, int, int, int, bool, bool>;
    static std::mutex mu;
    static std::map<Key, std::pair<int, int>> cache;
    const Key key{ny, nx, kh, kw, nimg, hsep != nullptr, u.qb != nullptr};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *blur_tile = it->second.first;
            *update_tile = it->second.second;
            return cudaSuccess;
        }
    }
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    // two rounds over the shapes, 8 timed launches each, best of the rounds:
    // the kernels of a small image take ~10 us, so single timings are noisy
    constexpr int reps = 8, rounds = 2;
    float tb[kNumTiles], tu[kNumTiles];
    for (int c = 0; c < kNumTiles; ++c) tb[c] = tu[c] = 1e30f;
    for (int rd = 0; rd < rounds && e == cudaSuccess; ++rd) {
        for (int c = 0; c < kNumTiles && e == cudaSuccess; ++c) {
            // a one-pass problem (u.qb set) launches no blur: only its update is timed
            for (int kind = u.qb ? 1 : 0; kind < 2 && e == cudaSuccess; ++kind) {
                for (int it = 0; it <= reps && e == cudaSuccess; ++it) {
                    if (it == 1) e = cudaEventRecord(e0, s);
                    if (e != cudaSuccess) break;
                    e = kind == 0 ? blur_raw(x, y, h, hsep, kh, kw, ny, nx, nimg, 1.0f, false, r, c, s)
                                  : update_raw(u, c, s);
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) break;
                float& best = kind == 0 ? tb[c] : tu[c];
                best = ms < best ? ms : best;
            }
        }
    }
    int bt = 0, ut = 0;
    for (int c = 1; c < kNumTiles; ++c) {
        if (tb[c] < tb[bt]) bt = c;
        if (tu[c] < tu[ut]) ut = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {bt, ut};
    *blur_tile = bt;
    *update_tile = ut;
    return cudaSuccess;
}

// ------------------------------------------------------------ final moments

__global__ void k_finalize(const float* __restrict__ mean, const float* __restrict__ m2,
                           int64_t npix, int64_t n_kept, int want_var, double* __restrict__ mmse,
                           double* __restrict__ out2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    mmse[i] = (double)mean[i];
    const double var = n_kept > 1 ? (double)m2[i] / (double)(n_kept - 1) : 0.0;
    out2[i] = want_var ? var : sqrt(var);
}

cudaError_t launch_finalize_moments(const float* mean, const float* m2, int64_t npix,
                                    int64_t n_kept, int want_var, double* mmse, double* out2,
                                    cudaStream_t s) {
    note_launch();
    k_finalize<<<ceil_div(npix, 256), 256, 0, s>>>(mean, m2, npix, n_kept, want_var, mmse, out2);
    return cudaGetLastError();
}

}  // namespace pnp
