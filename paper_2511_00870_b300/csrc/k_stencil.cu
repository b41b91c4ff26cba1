// Blur operator H, its adjoint, the fused PnP-ULA update and the final moments.
//
// H is the circular 2-D convolution of the Gaussian-deconvolution likelihood
// (Sec. III-A2): (h * x)[i,j] = sum_{a,b} h[a,b] x[i-a+ry, j-b+rx] (indices mod
// the image size). H^T is the correlation sum_{a,b} h[a,b] r[i+a-ry, j+b-rx].
// Both are evaluated as a correlation over a shared-memory tile that holds the
// output tile plus a (kh-1) x (kw-1) circular halo; the forward operator just
// uses the flipped kernel. Every output is a fixed-order sum over (a, b), so
// results do not depend on the tile shape or the launch.
#include "philox.cuh"
#include "pnp_internal.h"

namespace pnp {

constexpr int ST_TX = 64;    // tile width  (outputs)
constexpr int ST_TY = 16;    // tile height (outputs)
constexpr int ST_THREADS = 256;   // 16 x 16, 4 consecutive outputs per thread
constexpr int ST_MAXK = 31;

struct StencilSmem {
    int pitch;
};

// Load the (ST_TY + kh - 1) x (ST_TX + kw - 1) circular window whose top-left
// image coordinate is (i0 - ry, j0 - rx), and the kernel (flipped if `flip`).
__device__ __forceinline__ void load_window(const float* __restrict__ img, int ny, int nx, int i0,
                                            int j0, int kh, int kw, float* win, int pitch,
                                            const float* __restrict__ h, float* hs, bool flip) {
    const int ry = kh / 2, rx = kw / 2;
    const int wy = ST_TY + kh - 1, wx = ST_TX + kw - 1;
    for (int e = threadIdx.x; e < wy * wx; e += blockDim.x) {
        const int u = e / wx, v = e - u * wx;
        int gi = i0 - ry + u, gj = j0 - rx + v;
        gi %= ny; if (gi < 0) gi += ny;
        gj %= nx; if (gj < 0) gj += nx;
        win[u * pitch + v] = __ldg(img + (int64_t)gi * nx + gj);
    }
    const int kk = kh * kw;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) hs[e] = __ldg(h + (flip ? kk - 1 - e : e));
}

// acc[q] = sum_{a,b} hs[a,b] win[di + a][dj + q + b], q = 0..3
__device__ __forceinline__ void correlate4(const float* win, int pitch, const float* hs, int kh,
                                           int kw, int di, int dj, float acc[4]) {
    acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
    for (int a = 0; a < kh; ++a) {
        const float* row = win + (di + a) * pitch + dj;
        const float* hr = hs + a * kw;
        float w0 = row[0], w1 = row[1], w2 = row[2];
        for (int b = 0; b < kw; ++b) {
            const float w3 = row[b + 3];
            const float hv = hr[b];
            acc[0] = fmaf(hv, w0, acc[0]);
            acc[1] = fmaf(hv, w1, acc[1]);
            acc[2] = fmaf(hv, w2, acc[2]);
            acc[3] = fmaf(hv, w3, acc[3]);
            w0 = w1; w1 = w2; w2 = w3;
        }
    }
}

__global__ void __launch_bounds__(ST_THREADS) k_blur(const float* __restrict__ x,
                                                     const float* __restrict__ y,
                                                     const float* __restrict__ h, int kh, int kw,
                                                     int ny, int nx, float scale, bool adjoint,
                                                     float* __restrict__ out) {
    extern __shared__ float sm[];
    const int pitch = ST_TX + kw - 1 + 1;
    float* win = sm;
    float* hs = sm + (ST_TY + kh - 1) * pitch;
    const int64_t plane = (int64_t)ny * nx;
    const int img = blockIdx.z;
    const int i0 = blockIdx.y * ST_TY, j0 = blockIdx.x * ST_TX;
    // forward H: correlation with the flipped kernel; adjoint: with h itself
    load_window(x + img * plane, ny, nx, i0, j0, kh, kw, win, pitch, h, hs, !adjoint);
    __syncthreads();
    const int di = threadIdx.x / (ST_TX / 4), dj = (threadIdx.x % (ST_TX / 4)) * 4;
    const int i = i0 + di;
    if (i >= ny) return;
    float acc[4];
    correlate4(win, pitch, hs, kh, kw, di, dj, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + dj + q;
        if (j < nx) {
            const int64_t n = (int64_t)i * nx + j;
            float v = acc[q];
            if (y) v -= __ldg(y + n);
            out[img * plane + n] = v * scale;
        }
    }
}

static size_t stencil_smem(int kh, int kw) {
    const int pitch = ST_TX + kw - 1 + 1;
    return sizeof(float) * ((size_t)(ST_TY + kh - 1) * pitch + kh * kw);
}

cudaError_t launch_blur(const float* x, const float* y, const float* h, int kh, int kw, int ny,
                        int nx, int nimg, float* r, cudaStream_t s) {
    dim3 grid(ceil_div(nx, ST_TX), ceil_div(ny, ST_TY), nimg);
    timer_begin(T_BLUR, s);
    k_blur<<<grid, ST_THREADS, stencil_smem(kh, kw), s>>>(x, y, h, kh, kw, ny, nx, 1.0f, false, r);
    timer_end(T_BLUR, s);
    return cudaGetLastError();
}

cudaError_t launch_blur_adjoint(const float* r, const float* h, int kh, int kw, int ny, int nx,
                                int nimg, float scale, float* g, cudaStream_t s) {
    dim3 grid(ceil_div(nx, ST_TX), ceil_div(ny, ST_TY), nimg);
    k_blur<<<grid, ST_THREADS, stencil_smem(kh, kw), s>>>(r, nullptr, h, kh, kw, ny, nx, scale,
                                                          true, g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused x-update (Eq. 8): g = H^T r / sigma^2 from the shared-memory window
// of r, then x+ = x - gamma g + c_prior (d - x) + c_proj (clamp(x) - x)
// + c_noise xi and, when sampling, the FP32 Welford step
// delta = x+ - mean; mean += delta / n; m2 += delta (x+ - mean).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ST_THREADS) k_update(UpdateParams p) {
    extern __shared__ float sm[];
    const int kh = p.kh, kw = p.kw, ny = p.ny, nx = p.nx;
    const int pitch = ST_TX + kw - 1 + 1;
    float* win = sm;
    float* hs = sm + (ST_TY + kh - 1) * pitch;
    const int64_t plane = (int64_t)ny * nx;
    const int chain = blockIdx.z;
    const int i0 = blockIdx.y * ST_TY, j0 = blockIdx.x * ST_TX;
    load_window(p.r + chain * plane, ny, nx, i0, j0, kh, kw, win, pitch, p.h, hs, false);
    __syncthreads();
    const int di = threadIdx.x / (ST_TX / 4), dj = (threadIdx.x % (ST_TX / 4)) * 4;
    const int i = i0 + di;
    if (i >= ny || j0 + dj >= nx) return;
    float g[4];
    correlate4(win, pitch, hs, kh, kw, di, dj, g);

    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    float inv_n = p.inv_n;
    if (p.burn_dev) {
        const int64_t n = (int64_t)t + 1 - *p.burn_dev;
        inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
    }
    // Normals for the 4 pixels n0..n0+3 (flat row-major index); they span
    // at most two Philox groups.
    const int64_t n0 = (int64_t)i * nx + j0 + dj;
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (p.c_noise != 0.f) {
        const uint32_t m0 = (uint32_t)(n0 >> 2);
        float za[4], zb[4];
        normals_group(m0, t, (uint32_t)chain, p.key0, p.key1, za);
        const int off = (int)(n0 & 3);
        if (off == 0) {
            z[0] = za[0]; z[1] = za[1]; z[2] = za[2]; z[3] = za[3];
        } else {
            normals_group(m0 + 1, t, (uint32_t)chain, p.key0, p.key1, zb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = off + q;
                const float a = k == 0 ? za[0] : k == 1 ? za[1] : k == 2 ? za[2] : za[3];
                const float b = k == 4 ? zb[0] : k == 5 ? zb[1] : zb[2];
                z[q] = k < 4 ? a : b;
            }
        }
    }
    float* xc = p.x + chain * plane;
    const float* dc = p.d ? p.d + chain * plane : nullptr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + dj + q;
        if (j >= nx) break;
        const int64_t n = (int64_t)i * nx + j;
        const float xv = xc[n];
        float v = xv - p.gamma * (g[q] * p.inv_s2);
        if (dc) v += p.d_residual ? -p.c_prior * __ldg(dc + n) : p.c_prior * (__ldg(dc + n) - xv);
        const float pr = fminf(fmaxf(xv, 0.f), 1.f);
        v += p.c_proj * (pr - xv);
        v += p.c_noise * z[q];
        xc[n] = v;
        if (inv_n > 0.f) {
            float* mc = p.mean + chain * plane;
            float* qc = p.m2 + chain * plane;
            const float mo = mc[n];
            const float delta = v - mo;
            const float mn = mo + delta * inv_n;
            mc[n] = mn;
            qc[n] = qc[n] + delta * (v - mn);
        }
    }
}

cudaError_t launch_langevin_update(const UpdateParams& p, cudaStream_t s) {
    dim3 grid(ceil_div(p.nx, ST_TX), ceil_div(p.ny, ST_TY), p.nchain);
    timer_begin(T_UPDATE, s);
    k_update<<<grid, ST_THREADS, stencil_smem(p.kh, p.kw), s>>>(p);
    timer_end(T_UPDATE, s);
    return cudaGetLastError();
}

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
    k_finalize<<<ceil_div(npix, 256), 256, 0, s>>>(mean, m2, npix, n_kept, want_var, mmse, out2);
    return cudaGetLastError();
}

}  // namespace pnp
