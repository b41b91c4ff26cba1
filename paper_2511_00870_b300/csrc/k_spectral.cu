// Spectral gradient for the large (motion) blurs of Sec. IV-A.
//
// Under Gaussian noise the likelihood gradient is H^T (H x - y) / sigma^2 =
// ((H^T H) x - H^T y) / sigma^2, and H^T H, a circular convolution, is
// diagonal in the 2-D discrete Fourier basis: (H^T H) x = F^-1(|H^|^2 F(x)),
// with H^ = F(h placed circularly at the origin). For kernels of 65^2 to 129^2
// taps a direct stencil costs hundreds of FMAs per pixel; through the FFT the
// cost does not depend on the kernel. Per iteration:
//   K1  k_sp_rows_fwd_real  rows 2q and 2q + 1 of x as one complex row, its
//                           FFT split into the two rows' half spectra
//                           (nx / 2 columns: the DC and Nyquist terms, both
//                           real, share column 0), written in the panel layout;
//   K2  k_sp_cols           per pair of half-spectrum columns: forward FFT down
//                           the column, multiply by P = |H^|^2 / (2 ny nx) (for
//                           column 0 after separating its DC and Nyquist
//                           sequences), inverse FFT;
//   K3  k_sp_update         per row pair the full spectrum A' + i B' rebuilt
//                           from the half spectra, one inverse FFT, g = its
//                           real / imaginary part - H^T y, then the x-update,
//                           noise and Welford step of k_update's aligned path
//                           (update1 / welford1 / normals_group), x in place.
// H^T y is formed once per problem by the direct adjoint stencil, and P once
// from the full spectrum of the embedded kernel (k_sp_rows_fwd and k_sp_cols
// on complex rows).
//
// FFTs of length N = 2^m (64 <= N <= 4096) run in shared memory as Stockham
// stages of radix 16 (and one of radix 2, 4 or 8 for the remaining factor):
// stage (R, L) takes a[j + r N/R] (r < R) for each j < N/R, multiplies term r
// by w^(r k) with w = exp(-+2 pi i / (L R)) and k = j mod L, applies the
// R-point DFT (radix-2 decimation in time in registers, constant twiddles)
// and writes output s to (j div L) L R + k + s L. After the last stage the
// result is in natural order. Every thread holds 16 values per stage (16 / R
// groups), so a length-N transform uses N / 16 threads. Shared-memory index n
// is stored at n + n / 16 so that the first stage's stride-16 writes do not
// all fall on one bank. Twiddles w^n = exp(-2 pi i n / N) come from a table
// computed in FP64 on the host: a group reads w^k and w^(4 k) and forms the
// other powers it needs by at most three complex products.
//
// Spectrum layout ("panels" of 4 columns): element (r, c) of an ny x nx
// spectrum sits at ((c / 4) ny + r) 4 + c % 4, so a row is written and read
// as 32-byte pieces and a pair of columns is one contiguous run of 16-byte
// pieces.
#include "pdl.cuh"
#include "stencil_dev.cuh"

#include <cmath>
#include <vector>

namespace pnp {
namespace {

constexpr int SP_PANEL = 4;

__device__ __forceinline__ int pad16(int n) { return n + (n >> 4); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// cos and sin of 2 pi j / 16, j = 0..7
__host__ __device__ constexpr float c16(int j) {
    return j == 0 ? 1.0f
         : j == 1 ? 0.92387953251128674f
         : j == 2 ? 0.70710678118654752f
         : j == 3 ? 0.38268343236508977f
         : j == 4 ? 0.0f
         : j == 5 ? -0.38268343236508977f
         : j == 6 ? -0.70710678118654752f
                  : -0.92387953251128674f;
}
__host__ __device__ constexpr float s16(int j) {
    return j == 0 ? 0.0f
         : j == 1 ? 0.38268343236508977f
         : j == 2 ? 0.70710678118654752f
         : j == 3 ? 0.92387953251128674f
         : j == 4 ? 1.0f
         : j == 5 ? 0.92387953251128674f
         : j == 6 ? 0.70710678118654752f
                  : 0.38268343236508977f;
}

// In-register R-point DFT (R = 2, 4, 8, 16) in natural order, kernel
// exp(SIGN 2 pi i j k / R): radix-2 decimation in time,
// X[k] = E[k] + w^k O[k], X[k + R/2] = E[k] - w^k O[k].
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2* v) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = make_float2(a.x + b.x, a.y + b.y);
        v[1] = make_float2(a.x - b.x, a.y - b.y);
    } else {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft_reg<R / 2, SIGN>(e);
        dft_reg<R / 2, SIGN>(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            float2 t;
            if (k == 0) {
                t = o[0];
            } else if (4 * k == R) {
                // w^k = SIGN i
                t = SIGN < 0 ? make_float2(o[k].y, -o[k].x) : make_float2(-o[k].y, o[k].x);
            } else {
                const float c = c16(k * 16 / R), s = SIGN * s16(k * 16 / R);
                t = make_float2(o[k].x * c - o[k].y * s, o[k].x * s + o[k].y * c);
            }
            v[k] = make_float2(e[k].x + t.x, e[k].y + t.y);
            v[k + R / 2] = make_float2(e[k].x - t.x, e[k].y - t.y);
        }
    }
}

// One Stockham stage of radix R on a length-N transform in shared memory,
// by the nthr = N / 16 threads of one transform (tid < nthr). Synchronises
// the whole block twice: every thread of the block must call it.
template <int R, int SIGN>
__device__ __forceinline__ void sp_stage(float2* buf, int N, int L, int lgL,
                                         const float2* __restrict__ tw, int tid, int nthr) {
    constexpr int G = 16 / R;
    const int NR = N / R;
    float2 v[G][R];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = tid + g * nthr;
#pragma unroll
        for (int r = 0; r < R; ++r) v[g][r] = buf[pad16(j + r * NR)];
    }
    __syncthreads();
    const int step = N / (L * R);   // table stride of exp(-2 pi i / (L R))
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = tid + g * nthr;
        const int k = j & (L - 1);
        if (L > 1) {
            // w^(r k) for r < R from the table entries w^k and w^(4 k) (each
            // power within three complex products of them)
            float2 w1 = __ldg(tw + k * step);
            float2 w4 = R > 4 ? __ldg(tw + 4 * k * step) : w1;
            if (SIGN > 0) {
                w1.y = -w1.y;
                w4.y = -w4.y;
            }
            const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
            const float2 w8 = cmul(w4, w4), w12 = cmul(w8, w4);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int lo = r & 3, hi = r >> 2;
                const float2 wl = lo == 1 ? w1 : lo == 2 ? w2 : w3;
                const float2 wh = hi == 1 ? w4 : hi == 2 ? w8 : w12;
                const float2 w = hi == 0 ? wl : lo == 0 ? wh : cmul(wh, wl);
                v[g][r] = cmul(v[g][r], w);
            }
        }
        dft_reg<R, SIGN>(v[g]);
        const int base = ((j >> lgL) << lgL) * R + k;
#pragma unroll
        for (int s = 0; s < R; ++s) buf[pad16(base + s * L)] = v[g][s];
    }
    __syncthreads();
}

// Length-N (N = 2^lgN, 16 <= N) transform of buf in place, natural order in
// and out; the caller synchronises after filling buf.
template <int SIGN>
__device__ __forceinline__ void sp_fft(float2* buf, int N, int lgN, const float2* __restrict__ tw,
                                       int tid, int nthr) {
    int L = 1, lgL = 0, m = lgN;
    while (m >= 4) {
        sp_stage<16, SIGN>(buf, N, L, lgL, tw, tid, nthr);
        L <<= 4;
        lgL += 4;
        m -= 4;
    }
    if (m == 3) sp_stage<8, SIGN>(buf, N, L, lgL, tw, tid, nthr);
    else if (m == 2) sp_stage<4, SIGN>(buf, N, L, lgL, tw, tid, nthr);
    else if (m == 1) sp_stage<2, SIGN>(buf, N, L, lgL, tw, tid, nthr);
}

// Forward FFT of each row (r = blockIdx.x) of image blockIdx.y of x,
// imaginary part 0, into the full panel layout of Z (the kernel's spectrum at
// setup). nx / 16 threads.
__global__ void __launch_bounds__(256, 4) k_sp_rows_fwd(const float* __restrict__ x, float2* __restrict__ Z, int ny, int nx,
                              int lgnx, const float2* __restrict__ twx) {
    extern __shared__ float2 sp_buf[];
    const int r = blockIdx.x, img = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    pdl_wait();
    pdl_launch_dependents();
    const float* xr = x + ((int64_t)img * ny + r) * nx;
    float4 xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) xv[q] = __ldg(reinterpret_cast<const float4*>(xr + 4 * (tid + q * nthr)));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c0 = 4 * (tid + q * nthr);
        const float4 v = xv[q];
        sp_buf[pad16(c0)] = make_float2(v.x, 0.f);
        sp_buf[pad16(c0 + 1)] = make_float2(v.y, 0.f);
        sp_buf[pad16(c0 + 2)] = make_float2(v.z, 0.f);
        sp_buf[pad16(c0 + 3)] = make_float2(v.w, 0.f);
    }
    __syncthreads();
    sp_fft<-1>(sp_buf, nx, lgnx, twx, tid, nthr);
    float2* Zi = Z + (int64_t)img * ny * nx;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c0 = 4 * (tid + q * nthr);
        float4* dst = reinterpret_cast<float4*>(Zi + ((int64_t)(c0 >> 2) * ny + r) * SP_PANEL);
        const float2 a = sp_buf[pad16(c0)], b = sp_buf[pad16(c0 + 1)];
        const float2 c = sp_buf[pad16(c0 + 2)], d = sp_buf[pad16(c0 + 3)];
        dst[0] = make_float4(a.x, a.y, b.x, b.y);
        dst[1] = make_float4(c.x, c.y, d.x, d.y);
    }
}

// K2: columns 2 blockIdx.x and 2 blockIdx.x + 1 of image blockIdx.y of a
// spectrum of ncol columns (panel layout): forward FFT down each column; with
// P, multiply by P (real, same layout) and transform back (unnormalised
// inverse). With PN (half spectra of real rows, see K1), column 0 holds
// A[0] + i A[nx/2] of every row, two real sequences whose column transforms
// are separated as C0 = (C[ky] + conj C[-ky]) / 2 and
// CN = (C[ky] - conj C[-ky]) / 2i, scaled by P[ky][0] and PN[ky], and
// recombined as C0 + i CN before the inverse. Two transforms of ny / 16
// threads each.
__global__ void __launch_bounds__(512, 2) k_sp_cols(float2* __restrict__ Z, const float* __restrict__ P,
                                                    const float* __restrict__ PN, int ny, int ncol_total,
                                                    int lgny, const float2* __restrict__ twy) {
    extern __shared__ float2 sp_buf[];
    const int pair = blockIdx.x, img = blockIdx.y;
    const int panel = pair >> 1, half = pair & 1;
    const int tid = threadIdx.x, nthr = blockDim.x, ncol = ny >> 4;
    float2* b0 = sp_buf;
    float2* b1 = sp_buf + pad16(ny);
    pdl_wait();
    pdl_launch_dependents();
    float4* col = reinterpret_cast<float4*>(Z + (int64_t)img * ny * ncol_total +
                                            (int64_t)panel * ny * SP_PANEL + 2 * half);
    // element (r, 2 half + e) of the panel is float2 (r 4 + 2 half + e): the
    // pair is float4 2 r of col; nthr = ny / 8, so 8 rows per thread
    if (P) {
        const float* Pp = P + (int64_t)panel * ny * SP_PANEL;
        for (int r = tid * 8; r < ny; r += nthr * 8) prefetch_l2(Pp + 4 * r);   // 128-byte lines
    }
    float4 cv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) cv[q] = col[2 * (tid + q * nthr)];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int r = tid + q * nthr;
        b0[pad16(r)] = make_float2(cv[q].x, cv[q].y);
        b1[pad16(r)] = make_float2(cv[q].z, cv[q].w);
    }
    __syncthreads();
    const int which = tid >= ncol;
    float2* buf = which ? b1 : b0;
    const int ct = tid - which * ncol;
    sp_fft<-1>(buf, ny, lgny, twy, ct, ncol);
    if (P) {
        const float2* Pc = reinterpret_cast<const float2*>(P + (int64_t)panel * ny * SP_PANEL + 2 * half);
        const bool packed0 = PN && pair == 0;   // column 0 carries the DC and Nyquist columns
        if (packed0) {
            for (int ky = tid; ky <= ny / 2; ky += nthr) {
                const int m = (ny - ky) & (ny - 1);
                const float2 c = b0[pad16(ky)], cm = b0[pad16(m)];
                const float s0 = __ldg(Pc + 2 * ky).x, sn = __ldg(PN + ky);
                const float2 f0 = make_float2(0.5f * (c.x + cm.x) * s0, 0.5f * (c.y - cm.y) * s0);
                const float2 fn = make_float2(0.5f * (c.y + cm.y) * sn, 0.5f * (cm.x - c.x) * sn);
                b0[pad16(ky)] = make_float2(f0.x - fn.y, f0.y + fn.x);
                b0[pad16(m)] = make_float2(f0.x + fn.y, fn.x - f0.y);
            }
        }
        for (int r = tid; r < ny; r += nthr) {
            const float2 s = __ldg(Pc + 2 * r);
            if (!packed0) {
                const float2 u = b0[pad16(r)];
                b0[pad16(r)] = make_float2(u.x * s.x, u.y * s.x);
            }
            const float2 w = b1[pad16(r)];
            b1[pad16(r)] = make_float2(w.x * s.y, w.y * s.y);
        }
        __syncthreads();
        sp_fft<1>(buf, ny, lgny, twy, ct, ncol);
    }
    for (int r = tid; r < ny; r += nthr) {
        const float2 u = b0[pad16(r)], w = b1[pad16(r)];
        col[2 * r] = make_float4(u.x, u.y, w.x, w.y);
    }
}

// K1 (real input): rows 2q and 2q + 1 (q = blockIdx.x) of image blockIdx.y of
// x as one complex row z = a + i b; after its FFT Z the half spectra of the two
// real rows are 2A[k] = Z[k] + conj Z[-k] and 2B[k] = (Z[k] - conj Z[-k]) / i,
// k < nx / 2, with k = 0 holding the two real values (2A[0], 2A[nx/2]) (and
// the same for B). Written to rows 2q, 2q + 1 of the nx / 2-column panel layout
// (the factor 2 is taken out by P). nx / 16 threads.
__global__ void __launch_bounds__(256, 4) k_sp_rows_fwd_real(const float* __restrict__ x,
                                                             float2* __restrict__ Zh, int ny, int nx,
                                                             int lgnx, const float2* __restrict__ twx) {
    extern __shared__ float2 sp_buf[];
    const int q = blockIdx.x, img = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x, nxh = nx >> 1;
    pdl_wait();
    pdl_launch_dependents();
    const float* xa = x + ((int64_t)img * ny + 2 * q) * nx;
    const float* xb = xa + nx;
    float4 va[4], vb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        va[k] = __ldg(reinterpret_cast<const float4*>(xa + 4 * (tid + k * nthr)));
        vb[k] = __ldg(reinterpret_cast<const float4*>(xb + 4 * (tid + k * nthr)));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c0 = 4 * (tid + k * nthr);
        sp_buf[pad16(c0)] = make_float2(va[k].x, vb[k].x);
        sp_buf[pad16(c0 + 1)] = make_float2(va[k].y, vb[k].y);
        sp_buf[pad16(c0 + 2)] = make_float2(va[k].z, vb[k].z);
        sp_buf[pad16(c0 + 3)] = make_float2(va[k].w, vb[k].w);
    }
    __syncthreads();
    sp_fft<-1>(sp_buf, nx, lgnx, twx, tid, nthr);
    float2* Zi = Zh + (int64_t)img * ny * nxh;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int c0 = 4 * (tid + k * nthr);   // 4 of the nx / 2 half-spectrum columns
        float2 A[4], B[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c0 + e;
            if (c == 0) {
                const float2 z0 = sp_buf[pad16(0)], zn = sp_buf[pad16(nxh)];
                A[e] = make_float2(2.f * z0.x, 2.f * zn.x);
                B[e] = make_float2(2.f * z0.y, 2.f * zn.y);
            } else {
                const float2 zk = sp_buf[pad16(c)], zm = sp_buf[pad16(nx - c)];
                A[e] = make_float2(zk.x + zm.x, zk.y - zm.y);
                B[e] = make_float2(zk.y + zm.y, zm.x - zk.x);
            }
        }
        float4* da = reinterpret_cast<float4*>(Zi + ((int64_t)(c0 >> 2) * ny + 2 * q) * SP_PANEL);
        float4* db = reinterpret_cast<float4*>(Zi + ((int64_t)(c0 >> 2) * ny + 2 * q + 1) * SP_PANEL);
        da[0] = make_float4(A[0].x, A[0].y, A[1].x, A[1].y);
        da[1] = make_float4(A[2].x, A[2].y, A[3].x, A[3].y);
        db[0] = make_float4(B[0].x, B[0].y, B[1].x, B[1].y);
        db[1] = make_float4(B[2].x, B[2].y, B[3].x, B[3].y);
    }
}

// K3 (real output): the half spectra A', B' of rows 2q, 2q + 1 (q =
// blockIdx.x) of chain blockIdx.y rebuilt into Z' = A' + i B' over all nx
// frequencies (Z'[k] = A'[k] + i B'[k], Z'[nx - k] = conj A'[k] + i conj B'[k],
// the DC and Nyquist terms from column 0), one inverse FFT, then g = Re(.) for
// row 2q and Im(.) for row 2q + 1 minus H^T y, and the x-update of k_update's
// aligned path on both rows, in place.
__global__ void __launch_bounds__(256, 4) k_sp_update(const UpdateParams p, const float2* __restrict__ Zh,
                                                      int lgnx, const float2* __restrict__ twx) {
    extern __shared__ float2 sp_buf[];
    const int q = blockIdx.x, chain = blockIdx.y;
    const int ny = p.ny, nx = p.nx, nxh = nx >> 1;
    const int tid = threadIdx.x, nthr = blockDim.x;
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    float inv_n = p.inv_n;
    if (p.burn_dev) {
        const int64_t n = (int64_t)t + 1 - *p.burn_dev;
        inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
    }
    const int64_t plane = (int64_t)ny * nx, cofs = (int64_t)chain * plane;
    {
        // the update's operands head for L2 while the rows are transformed
        // (one 128-byte line per 8 threads)
        for (int rr = 0; rr < 2; ++rr) {
            const int64_t nrow = (int64_t)(2 * q + rr) * nx, crow = cofs + nrow;
            for (int c = tid * 32; c < nx; c += nthr * 32) {
                prefetch_l2(p.qb + nrow + c);
                prefetch_l2(p.x + crow + c);
                if (p.d) prefetch_l2(p.d + crow + c);
                if (p.mean) {
                    prefetch_l2(p.mean + crow + c);
                    prefetch_l2(p.m2 + crow + c);
                }
            }
        }
    }
    const float2* Zi = Zh + (int64_t)chain * ny * nxh;
    float4 za[4], zb[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int64_t pc = (int64_t)(tid + k * nthr) * ny;
        const float4* sa = reinterpret_cast<const float4*>(Zi + (pc + 2 * q) * SP_PANEL);
        const float4* sb = reinterpret_cast<const float4*>(Zi + (pc + 2 * q + 1) * SP_PANEL);
        za[2 * k] = sa[0];
        za[2 * k + 1] = sa[1];
        zb[2 * k] = sb[0];
        zb[2 * k + 1] = sb[1];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int c0 = 4 * (tid + k * nthr);
        const float2 A[4] = {make_float2(za[2 * k].x, za[2 * k].y), make_float2(za[2 * k].z, za[2 * k].w),
                             make_float2(za[2 * k + 1].x, za[2 * k + 1].y),
                             make_float2(za[2 * k + 1].z, za[2 * k + 1].w)};
        const float2 B[4] = {make_float2(zb[2 * k].x, zb[2 * k].y), make_float2(zb[2 * k].z, zb[2 * k].w),
                             make_float2(zb[2 * k + 1].x, zb[2 * k + 1].y),
                             make_float2(zb[2 * k + 1].z, zb[2 * k + 1].w)};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c0 + e;
            if (c == 0) {
                sp_buf[pad16(0)] = make_float2(A[e].x, B[e].x);
                sp_buf[pad16(nxh)] = make_float2(A[e].y, B[e].y);
            } else {
                sp_buf[pad16(c)] = make_float2(A[e].x - B[e].y, A[e].y + B[e].x);
                sp_buf[pad16(nx - c)] = make_float2(A[e].x + B[e].y, B[e].x - A[e].y);
            }
        }
    }
    __syncthreads();
    sp_fft<1>(sp_buf, nx, lgnx, twx, tid, nthr);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int r = 2 * q + rr;
        float* xc = p.x + cofs;
        const float* dc = p.d ? p.d + cofs : nullptr;
        float* mc = p.mean ? p.mean + cofs : nullptr;
        float* qc = p.m2 ? p.m2 + cofs : nullptr;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c0 = 4 * (tid + k * nthr);
            const int64_t n0 = (int64_t)r * nx + c0;
            const float4 bv = __ldg(reinterpret_cast<const float4*>(p.qb + n0));
            const float4 dv = dc ? __ldg(reinterpret_cast<const float4*>(dc + n0)) : zero4;
            float4 mo = zero4, qo = zero4;
            if (inv_n > 0.f) {
                mo = *reinterpret_cast<const float4*>(mc + n0);
                qo = *reinterpret_cast<const float4*>(qc + n0);
            }
            const float4 xv = *reinterpret_cast<const float4*>(xc + n0);
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (p.c_noise != 0.f)
                normals_group((uint32_t)(n0 >> 2), t, (uint32_t)chain, p.key0, p.key1, z);
            float gr[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 w = sp_buf[pad16(c0 + e)];
                gr[e] = rr == 0 ? w.x : w.y;
            }
            float4 v;
            v.x = update1(p, xv.x, gr[0] - bv.x, dv.x, z[0], 0.f);
            v.y = update1(p, xv.y, gr[1] - bv.y, dv.y, z[1], 0.f);
            v.z = update1(p, xv.z, gr[2] - bv.z, dv.z, z[2], 0.f);
            v.w = update1(p, xv.w, gr[3] - bv.w, dv.w, z[3], 0.f);
            *reinterpret_cast<float4*>(xc + n0) = v;
            if (inv_n > 0.f) {
                welford1(v.x, inv_n, mo.x, qo.x);
                welford1(v.y, inv_n, mo.y, qo.y);
                welford1(v.z, inv_n, mo.z, qo.z);
                welford1(v.w, inv_n, mo.w, qo.w);
                *reinterpret_cast<float4*>(mc + n0) = mo;
                *reinterpret_cast<float4*>(qc + n0) = qo;
            }
        }
    }
    if (p.arrive) {
        __syncthreads();
        if (tid == 0 && atomicAdd(p.arrive, 1u) == gridDim.x * gridDim.y - 1) {
            *p.arrive = 0u;
            *const_cast<uint32_t*>(p.t_dev) = t + 1u;
        }
    }
}

// h placed circularly at the origin: hc[(a - kh/2) mod ny][(b - kw/2) mod nx]
// = h[a][b] (kh <= ny, kw <= nx, so no two taps meet).
__global__ void k_sp_embed(const float* __restrict__ h, int kh, int kw, int ny, int nx,
                           float* __restrict__ hc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kh * kw) return;
    const int a = e / kw, b = e - a * kw;
    int i = a - kh / 2, j = b - kw / 2;
    i += i < 0 ? ny : 0;
    j += j < 0 ? nx : 0;
    hc[(int64_t)i * nx + j] = h[e];
}

// P for the half spectra: P[r][c] = |H^[r][c]|^2 scale (c < nx / 2, half
// panel layout) and PN[r] = |H^[r][nx / 2]|^2 scale, from the full spectrum Hs
// (full panel layout). One thread per (r, c <= nx / 2).
__global__ void k_sp_half_power(const float2* __restrict__ Hs, int ny, int nx, float scale,
                                float* __restrict__ P, float* __restrict__ PN) {
    const int nxh = nx >> 1;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ny * (nxh + 1)) return;
    const int r = (int)(e / (nxh + 1)), c = (int)(e - (int64_t)r * (nxh + 1));
    const float2 v = Hs[((int64_t)(c >> 2) * ny + r) * SP_PANEL + (c & 3)];
    const float pw = (float)(((double)v.x * v.x + (double)v.y * v.y) * scale);
    if (c == nxh) PN[r] = pw;
    else P[((int64_t)(c >> 2) * ny + r) * SP_PANEL + (c & 3)] = pw;
}

int ilog2_exact(int n) {
    int m = 0;
    while ((1 << m) < n) ++m;
    return (1 << m) == n ? m : -1;
}

// exp(-2 pi i n / N), n < N, rounded from FP64
cudaError_t upload_twiddles(int N, float2** out) {
    std::vector<float2> t(N);
    for (int n = 0; n < N; ++n) {
        const double a = -2.0 * 3.14159265358979323846 * (double)n / (double)N;
        t[n] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    cudaError_t e = cudaMalloc(out, sizeof(float2) * N);
    if (e == cudaSuccess) e = cudaMemcpy(*out, t.data(), sizeof(float2) * N, cudaMemcpyHostToDevice);
    return e;
}

size_t rows_smem(int nx) { return sizeof(float2) * (size_t)(nx + nx / 16); }
size_t cols_smem(int ny) { return 2 * sizeof(float2) * (size_t)(ny + ny / 16); }

}  // namespace

bool spectral_eligible(int ny, int nx, int kh, int kw) {
    const int ly = ilog2_exact(ny), lx = ilog2_exact(nx);
    return ly >= 6 && ly <= 12 && lx >= 6 && lx <= 12 && kh <= ny && kw <= nx;
}

void spectral_free(SpectralPlan* S) {
    if (!S) return;
    cudaFree(S->Z);
    cudaFree(S->P);
    cudaFree(S->PN);
    cudaFree(S->twx);
    cudaFree(S->twy);
    delete S;
}

cudaError_t spectral_setup(const float* h, int kh, int kw, int ny, int nx, int nchain,
                           cudaStream_t s, SpectralPlan** out) {
    *out = nullptr;
    if (!spectral_eligible(ny, nx, kh, kw) || nchain < 1) return cudaErrorNotSupported;
    SpectralPlan* S = new SpectralPlan();
    S->ny = ny;
    S->nx = nx;
    S->lgny = ilog2_exact(ny);
    S->lgnx = ilog2_exact(nx);
    const size_t npix = (size_t)ny * nx, nhalf = npix / 2;
    float* hc = nullptr;
    float2* Hs = nullptr;   // full spectrum of the kernel, setup only
    cudaError_t e = cudaFuncSetAttribute(k_sp_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cols_smem(4096));
    if (e == cudaSuccess) e = cudaMalloc(&S->Z, sizeof(float2) * nhalf * nchain);
    if (e == cudaSuccess) e = cudaMalloc(&S->P, sizeof(float) * nhalf);
    if (e == cudaSuccess) e = cudaMalloc(&S->PN, sizeof(float) * ny);
    if (e == cudaSuccess) e = upload_twiddles(nx, &S->twx);
    if (e == cudaSuccess) e = upload_twiddles(ny, &S->twy);
    if (e == cudaSuccess) e = cudaMalloc(&hc, sizeof(float) * npix);
    if (e == cudaSuccess) e = cudaMalloc(&Hs, sizeof(float2) * npix);
    if (e == cudaSuccess) e = cudaMemsetAsync(hc, 0, sizeof(float) * npix, s);
    if (e == cudaSuccess) {
        const int n = kh * kw;
        k_sp_embed<<<(n + 255) / 256, 256, 0, s>>>(h, kh, kw, ny, nx, hc);
        note_launch();
        e = cudaGetLastError();
    }
    // full spectrum of the kernel (complex row FFTs, then column FFTs)
    if (e == cudaSuccess)
        e = launch_pdl(k_sp_rows_fwd, dim3(ny, 1), dim3(nx / 16), rows_smem(nx), s, (const float*)hc,
                       Hs, ny, nx, S->lgnx, (const float2*)S->twx);
    if (e == cudaSuccess)
        e = launch_pdl(k_sp_cols, dim3(nx / 2, 1), dim3(ny / 8), cols_smem(ny), s, Hs,
                       (const float*)nullptr, (const float*)nullptr, ny, nx, S->lgny,
                       (const float2*)S->twy);
    // P = |H^|^2 / (2 ny nx): the factor 2 of the stored half spectra and the
    // 1 / (ny nx) of the inverse transforms
    if (e == cudaSuccess) {
        const int64_t n = (int64_t)ny * (nx / 2 + 1);
        k_sp_half_power<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            Hs, ny, nx, (float)(0.5 / (double)npix), S->P, S->PN);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(hc);
    cudaFree(Hs);
    if (e != cudaSuccess) {
        spectral_free(S);
        return e;
    }
    *out = S;
    return cudaSuccess;
}

cudaError_t spectral_pre(const SpectralPlan& S, const float* x, int nchain, cudaStream_t s) {
    timer_begin(T_BLUR, s);
    cudaError_t e = launch_pdl(k_sp_rows_fwd_real, dim3(S.ny / 2, nchain), dim3(S.nx / 16),
                               rows_smem(S.nx), s, x, S.Z, S.ny, S.nx, S.lgnx, (const float2*)S.twx);
    if (e == cudaSuccess)
        e = launch_pdl(k_sp_cols, dim3(S.nx / 4, nchain), dim3(S.ny / 8), cols_smem(S.ny), s, S.Z,
                       (const float*)S.P, (const float*)S.PN, S.ny, S.nx / 2, S.lgny,
                       (const float2*)S.twy);
    timer_end(T_BLUR, s);
    return e;
}

cudaError_t spectral_update(const SpectralPlan& S, const UpdateParams& p, cudaStream_t s) {
    if (!p.qb || p.ny != S.ny || p.nx != S.nx || p.z2) return cudaErrorInvalidValue;
    timer_begin(T_UPDATE, s);
    const cudaError_t e = launch_pdl(k_sp_update, dim3(S.ny / 2, p.nchain), dim3(S.nx / 16),
                                     rows_smem(S.nx), s, p, (const float2*)S.Z, S.lgnx,
                                     (const float2*)S.twx);
    timer_end(T_UPDATE, s);
    return e;
}

}  // namespace pnp
