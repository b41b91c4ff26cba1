// DDFB denoiser (Sec. II-B, Example 2): an unrolled dual forward-backward
// algorithm. With W_k the 1 -> P channel 3 x 3 analysis convolution (zero
// padding), W_k^* its adjoint and HT the hard-tanh clip to [-ht, ht]:
//   u_0 = W_K v
//   u_k = HT( u_{k-1} + gamma_k W_k proj_[0,1](v - W_k^* u_{k-1}) ),  k = 1 .. K-1
//   D(v) = proj_[0,1]( v - gamma_K W_K^* u_{K-1} )
// One launch per dual layer, one for the output. The work per pixel is small
// (P x 9 multiply-adds per operator), so each launch streams the P-channel
// dual variable once in and once out of HBM:
//   * a block owns a 32 x 8 tile; the P channels are staged in shared memory
//     16 at a time with a 2-pixel halo, and each thread accumulates W_k^* u at
//     the tile + 1-pixel halo positions it owns (s needs one more ring than the
//     tile for the following W_k);
//   * the update re-reads each pixel's own P dual values (just staged by the
//     same block, so from L2) instead of holding them in registers: at about
//     40 registers a thread, several blocks share an SM and hide each other's
//     load latency;
//   * the layer's filters are a by-value kernel parameter: every multiply-add
//     takes its weight from the constant bank;
//   * the first dual layer computes u_0 = W_K v from v on the fly (u_0 is never
//     written), the output launch reads u_{K-1} once.
#include "pdl.cuh"
#include "pnp_internal.h"

namespace pnp {

namespace {

constexpr int DB_TW = 32, DB_TH = 8, DB_CH = 16;

struct DdfbFilters {
    float w[64 * 9];    // W_k (or W_K for the output launch), [p][3][3]
    float wK[64 * 9];   // W_K, used by the first dual layer for u_0 = W_K v
};

// MODE 0: dual layer from u_in; MODE 1: first dual layer (u_in = W_K v);
// MODE 2: output D(v) = clip(v - gam W_K^* u_in).
template <int P, int MODE>
__global__ void __launch_bounds__(256, 4) k_ddfb(const float* __restrict__ v,
                                              const float* __restrict__ uin,
                                              float* __restrict__ out, int ny, int nx, float gam,
                                              float ht, const __grid_constant__ DdfbFilters L) {
    constexpr int HALO = MODE == 2 ? 1 : 2;            // u ring around the tile
    constexpr int UH = DB_TH + 2 * HALO, UW = DB_TW + 2 * HALO;
    constexpr int SH = DB_TH + 2, SW = DB_TW + 2;      // s: tile + 1 ring (dual layers)
    constexpr int NPOS = MODE == 2 ? DB_TH * DB_TW : SH * SW;
    constexpr int VH = DB_TH + 6, VW = DB_TW + 6;      // v: tile + 3 rings (first layer)
    __shared__ float us[DB_CH][UH][UW];
    __shared__ float ss[SH][SW];
    __shared__ float vs[MODE == 1 ? VH : 1][MODE == 1 ? VW : 1];

    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int img = blockIdx.z;
    const int64_t plane = (int64_t)ny * nx;
    const int i0 = blockIdx.y * DB_TH, j0 = blockIdx.x * DB_TW;
    const float* vi = v + img * plane;
    const float* ui = uin ? uin + img * (int64_t)P * plane : nullptr;
    pdl_wait();
    pdl_launch_dependents();

    if constexpr (MODE == 1) {
        for (int it = tid; it < VH * VW; it += 256) {
            const int r = it / VW, c = it - r * VW;
            const int gi = i0 - 3 + r, gj = j0 - 3 + c;
            vs[r][c] = (gi >= 0 && gi < ny && gj >= 0 && gj < nx) ? __ldg(vi + (int64_t)gi * nx + gj)
                                                                 : 0.f;
        }
    }
    // positions this thread accumulates W^* u at (at most two)
    int pr[2], pc[2];
    bool pv[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int pos = tid + 256 * k;
        pv[k] = pos < NPOS;
        if (MODE == 2) {
            pr[k] = ty;
            pc[k] = tx;
        } else {
            pr[k] = pv[k] ? pos / SW : 0;
            pc[k] = pv[k] ? pos - pr[k] * SW : 0;
        }
    }
    float sacc[2] = {0.f, 0.f};

#pragma unroll
    for (int c0 = 0; c0 < P; c0 += DB_CH) {
        __syncthreads();   // previous chunk consumed (and vs filled)
        for (int it = tid; it < DB_CH * UH * UW; it += 256) {
            const int ch = it / (UH * UW);
            const int rem = it - ch * (UH * UW);
            const int r = rem / UW, c = rem - r * UW;
            const int gi = i0 - HALO + r, gj = j0 - HALO + c;
            const bool inside = gi >= 0 && gi < ny && gj >= 0 && gj < nx;
            float val = 0.f;
            if (inside) {
                if constexpr (MODE == 1) {
                    // u_0 = W_K v: correlation of v with the channel's filter
                    const float* wk = L.wK + (c0 + ch) * 9;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) val = fmaf(wk[a * 3 + b], vs[r + a][c + b], val);
                } else {
                    val = __ldg(ui + (int64_t)(c0 + ch) * plane + (int64_t)gi * nx + gj);
                }
            }
            us[ch][r][c] = val;
        }
        __syncthreads();
        // W^* u at the owned positions: sum_p sum_ab w[p][a][b] u_p(q - a + 1, q - b + 1)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!pv[k]) continue;
            float acc = sacc[k];
            // the staged u block starts one ring further out than the positions
            // (HALO vs HALO - 1 rings), so u(q - a + 1) is staged row pr + 2 - a
            const int rb = pr[k] + 2, cb = pc[k] + 2;
#pragma unroll
            for (int ch = 0; ch < DB_CH; ++ch)
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
                        acc = fmaf(L.w[(c0 + ch) * 9 + a * 3 + b], us[ch][rb - a][cb - b], acc);
            sacc[k] = acc;
        }
    }

    const int i = i0 + ty, j = j0 + tx;
    const bool own = i < ny && j < nx;
    if constexpr (MODE == 2) {
        if (own) {
            const float d = __ldg(vi + (int64_t)i * nx + j) - gam * sacc[0];
            out[img * plane + (int64_t)i * nx + j] = fminf(fmaxf(d, 0.f), 1.f);
        }
        return;
    }
    // s = proj_[0,1](v - W_k^* u) on the tile + 1 ring, zero outside the image
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!pv[k]) continue;
        const int gi = i0 - 1 + pr[k], gj = j0 - 1 + pc[k];
        float sv = 0.f;
        if (gi >= 0 && gi < ny && gj >= 0 && gj < nx)
            sv = fminf(fmaxf(__ldg(vi + (int64_t)gi * nx + gj) - sacc[k], 0.f), 1.f);
        ss[pr[k]][pc[k]] = sv;
    }
    __syncthreads();
    if (!own) return;
    float sr[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) sr[a * 3 + b] = ss[ty + a][tx + b];
    float* uo = out + img * (int64_t)P * plane + (int64_t)i * nx + j;
    const float* uc = ui + (int64_t)i * nx + j;
#pragma unroll 4
    for (int p = 0; p < P; ++p) {
        // (W_k s)_p at the pixel: correlation of s with the channel's filter
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q) t = fmaf(L.w[p * 9 + q], sr[q], t);
        float u;
        if constexpr (MODE == 1) {
            // u_0 = W_K v at the pixel, from the staged v
            u = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) u = fmaf(L.wK[p * 9 + a * 3 + b], vs[ty + 2 + a][tx + 2 + b], u);
        } else {
            u = __ldg(uc + (int64_t)p * plane);
        }
        const float un = fmaf(gam, t, u);
        uo[(int64_t)p * plane] = fminf(fmaxf(un, -ht), ht);
    }
}

template <int P>
cudaError_t ddfb_forward_P(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                           float* d, float* scratch, cudaStream_t s) {
    const int K = D.K;
    const size_t ufl = (size_t)nimg * P * ny * nx;
    float* ua = scratch;
    float* ub = scratch + ufl;
    dim3 grid((nx + DB_TW - 1) / DB_TW, (ny + DB_TH - 1) / DB_TH, nimg);
    DdfbFilters F;
    const float* WK = D.ddfb_w + (size_t)(K - 1) * P * 9;
    for (int q = 0; q < P * 9; ++q) F.wK[q] = WK[q];
    cudaError_t e = cudaSuccess;
    const float* cur = nullptr;
    for (int k = 0; k < K - 1 && e == cudaSuccess; ++k) {
        const float* Wk = D.ddfb_w + (size_t)k * P * 9;
        for (int q = 0; q < P * 9; ++q) F.w[q] = Wk[q];
        float* nxt = (k % 2 == 0) ? ua : ub;
        timer_begin(T_CONV_FP32, s);
        if (k == 0)
            e = launch_pdl(k_ddfb<P, 1>, grid, dim3(256), 0, s, x, (const float*)nullptr, nxt, ny,
                           nx, D.ddfb_gamma[k], D.ddfb_ht, F);
        else
            e = launch_pdl(k_ddfb<P, 0>, grid, dim3(256), 0, s, x, cur, nxt, ny, nx,
                           D.ddfb_gamma[k], D.ddfb_ht, F);
        timer_end(T_CONV_FP32, s);
        cur = nxt;
    }
    if (e != cudaSuccess) return e;
    for (int q = 0; q < P * 9; ++q) F.w[q] = WK[q];
    timer_begin(T_CONV_EDGE, s);
    e = launch_pdl(k_ddfb<P, 2>, grid, dim3(256), 0, s, x, cur, d, ny, nx, D.ddfb_gamma[K - 1],
                   D.ddfb_ht, F);
    timer_end(T_CONV_EDGE, s);
    return e;
}

}  // namespace

cudaError_t ddfb_forward(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, float* scratch, cudaStream_t s) {
    if (rects || D.K < 2) return cudaErrorInvalidValue;   // direct layout only
    switch (D.F) {
        case 16: return ddfb_forward_P<16>(D, x, ny, nx, nimg, d, scratch, s);
        case 32: return ddfb_forward_P<32>(D, x, ny, nx, nimg, d, scratch, s);
        case 64: return ddfb_forward_P<64>(D, x, ny, nx, nimg, d, scratch, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pnp
