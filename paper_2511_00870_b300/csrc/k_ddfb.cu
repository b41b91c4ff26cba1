// DDFB denoiser (Sec. II-B, Example 2): an unrolled dual forward-backward
// algorithm. With W_k the 1 -> P channel 3 x 3 analysis convolution (zero
// padding), W_k^* its adjoint and HT the hard-tanh clip to [-ht, ht]:
//   u_0 = W_K v
//   u_k = HT( u_{k-1} + gamma_k W_k proj_[0,1](v - W_k^* u_{k-1}) ),  k = 1 .. K-1
//   D(v) = proj_[0,1]( v - gamma_K W_K^* u_{K-1} )
// One launch per dual layer, one for the output. The work per pixel is small
// (P x 9 multiply-adds per operator), so each launch streams the P-channel
// dual variable once in and once out of HBM:
//   * a block owns a 32 x 8 tile; the P channels stream through shared
//     memory 8 at a time with a 2-pixel halo, double buffered: 16-byte
//     asynchronous copies of the next group (source offsets computed once per
//     thread, the pattern repeats for every group) are in flight while the
//     current one is reduced;
//   * W_k^* u is accumulated for vertical pairs of positions over the tile +
//     1-pixel ring (s needs one more ring than the tile for the following W_k):
//     a 4 x 3 window of each channel gives both sums;
//   * the update re-reads each pixel's own P dual values (just staged by the
//     same block, so from L2) instead of holding them in registers, which
//     keeps four blocks per SM;
//   * the layer's filters are a by-value kernel parameter: every multiply-add
//     takes its weight from the constant bank;
//   * the first dual layer takes W_1^* W_K v as one 5 x 5 filter of v away from
//     the image border and u_0 = W_K v per pixel for its update (u_0 is never
//     written); the output launch reads u_{K-1} once.
#include "pdl.cuh"
#include "pnp_internal.h"

namespace pnp {

namespace {

constexpr int DB_TW = 32, DB_TH = 8, DB_CH = 8;

struct DdfbFilters {
    float w[64 * 9];    // W_k (or W_K for the output launch), [p][3][3]
    float wK[64 * 9];   // W_K, used by the first dual layer for u_0 = W_K v
    float c5[25];       // first dual layer: the 5 x 5 filter of W_1^* W_K (see k_ddfb)
    float m81[81];      // M[a b][c d] = sum_p w_1[p][a][b] w_K[p][c][d] (border pixels)
};

// asynchronous global -> shared copies; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int MODE>
struct DdfbGeom {
    static constexpr int HALO = MODE == 2 ? 1 : 2;          // u ring around the tile
    static constexpr int UH = DB_TH + 2 * HALO;
    // staged rows hold columns j0 - 4 .. j0 + 35 (a 16-byte aligned span that
    // contains the columns j0 - HALO .. j0 + 31 + HALO, at offset CX)
    static constexpr int UP = DB_TW + 8, CX = 4 - HALO;
    static constexpr int SH = MODE == 2 ? DB_TH : DB_TH + 2;  // W^* u positions: tile (+1 ring)
    static constexpr int SW = MODE == 2 ? DB_TW : DB_TW + 2;
    static constexpr int NPAIR = SW * (SH / 2);               // vertical pairs of positions
    static constexpr int VH = DB_TH + 6, VW = DB_TW + 6;      // v: tile + 3 rings (first layer)
    static constexpr int USTAGE = MODE == 1 ? 0 : 2 * DB_CH * UH * UP;   // channel groups
    static constexpr size_t SMEM =
        sizeof(float) * (USTAGE + (DB_TH + 2) * (DB_TW + 2) + (MODE == 1 ? VH * VW : 0));
};

// MODE 0: dual layer from u_in; MODE 1: first dual layer (u_in = W_K v);
// MODE 2: output D(v) = clip(v - gam W_K^* u_in).
// The first dual layer needs W_1^* W_K v. Away from the image border (all nine
// pixels q - a + 1 inside the image) that is one 5 x 5 correlation of v,
// C[e][f] = sum_p sum_{c - a = e - 2, d - b = f - 2} w_1[p][a][b] w_K[p][c][d],
// so the P-channel u_0 is never formed there. On the border rows and columns
// u_0 is zero outside the image, so the terms whose pixel q - a + 1 falls
// outside drop out: the sum runs over the (a, b) inside, with the channel sum
// folded into M[a b][c d] = sum_p w_1[p][a][b] w_K[p][c][d].
template <int P, int MODE>
__global__ void __launch_bounds__(256, 4) k_ddfb(const float* __restrict__ v,
                                              const float* __restrict__ uin,
                                              float* __restrict__ out, int ny, int nx, float gam,
                                              float ht, const __grid_constant__ DdfbFilters L) {
    using G = DdfbGeom<MODE>;
    constexpr int UH = G::UH, HALO = G::HALO, UP = G::UP, CX = G::CX;
    constexpr int NCH = P / DB_CH;
    extern __shared__ float4 sm4[];
    float* us = reinterpret_cast<float*>(sm4);                 // [2][DB_CH][UH][UP]
    float* ss = us + G::USTAGE;                                // [DB_TH + 2][DB_TW + 2]
    float* vs = ss + (DB_TH + 2) * (DB_TW + 2);                // [VH][VW] (first layer)

    const int tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int img = blockIdx.z;
    const int64_t plane = (int64_t)ny * nx;
    const int i0 = blockIdx.y * DB_TH, j0 = blockIdx.x * DB_TW;
    const float* vi = v + img * plane;
    const float* ui = uin ? uin + img * (int64_t)P * plane : vi;
    pdl_wait();
    pdl_launch_dependents();

    // A group's copies: with rows of whole float4s (nx % 4 == 0) 16-byte copies
    // whose source offsets within a channel group are computed once (the
    // pattern repeats for every group); otherwise 4-byte copies.
    const bool vec = (nx & 3) == 0 && (reinterpret_cast<uintptr_t>(ui) & 15) == 0;
    constexpr int NV = DB_CH * UH * (UP / 4);
    constexpr int KV = (NV + 255) / 256;
    int64_t voff[KV];
    int vso[KV];
    bool vin[KV], vok[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
        const int it = tid + 256 * k;
        vok[k] = it < NV;
        const int ch = it / (UH * (UP / 4));
        const int rem = it - ch * (UH * (UP / 4));
        const int r = rem / (UP / 4), c4 = rem - r * (UP / 4);
        const int gi = i0 - HALO + r, gj = j0 - 4 + 4 * c4;
        vin[k] = vok[k] && gi >= 0 && gi < ny && gj >= 0 && gj < nx;
        voff[k] = vin[k] ? (int64_t)ch * plane + (int64_t)gi * nx + gj : 0;
        vso[k] = (ch * UH + r) * UP + 4 * c4;
    }
    auto stage = [&](int buf, int c0) {
        float* dst = us + buf * DB_CH * UH * UP;
        if (vec) {
            const float* base = ui + (int64_t)c0 * plane;
#pragma unroll
            for (int k = 0; k < KV; ++k)
                if (vok[k]) cp_async16(dst + vso[k], vin[k] ? base + voff[k] : ui, vin[k] ? 16 : 0);
        } else {
            for (int it = tid; it < DB_CH * UH * UP; it += 256) {
                const int ch = it / (UH * UP);
                const int rem = it - ch * (UH * UP);
                const int r = rem / UP, c = rem - r * UP;
                const int gi = i0 - HALO + r, gj = j0 - 4 + c;
                const bool inside = gi >= 0 && gi < ny && gj >= 0 && gj < nx;
                const float* src = inside ? ui + (int64_t)(c0 + ch) * plane + (int64_t)gi * nx + gj : ui;
                cp_async4(dst + it, src, inside ? 4 : 0);
            }
        }
        cp_async_commit();
    };

    // the vertical pair of W^* u positions this thread accumulates
    const bool act = tid < G::NPAIR;
    const int pc = act ? tid % G::SW : 0, pr = act ? 2 * (tid / G::SW) : 0;
    float acc0 = 0.f, acc1 = 0.f;

    if constexpr (MODE == 1) {
        for (int it = tid; it < G::VH * G::VW; it += 256) {
            const int r = it / G::VW, c = it - r * G::VW;
            const int gi = i0 - 3 + r, gj = j0 - 3 + c;
            vs[it] = (gi >= 0 && gi < ny && gj >= 0 && gj < nx) ? __ldg(vi + (int64_t)gi * nx + gj) : 0.f;
        }
        __syncthreads();
        if (act) {
            // position (pr + t, pc) is vs row pr + t + 2, column pc + 2; the 5 x 5
            // filter reads vs rows pr + t .. pr + t + 4, columns pc .. pc + 4
            float vw6[6][5];
#pragma unroll
            for (int e = 0; e < 6; ++e)
#pragma unroll
                for (int f = 0; f < 5; ++f) vw6[e][f] = vs[(pr + e) * G::VW + pc + f];
#pragma unroll
            for (int e = 0; e < 5; ++e)
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    acc0 = fmaf(L.c5[e * 5 + f], vw6[e][f], acc0);
                    acc1 = fmaf(L.c5[e * 5 + f], vw6[e + 1][f], acc1);
                }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int gi = i0 - 1 + pr + t, gj = j0 - 1 + pc;
                const bool inside = gi >= 0 && gi < ny && gj >= 0 && gj < nx;
                if (!inside || (gi >= 1 && gi <= ny - 2 && gj >= 1 && gj <= nx - 2)) continue;
                // image border: u_0(r) = (W_K v)(r) only for r inside the image
                const int lr = pr + t + 2, lc = pc + 2;
                float acc = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int ri = gi - a + 1, rj = gj - b + 1;
                        if (ri < 0 || ri >= ny || rj < 0 || rj >= nx) continue;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
#pragma unroll
                            for (int d = 0; d < 3; ++d)
                                acc = fmaf(L.m81[(a * 3 + b) * 9 + c * 3 + d],
                                           vs[(lr - a + c) * G::VW + lc - b + d], acc);
                    }
                if (t) acc1 = acc;
                else acc0 = acc;
            }
        }
    } else {
        stage(0, 0);
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            const int c0 = k * DB_CH;
            float* ub = us + (k & 1) * DB_CH * UH * UP;
            if (k + 1 < NCH) {
                stage((k + 1) & 1, c0 + DB_CH);   // next group in flight
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            // W^* u at (q, q + one row): sum_p sum_ab w[p][a][b] u_p(q - a + 1, q - b + 1);
            // the staged block starts one ring further out than the positions, so
            // u(q - a + 1) is staged row pr + 2 - a
            if (act) {
#pragma unroll
                for (int ch = 0; ch < DB_CH; ++ch) {
                    const float* uc = ub + ch * UH * UP + CX;
                    float uw[4][3];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) uw[a][b] = uc[(pr + a) * UP + pc + b];
                    const float* wk = L.w + (c0 + ch) * 9;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            acc0 = fmaf(wk[a * 3 + b], uw[2 - a][2 - b], acc0);
                            acc1 = fmaf(wk[a * 3 + b], uw[3 - a][2 - b], acc1);
                        }
                }
            }
            __syncthreads();   // group consumed before its buffer refills
        }
    }

    if constexpr (MODE == 2) {
        if (act) {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = i0 + pr + t, j = j0 + pc;
                if (i < ny && j < nx) {
                    const float d = __ldg(vi + (int64_t)i * nx + j) - gam * (t ? acc1 : acc0);
                    out[img * plane + (int64_t)i * nx + j] = fminf(fmaxf(d, 0.f), 1.f);
                }
            }
        }
        return;
    }
    // s = proj_[0,1](v - W_k^* u) on the tile + 1 ring, zero outside the image
    if (act) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int gi = i0 - 1 + pr + t, gj = j0 - 1 + pc;
            float sv = 0.f;
            if (gi >= 0 && gi < ny && gj >= 0 && gj < nx)
                sv = fminf(fmaxf(__ldg(vi + (int64_t)gi * nx + gj) - (t ? acc1 : acc0), 0.f), 1.f);
            ss[(pr + t) * (DB_TW + 2) + pc] = sv;
        }
    }
    __syncthreads();
    const int i = i0 + ty, j = j0 + tx;
    if (i >= ny || j >= nx) return;
    float sr[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) sr[a * 3 + b] = ss[(ty + a) * (DB_TW + 2) + tx + b];
    float vw[3][3];
    if constexpr (MODE == 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) vw[a][b] = vs[(ty + 2 + a) * G::VW + tx + 2 + b];
    }
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
            u = 0.f;   // u_0 = W_K v at the pixel
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) u = fmaf(L.wK[p * 9 + a * 3 + b], vw[a][b], u);
        } else {
            u = __ldg(uc + (int64_t)p * plane);
        }
        const float un = fmaf(gam, t, u);
        uo[(int64_t)p * plane] = fminf(fmaxf(un, -ht), ht);
    }
}

template <int P, int MODE>
cudaError_t ddfb_launch(dim3 grid, cudaStream_t s, const float* x, const float* u, float* out,
                        int ny, int nx, float gam, float ht, const DdfbFilters& F) {
    constexpr size_t smem = DdfbGeom<MODE>::SMEM;
    static_assert(smem <= 48 * 1024, "dynamic shared memory above 48 KB needs an opt-in");
    return launch_pdl(k_ddfb<P, MODE>, grid, dim3(256), smem, s, x, u, out, ny, nx, gam, ht, F);
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
    // first dual layer: M[a b][c d] = sum_p w_1[p][a][b] w_K[p][c][d] and the
    // 5 x 5 filter of W_1^* W_K, C[e][f] = sum over c - a = e - 2, d - b = f - 2
    // of M (interior pixels), both accumulated in FP64
    const float* W1 = D.ddfb_w;
    double M[81], C[25] = {0.0};
    for (int ab = 0; ab < 9; ++ab)
        for (int cd = 0; cd < 9; ++cd) {
            double m = 0.0;
            for (int p = 0; p < P; ++p) m += (double)W1[p * 9 + ab] * WK[p * 9 + cd];
            M[ab * 9 + cd] = m;
            F.m81[ab * 9 + cd] = (float)m;
            const int e = cd / 3 - ab / 3 + 2, f = cd % 3 - ab % 3 + 2;
            C[e * 5 + f] += m;
        }
    for (int q = 0; q < 25; ++q) F.c5[q] = (float)C[q];
    cudaError_t e = cudaSuccess;
    const float* cur = nullptr;
    for (int k = 0; k < K - 1 && e == cudaSuccess; ++k) {
        const float* Wk = D.ddfb_w + (size_t)k * P * 9;
        for (int q = 0; q < P * 9; ++q) F.w[q] = Wk[q];
        float* nxt = (k % 2 == 0) ? ua : ub;
        // dual layers under conv_fp32; the first layer and the output under conv_edge
        const int tid = k == 0 ? T_CONV_EDGE : T_CONV_FP32;
        timer_begin(tid, s);
        if (k == 0)
            e = ddfb_launch<P, 1>(grid, s, x, nullptr, nxt, ny, nx, D.ddfb_gamma[k], D.ddfb_ht, F);
        else
            e = ddfb_launch<P, 0>(grid, s, x, cur, nxt, ny, nx, D.ddfb_gamma[k], D.ddfb_ht, F);
        timer_end(tid, s);
        cur = nxt;
    }
    if (e != cudaSuccess) return e;
    for (int q = 0; q < P * 9; ++q) F.w[q] = WK[q];
    timer_begin(T_CONV_EDGE, s);
    e = ddfb_launch<P, 2>(grid, s, x, cur, d, ny, nx, D.ddfb_gamma[K - 1], D.ddfb_ht, F);
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
