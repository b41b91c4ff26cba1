// Device code shared by the stencil kernels (k_stencil.cu) and the one-pass
// update (k_update_os.cu): tile geometry, asynchronous copies, separable taps,
// the two separable passes and the per-pixel x-update and Welford step. Both
// files inline the same functions, so a pixel gets bitwise the same result
// from either kernel.
#pragma once
#include <stdint.h>

#include "philox.cuh"
#include "pnp_internal.h"

namespace pnp {

constexpr int ST_TX = 64;     // tile width (outputs): 16 threads x 4 columns
constexpr int ST_MAXK = 31;

// Rows per item of the separable vertical pass, independent of the tile's R:
// an item reads SEP_VR + kh - 1 window rows for 4 SEP_VR outputs. Every tile
// height (R * BY, BY a multiple of 8) is a multiple of it.
constexpr int SEP_VR = 4;

// Shared-memory window of a tile: its column 0 is image column j0 - AL (AL =
// rx rounded up to a multiple of 4), so that a 16-byte-aligned image row maps
// onto 16-byte-aligned shared memory; output column j0 + v then reads window
// columns v + SHIFT .. v + SHIFT + KW - 1 (SHIFT = AL - rx, folded into the
// register indices at compile time).
template <int KW>
struct Geom {
    static constexpr int RX = KW / 2;
    static constexpr int AL = (RX + 3) & ~3;
    static constexpr int SHIFT = AL - RX;
    static constexpr int WXA = ST_TX + 2 * AL;        // window columns loaded
    static constexpr int KWP = (KW + 3) & ~3;         // tap row pitch
    static constexpr int NW4 = (KW + 3 + 3) / 4 + (SHIFT > 0 ? 1 : 0);   // float4 per thread row
    static constexpr int WP = WXA > ST_TX + 4 * NW4 ? WXA : ST_TX + 4 * NW4;   // pitch (floats)
    static_assert(60 + 4 * NW4 <= WP, "window row read past the pitch");
    static_assert(4 * NW4 >= SHIFT + KW + 3, "window slice too short");
    static_assert(WXA % 4 == 0 && WP % 4 == 0, "16-byte rows");
};


// c mod n for c in [-n, 2n); anything else (rows of a ragged tile past the
// image, never used) is clamped into the image.
__device__ __forceinline__ int wrap(int c, int n) {
    c += c < 0 ? n : 0;
    c -= c >= n ? n : 0;
    return min(max(c, 0), n - 1);
}

// Asynchronous global -> shared copies (cp.async): every thread issues all of
// its copies of a window before waiting for any, so the whole window is in
// flight at once instead of one load per thread at a time.
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void prefetch_l2(const float* p) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Separable taps from hsep = [u (kh) | v (KW) | u flipped | v flipped]: v
// zero-padded to KWP, then u.
template <int KW>
__device__ __forceinline__ void load_taps_sep(const float* __restrict__ hsep, int kh, bool flip,
                                              float* vs, float* us) {
    using G = Geom<KW>;
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const float* src = hsep + (flip ? kh + KW : 0);
    for (int e = tid; e < G::KWP + kh; e += nt) {
        if (e < G::KWP) vs[e] = e < KW ? __ldg(src + kh + e) : 0.f;
        else us[e - G::KWP] = __ldg(src + (e - G::KWP));
    }
}

// Separable kernels run the vertical pass first, over every window column:
//   V[o][c] = sum_a us[a] win[o + a][c]          (a ascending, from 0)
// for the tile's `rows` output rows, then the horizontal pass over V:
//   out[o][j] = sum_b vs[b] V[o][j + SHIFT + b]  (b ascending, from 0).
// The vertical pass does rows x window-width x kh FMAs, so its cost per
// output does not grow with the window's (kh - 1)-row halo, and its FMAs pair
// up on the two halves of each 128-bit shared-memory load (packed FP32 FMA,
// each component rounded exactly as fmaf). V is stored with row pairs
// interleaved, element (o, c) at ((o / 2) WP + c) 2 + o % 2, so that the
// horizontal pass can advance two output rows per packed FMA. Every output is
// the same fixed-order sum whatever the tile.
__device__ __forceinline__ int vidx(int o, int c, int wp) { return ((o >> 1) * wp + c) * 2 + (o & 1); }

template <int KW, int R>
__device__ __forceinline__ void sep_vert(const float* win, const float* us, int kh, int rows,
                                         float* V) {
    using G = Geom<KW>;
    constexpr int NC4 = G::WXA / 4;
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nrb = rows / R;
    // the four columns of rows o, o + 1 of an item into V
    auto put2 = [&](int o, int c4, float a0, float a1, float a2, float a3, float b0, float b1,
                    float b2, float b3) {
        float* d = V + vidx(o, 4 * c4, G::WP);
        *reinterpret_cast<float4*>(d) = make_float4(a0, b0, a1, b1);
        *reinterpret_cast<float4*>(d + 4) = make_float4(a2, b2, a3, b3);
    };
    auto put1 = [&](int o, int c4, float a0, float a1, float a2, float a3) {
        V[vidx(o, 4 * c4, G::WP)] = a0;
        V[vidx(o, 4 * c4 + 1, G::WP)] = a1;
        V[vidx(o, 4 * c4 + 2, G::WP)] = a2;
        V[vidx(o, 4 * c4 + 3, G::WP)] = a3;
    };
    if (kh == KW) {
        float2 u2[KW];
#pragma unroll
        for (int a = 0; a < KW; ++a) u2[a] = make_float2(us[a], us[a]);
        for (int it = tid; it < nrb * NC4; it += nt) {
            const int rb = it / NC4, c4 = it - rb * NC4;
            const float* src = win + rb * R * G::WP + 4 * c4;
            float2 lo[R], hi[R];
#pragma unroll
            for (int o = 0; o < R; ++o) lo[o] = hi[o] = make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < R + KW - 1; ++u) {
                const float4 v = *reinterpret_cast<const float4*>(src + u * G::WP);
                const float2 vl = make_float2(v.x, v.y), vh = make_float2(v.z, v.w);
#pragma unroll
                for (int o = 0; o < R; ++o) {
                    const int a = u - o;
                    if (a < 0 || a >= KW) continue;
                    lo[o] = __ffma2_rn(u2[a], vl, lo[o]);
                    hi[o] = __ffma2_rn(u2[a], vh, hi[o]);
                }
            }
            if constexpr (R % 2 == 0) {
#pragma unroll
                for (int o = 0; o < R; o += 2)
                    put2(rb * R + o, c4, lo[o].x, lo[o].y, hi[o].x, hi[o].y, lo[o + 1].x,
                         lo[o + 1].y, hi[o + 1].x, hi[o + 1].y);
            } else {
#pragma unroll
                for (int o = 0; o < R; ++o) put1(rb * R + o, c4, lo[o].x, lo[o].y, hi[o].x, hi[o].y);
            }
        }
    } else {
        for (int it = tid; it < nrb * NC4; it += nt) {
            const int rb = it / NC4, c4 = it - rb * NC4;
            const float* src = win + rb * R * G::WP + 4 * c4;
            float acc[R][4];
#pragma unroll
            for (int o = 0; o < R; ++o)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[o][q] = 0.f;
#pragma unroll 1
            for (int u = 0; u < R + kh - 1; ++u) {
                const float4 v = *reinterpret_cast<const float4*>(src + u * G::WP);
#pragma unroll
                for (int o = 0; o < R; ++o) {
                    const int a = u - o;
                    if (a < 0 || a >= kh) continue;
                    const float ua = us[a];
                    acc[o][0] = fmaf(ua, v.x, acc[o][0]);
                    acc[o][1] = fmaf(ua, v.y, acc[o][1]);
                    acc[o][2] = fmaf(ua, v.z, acc[o][2]);
                    acc[o][3] = fmaf(ua, v.w, acc[o][3]);
                }
            }
            if constexpr (R % 2 == 0) {
#pragma unroll
                for (int o = 0; o < R; o += 2)
                    put2(rb * R + o, c4, acc[o][0], acc[o][1], acc[o][2], acc[o][3],
                         acc[o + 1][0], acc[o + 1][1], acc[o + 1][2], acc[o + 1][3]);
            } else {
#pragma unroll
                for (int o = 0; o < R; ++o)
                    put1(rb * R + o, c4, acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
            }
        }
    }
}

// Horizontal pass: acc[o][q] = sum_b vs[b] V[ty R + o][4 tx + SHIFT + q + b];
// with an even R, rows (o, o + 1) advance together in packed FMAs on the
// interleaved pairs (V[o][c], V[o + 1][c]).
template <int KW, int R>
__device__ __forceinline__ void sep_horz(const float* V, const float* vs, int ty, int tx,
                                         float acc[R][4]) {
    using G = Geom<KW>;
    if constexpr (R % 2 == 0) {
        float2 h2[KW];
#pragma unroll
        for (int b = 0; b < KW; ++b) h2[b] = make_float2(vs[b], vs[b]);
#pragma unroll
        for (int o = 0; o < R; o += 2) {
            float2 p[4 * G::NW4];
            const float4* src = reinterpret_cast<const float4*>(V + vidx(ty * R + o, 4 * tx, G::WP));
#pragma unroll
            for (int k = 0; k < 2 * G::NW4; ++k) {
                const float4 v = src[k];
                p[2 * k] = make_float2(v.x, v.y);
                p[2 * k + 1] = make_float2(v.z, v.w);
            }
            float2 a2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) a2[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < KW; ++b) {
#pragma unroll
                for (int q = 0; q < 4; ++q) a2[q] = __ffma2_rn(h2[b], p[G::SHIFT + q + b], a2[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[o][q] = a2[q].x;
                acc[o + 1][q] = a2[q].y;
            }
        }
    } else {
        float hr[KW];
#pragma unroll
        for (int b = 0; b < KW; ++b) hr[b] = vs[b];
#pragma unroll
        for (int o = 0; o < R; ++o) {
            const int row = ty * R + o;
            float w[4 * G::NW4];
#pragma unroll
            for (int c = 0; c < 4 * G::NW4; ++c) w[c] = V[vidx(row, 4 * tx + c, G::WP)];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[o][q] = 0.f;
#pragma unroll
            for (int b = 0; b < KW; ++b) {
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[o][q] = fmaf(hr[b], w[G::SHIFT + q + b], acc[o][q]);
            }
        }
    }
}

__device__ __forceinline__ float update1(const UpdateParams& p, float xv, float gq, float dv,
                                         float zq, float z2v) {
    float v = xv - p.gamma * (gq * p.inv_s2);
    if (p.z2) v -= p.c_z2 * (xv - z2v);   // Poisson: (gamma / rho2)(x - z2)
    if (p.d) v += p.d_residual ? -p.c_prior * dv : p.c_prior * (dv - xv);
    const float pr = fminf(fmaxf(xv, 0.f), 1.f);
    v += p.c_proj * (pr - xv);
    v += p.c_noise * zq;
    return v;
}

__device__ __forceinline__ void welford1(float v, float inv_n, float& mo, float& q) {
    const float delta = v - mo;
    const float mn = mo + delta * inv_n;
    q = q + delta * (v - mn);
    mo = mn;
}

}  // namespace pnp
