// Counter-based Gaussian draws for the Langevin noise xi (Eq. 8).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies, xor with the odd words and the round key, word
// permutation; the key is bumped by the golden-ratio Weyl constants between
// rounds. Counter (n/4, t, chain, 0), key (seed_lo, seed_hi): the draw for a
// pixel depends only on (seed, t, chain, n), so it is the same for any block
// split, tile shape or batch mix.
#pragma once
#include <stdint.h>

namespace pnp {

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// -2 ln(u) for u = ((w >> 8) + 1/2) 2^-24, from the hardware base-2
// logarithm (__logf) where that is accurate enough and a power series where it
// is not, with no divergent branch:
// * u < 1/2: ln u = __logf(u), u exact; CUDA bounds __logf off [1/2, 2] by
//   3 ulp, so the relative error of -2 ln u stays below 4e-7;
// * u >= 1/2: ln u = ln(1 - v) with v = 1 - u = (2^24 - 1 - m + 1/2) 2^-24
//   exact. For v < 1/8 the series -(v + v^2/2 + ... + v^9/9), whose
//   truncation is below v^10 / (10 (1 - v)) < 2e-10 v; for v >= 1/8,
//   __logf(1 - v) with 1 - v in [1/2, 7/8] rounded to FP32 (at most 2^-25,
//   i.e. 6e-8 on ln), where CUDA bounds the absolute error of __logf by
//   2^-21.41: together below 3.2e-6 of |ln u| >= 0.13.
__device__ __forceinline__ float neg2_log_uniform(uint32_t w) {
    const uint32_t m = w >> 8;
    const bool lo = m < (1u << 23);
    const float v = ((float)((1u << 24) - 1u - m) + 0.5f) * 5.9604644775390625e-08f;
    const float u = lo ? ((float)m + 0.5f) * 5.9604644775390625e-08f : 1.0f - v;
    float sr = 1.0f / 9.0f;
    sr = fmaf(sr, v, 1.0f / 8.0f);
    sr = fmaf(sr, v, 1.0f / 7.0f);
    sr = fmaf(sr, v, 1.0f / 6.0f);
    sr = fmaf(sr, v, 1.0f / 5.0f);
    sr = fmaf(sr, v, 0.25f);
    sr = fmaf(sr, v, 1.0f / 3.0f);
    sr = fmaf(sr, v, 0.5f);
    sr = fmaf(sr, v, 1.0f);
    const float series = 2.0f * (v * sr);           // -2 ln(1 - v)
    const float hw = -2.0f * __logf(u);
    return (!lo && v < 0.125f) ? series : hw;
}

// sin and cos of 2 pi u (u as above) from the hardware sine and cosine
// (__sincosf) of the angle pi a, a = 2u (u < 1/2) or 2u - 2 (u >= 1/2), exact
// in FP32 and in [-1, 1): on [-pi, pi] CUDA bounds their absolute error by
// 2^-21.41; the rounding of pi a adds at most 2^-22 pi.
__device__ __forceinline__ void sincos_2pi_uniform(uint32_t w, float* s, float* c) {
    const uint32_t m = w >> 8;
    float a;
    if (m < (1u << 23)) a = ((float)m + 0.5f) * 1.1920928955078125e-07f;
    else a = -(((float)((1u << 24) - 1u - m) + 0.5f) * 1.1920928955078125e-07f);
    __sincosf(a * 3.14159265358979323846f, s, c);
}

// The four normals of group m: Box-Muller on (w0, w1) and (w2, w3). `stream`
// is the counter's last word: 0 drives the x-update's xi, 1 and 2 the
// auxiliary variables' zeta_1 and zeta_2 of the Poisson sampler.
__device__ __forceinline__ void normals_group(uint32_t m, uint32_t t, uint32_t chain, uint32_t k0,
                                              uint32_t k1, float z[4], uint32_t stream = 0) {
    const U4 r = philox4x32_10(U4{m, t, chain, stream}, k0, k1);
    float s, c;
    float rad = sqrtf(neg2_log_uniform(r.x));
    sincos_2pi_uniform(r.y, &s, &c);
    z[0] = rad * c;
    z[1] = rad * s;
    rad = sqrtf(neg2_log_uniform(r.z));
    sincos_2pi_uniform(r.w, &s, &c);
    z[2] = rad * c;
    z[3] = rad * s;
}

}  // namespace pnp
