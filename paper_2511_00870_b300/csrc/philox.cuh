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

// ln(u) for u = ((w >> 8) + 1/2) 2^-24. Both branches feed an exactly
// representable FP32 argument: u itself when u < 1/2, and 1 - u to log1pf
// otherwise (u = (m + 1/2) 2^-24 is not exact in FP32 once m >= 2^23).
__device__ __forceinline__ float log_uniform(uint32_t w) {
    const uint32_t m = w >> 8;
    if (m < (1u << 23)) return logf(((float)m + 0.5f) * 5.9604644775390625e-08f);
    return log1pf(-(((float)((1u << 24) - 1u - m) + 0.5f) * 5.9604644775390625e-08f));
}

// sin / cos of 2 pi u with u as above, via sincospif on the exact argument
// 2u (u < 1/2) or 2u - 2 (u >= 1/2).
__device__ __forceinline__ void sincos_2pi_uniform(uint32_t w, float* s, float* c) {
    const uint32_t m = w >> 8;
    float a;
    if (m < (1u << 23)) a = ((float)m + 0.5f) * 1.1920928955078125e-07f;
    else a = -(((float)((1u << 24) - 1u - m) + 0.5f) * 1.1920928955078125e-07f);
    sincospif(a, s, c);
}

// The four normals of group m: Box-Muller on (w0, w1) and (w2, w3). `stream`
// is the counter's last word: 0 drives the x-update's xi, 1 and 2 the
// auxiliary variables' zeta_1 and zeta_2 of the Poisson sampler.
__device__ __forceinline__ void normals_group(uint32_t m, uint32_t t, uint32_t chain, uint32_t k0,
                                              uint32_t k1, float z[4], uint32_t stream = 0) {
    const U4 r = philox4x32_10(U4{m, t, chain, stream}, k0, k1);
    float s, c;
    float rad = sqrtf(-2.0f * log_uniform(r.x));
    sincos_2pi_uniform(r.y, &s, &c);
    z[0] = rad * c;
    z[1] = rad * s;
    rad = sqrtf(-2.0f * log_uniform(r.z));
    sincos_2pi_uniform(r.w, &s, &c);
    z[2] = rad * c;
    z[3] = rad * s;
}

}  // namespace pnp
