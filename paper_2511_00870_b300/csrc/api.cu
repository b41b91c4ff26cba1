// C ABI of libpnp: argument checking, device buffers, step scheduling and
// CUDA-graph replay around the kernels of k_stencil.cu, k_conv_simt.cu and
// k_conv_tc.cu. Every compute step runs on the GPU; the host only validates,
// allocates, derives the step sizes (Eq. 10) and enqueues work.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "pnp_internal.h"

namespace pnp {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
pnp_status fail(pnp_status st, const std::string& msg) {
    g_err = msg;
    return st;
}
pnp_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PNP_ENOMEM : PNP_ECUDA;
}

pnp_status take_timeout(int* flag, cudaStream_t s, const char* who) {
    if (!flag) return PNP_OK;
    int h = 0;
    PNP_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PNP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h == 0) return PNP_OK;
    PNP_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    PNP_CUDA_TRY(cudaStreamSynchronize(s));
    return fail(PNP_ETIMEOUT, std::string(who) +
                                  ": a bounded wait on the device (tensor-core denoiser layer or "
                                  "pipelined update) ran out; the affected results are incomplete");
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

// ------------------------------------------------------------ kernel timer
struct TimerSlot {
    std::vector<cudaEvent_t> begin, end;
    size_t used = 0;
};
static TimerSlot g_timers[T_COUNT];
static bool g_timing = false;
static bool g_pdl = true;
bool pdl_enabled() { return g_pdl; }
static std::atomic<int64_t> g_launches{0};
static std::atomic<int> g_spectral{1};   // spectral gradient for eligible wide-blur problems
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static const char* g_timer_names[T_COUNT] = {"blur", "update", "conv_fp32", "conv_tc", "conv_edge", "conv_last",
                                              "zupdate"};

bool timer_enabled() { return g_timing; }
void timer_begin(int id, cudaStream_t s) {
    if (!g_timing) return;
    TimerSlot& t = g_timers[id];
    if (t.used == t.begin.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        t.begin.push_back(a);
        t.end.push_back(b);
    }
    cudaEventRecord(t.begin[t.used], s);
}
void timer_end(int id, cudaStream_t s) {
    if (!g_timing) return;
    TimerSlot& t = g_timers[id];
    cudaEventRecord(t.end[t.used], s);
    ++t.used;
}

cudaError_t conv_tc_layer(const __nv_bfloat16* in, const __nv_bfloat16* wblob, const float* bias_host,
                          int ny, int nx, int nimg, const Rect* rects, __nv_bfloat16* out,
                          int* err, cudaStream_t s);

}  // namespace pnp

using namespace pnp;


// ------------------------------------------------------------------ helpers

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static pnp_status dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return PNP_OK;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(PNP_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return PNP_OK;
}

static void dfree(void* p) {
    if (p) cudaFree(p);
}

static uint16_t f32_to_bf16_rne(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16 | ((u & 0xffff) ? 0x40 : 0));
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

static float bf16_to_f32(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// ------------------------------------------------------------------ misc API

extern "C" const char* pnp_last_error(void) { return g_err.c_str(); }
extern "C" const char* pnp_version(void) { return "pnp-b300 0.1 (sm_103a)"; }

extern "C" pnp_status pnp_stepsizes(double hnorm, double sigma, double alpha, double eps,
                                    double lip_eps, double c, double* lambda, double* gamma) {
    if (!(hnorm > 0) || !(sigma > 0) || !(eps > 0) || alpha < 0 || lip_eps < 0 || !(c > 0) ||
        !(c < 1) || !lambda || !gamma)
        return fail(PNP_EINVAL, "pnp_stepsizes: need hnorm, sigma, eps > 0, alpha, L_eps >= 0, 0 < c < 1");
    const double L = hnorm * hnorm / (sigma * sigma);
    const double prior = alpha * lip_eps / (eps * eps);
    const double lam = 0.99 / (4.0 * L + 2.0 * prior);
    *lambda = lam;
    *gamma = c / (3.0 * (L + prior + 1.0 / lam));
    return PNP_OK;
}

extern "C" pnp_status pnp_stepsizes_poisson(double hnorm, double eta, double rho1, double rho2,
                                            double alpha, double eps, double lip_eps, double c,
                                            double* lambda, double* gamma, double* kappa1,
                                            double* kappa2) {
    if (!(hnorm > 0) || !(eta > 0) || !(rho1 > 0) || !(rho2 > 0) || !(eps > 0) || alpha < 0 ||
        lip_eps < 0 || !(c > 0) || !(c < 1) || !lambda || !gamma || !kappa1 || !kappa2)
        return fail(PNP_EINVAL, "pnp_stepsizes_poisson: need hnorm, eta, rho1, rho2, eps > 0, "
                                "alpha, L_eps >= 0, 0 < c < 1");
    const double c1 = eta * hnorm * eta * hnorm / rho1, c2 = 1.0 / rho2;
    const double prior = alpha * lip_eps / (eps * eps);
    const double lam = 0.99 / (4.0 * c1 + 4.0 * c2 + 2.0 * prior);
    *lambda = lam;
    *gamma = c / (3.0 * (prior + c1 + c2 + 1.0 / lam));
    *kappa1 = 0.99 * rho1;
    *kappa2 = 0.99 * rho2;
    return PNP_OK;
}

// ------------------------------------------------------------------ denoiser

extern "C" pnp_status pnp_create_denoiser(int K, int F, const float* weights, const float* biases,
                                          double lipschitz_eps, pnp_denoiser** out) {
    if (!out) return fail(PNP_EINVAL, "pnp_create_denoiser: out is NULL");
    *out = nullptr;
    if (K < 2 || !(F == 16 || F == 32 || F == 64) || !weights || !biases || !(lipschitz_eps >= 0))
        return fail(PNP_EINVAL, "pnp_create_denoiser: need K >= 2, F in {16,32,64}, weights, biases");
    pnp_denoiser* den = new pnp_denoiser();
    DenoiserDev& D = den->dev;
    D.K = K;
    D.F = F;
    D.lip = lipschitz_eps;
    cudaGetDevice(&den->device);
    {
        pnp_status fs = dalloc(&den->err, 1);
        if (fs != PNP_OK) {
            pnp_destroy_denoiser(den);
            return fs;
        }
        cudaMemset(den->err, 0, sizeof(int));
        // the allocation-free entry point's fixed area is reserved now, while
        // device memory is still available, rather than at its first call
        if (noalloc_reserve() != PNP_OK) {
            cudaGetLastError();
            set_error("");
        }
    }
    std::vector<int> cin(K), cout(K);
    for (int k = 0; k < K; ++k) {
        cin[k] = k == 0 ? 1 : F;
        cout[k] = k == K - 1 ? 1 : F;
    }
    D.w32_off = new int64_t[K];
    D.b_off = new int64_t[K];
    int64_t nw = 0, nb = 0, wsrc = 0;
    std::vector<int64_t> src_off(K);
    for (int k = 0; k < K; ++k) {
        D.w32_off[k] = nw;
        D.b_off[k] = nb;
        src_off[k] = wsrc;
        const int64_t sz = (int64_t)cin[k] * 9 * cout[k];
        wsrc += sz;
        nw += (sz + 3) & ~(int64_t)3;
        nb += (cout[k] + 3) & ~3;
    }
    // FP32 [cin][9][cout] per layer
    std::vector<float> w32(nw, 0.f), b32(nb, 0.f);
    int64_t bsrc = 0;
    for (int k = 0; k < K; ++k) {
        const float* W = weights + src_off[k];
        for (int co = 0; co < cout[k]; ++co)
            for (int ci = 0; ci < cin[k]; ++ci)
                for (int t = 0; t < 9; ++t)
                    w32[D.w32_off[k] + ((int64_t)ci * 9 + t) * cout[k] + co] =
                        W[((int64_t)co * cin[k] + ci) * 9 + t];
        for (int co = 0; co < cout[k]; ++co) b32[D.b_off[k] + co] = biases[bsrc + co];
        bsrc += cout[k];
    }
    pnp_status st = PNP_OK;
    if ((st = dalloc(&D.w32, nw)) != PNP_OK || (st = dalloc(&D.b32, nb)) != PNP_OK) {
        pnp_destroy_denoiser(den);
        return st;
    }
    cudaMemcpy(D.w32, w32.data(), nw * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(D.b32, b32.data(), nb * 4, cudaMemcpyHostToDevice);
    D.hw = new float[wsrc];
    D.hb = new float[bsrc];
    memcpy(D.hw, weights, wsrc * 4);
    memcpy(D.hb, biases, bsrc * 4);
    if (F == 64) {
        // tensor-core blobs of the F -> F layers, BF16 [dx][cg][dy*64 + co][8 ci]:
        // for a fixed column shift dx the three kernel rows are stacked along N
        const int nmid = K - 2;
        std::vector<uint16_t> blob((size_t)std::max(nmid, 1) * 9 * 8 * 64 * 8, 0);
        for (int m = 0; m < nmid; ++m) {
            const float* W = weights + src_off[m + 1];
            for (int dx = 0; dx < 3; ++dx)
                for (int cg = 0; cg < 8; ++cg)
                    for (int dy = 0; dy < 3; ++dy)
                        for (int co = 0; co < 64; ++co)
                            for (int c8 = 0; c8 < 8; ++c8)
                                blob[(((((size_t)m * 3 + dx) * 8 + cg) * 192 + dy * 64 + co) * 8) + c8] =
                                    f32_to_bf16_rne(W[((int64_t)co * 64 + cg * 8 + c8) * 9 + dy * 3 + dx]);
        }
        // last layer: [dx][cg][16 rows][8 ci], row dy = kernel row dy, rows 3..15 zero
        std::vector<uint16_t> blob_last(3 * 8 * 16 * 8, 0);
        for (int dx = 0; dx < 3; ++dx)
            for (int cg = 0; cg < 8; ++cg)
                for (int dy = 0; dy < 3; ++dy)
                    for (int c8 = 0; c8 < 8; ++c8)
                        blob_last[(((size_t)dx * 8 + cg) * 16 + dy) * 8 + c8] =
                            f32_to_bf16_rne(weights[src_off[K - 1] + (int64_t)(cg * 8 + c8) * 9 + dy * 3 + dx]);
        // first layer: [kc][co][8], K = [w_hi(9) | w_hi(9) | w_lo(9) | b_hi | b_lo | 0 0 0]
        std::vector<uint16_t> blob_first(4 * 64 * 8, 0);
        for (int co = 0; co < 64; ++co) {
            auto put = [&](int k, float v) { blob_first[((size_t)(k / 8) * 64 + co) * 8 + k % 8] = f32_to_bf16_rne(v); };
            auto head = [](float v) { return bf16_to_f32(f32_to_bf16_rne(v)); };
            for (int t = 0; t < 9; ++t) {
                const float w = weights[src_off[0] + (int64_t)co * 9 + t];
                put(t, w);
                put(9 + t, w);
                put(18 + t, w - head(w));
            }
            put(27, biases[co]);
            put(28, biases[co] - head(biases[co]));
        }
        if ((st = dalloc(&D.wtc_first, blob_first.size())) != PNP_OK) {
            pnp_destroy_denoiser(den);
            return st;
        }
        cudaMemcpy(D.wtc_first, blob_first.data(), blob_first.size() * 2, cudaMemcpyHostToDevice);
        if ((st = dalloc(&D.wtc_last, blob_last.size())) != PNP_OK) {
            pnp_destroy_denoiser(den);
            return st;
        }
        cudaMemcpy(D.wtc_last, blob_last.data(), blob_last.size() * 2, cudaMemcpyHostToDevice);
        // E4M3 variant: per-output-channel scales amax / 448, same stacking with
        // 16-channel groups: [dx][4 cg][rows][16 ci]
        D.w8_scale = new float[(size_t)K * 64];
        for (size_t i = 0; i < (size_t)K * 64; ++i) D.w8_scale[i] = 1.f;
        for (int k = 1; k < K; ++k) {
            const float* W = weights + src_off[k];
            for (int co = 0; co < cout[k]; ++co) {
                float m = 0.f;
                for (int i = 0; i < 64 * 9; ++i) m = std::max(m, std::fabs(W[(int64_t)co * 64 * 9 + i]));
                D.w8_scale[k * 64 + co] = m > 0.f ? m / 448.f : 1.f;
            }
        }
        std::vector<float> st8((size_t)std::max(nmid, 1) * 3 * 4 * 192 * 16, 0.f);
        for (int m = 0; m < nmid; ++m) {
            const float* W = weights + src_off[m + 1];
            for (int dx = 0; dx < 3; ++dx)
                for (int cg = 0; cg < 4; ++cg)
                    for (int dy = 0; dy < 3; ++dy)
                        for (int co = 0; co < 64; ++co)
                            for (int c16 = 0; c16 < 16; ++c16)
                                st8[((((size_t)m * 3 + dx) * 4 + cg) * 192 + dy * 64 + co) * 16 + c16] =
                                    W[((int64_t)co * 64 + cg * 16 + c16) * 9 + dy * 3 + dx] /
                                    D.w8_scale[(m + 1) * 64 + co];
        }
        std::vector<float> st8l(3 * 4 * 16 * 16, 0.f);
        for (int dx = 0; dx < 3; ++dx)
            for (int cg = 0; cg < 4; ++cg)
                for (int dy = 0; dy < 3; ++dy)
                    for (int c16 = 0; c16 < 16; ++c16)
                        st8l[(((size_t)dx * 4 + cg) * 16 + dy) * 16 + c16] =
                            weights[src_off[K - 1] + (int64_t)(cg * 16 + c16) * 9 + dy * 3 + dx] /
                            D.w8_scale[(K - 1) * 64];
        float* stage = nullptr;
        if ((st = dalloc(&D.wtc8, st8.size())) != PNP_OK || (st = dalloc(&D.wtc8_last, st8l.size())) != PNP_OK ||
            (st = dalloc(&stage, st8.size())) != PNP_OK) {
            pnp_destroy_denoiser(den);
            return st;
        }
        cudaMemcpy(stage, st8.data(), st8.size() * 4, cudaMemcpyHostToDevice);
        convert_e4m3(stage, D.wtc8, st8.size(), 0);
        cudaMemcpy(stage, st8l.data(), st8l.size() * 4, cudaMemcpyHostToDevice);
        convert_e4m3(stage, D.wtc8_last, st8l.size(), 0);
        cudaDeviceSynchronize();
        cudaFree(stage);
        int64_t b_last = 0;
        for (int k = 0; k < K - 1; ++k) b_last += cout[k];
        D.last_bias = biases[b_last];
        if ((st = dalloc(&D.wtc, blob.size())) != PNP_OK) {
            pnp_destroy_denoiser(den);
            return st;
        }
        cudaMemcpy(D.wtc, blob.data(), blob.size() * 2, cudaMemcpyHostToDevice);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        pnp_destroy_denoiser(den);
        return cuda_fail(e, "pnp_create_denoiser");
    }
    *out = den;
    return PNP_OK;
}

extern "C" pnp_status pnp_create_ddfb(int K, int P, const float* filters, const float* gammas,
                                      double ht, pnp_denoiser** out) {
    if (!out) return fail(PNP_EINVAL, "pnp_create_ddfb: out is NULL");
    *out = nullptr;
    if (K < 2 || K > 32 || !(P == 16 || P == 32 || P == 64) || !filters || !gammas ||
        !(ht > 0) || !std::isfinite(ht))
        return fail(PNP_EINVAL, "pnp_create_ddfb: need 2 <= K <= 32, P in {16,32,64}, filters, "
                                "gammas and ht > 0");
    for (int i = 0; i < K * P * 9; ++i)
        if (!std::isfinite(filters[i])) return fail(PNP_EINVAL, "pnp_create_ddfb: filters not finite");
    for (int k = 0; k < K; ++k)
        if (!(gammas[k] > 0) || !std::isfinite(gammas[k]))
            return fail(PNP_EINVAL, "pnp_create_ddfb: gammas must be > 0");
    pnp_denoiser* den = new pnp_denoiser();
    DenoiserDev& D = den->dev;
    cudaGetDevice(&den->device);   // host-only: the DDFB kernels have no bounded waits
    D.K = K;
    D.F = P;
    D.lip = 1.0;   // D is a (relaxed) proximity operator: Id - D is nonexpansive
    D.ddfb = true;
    D.ddfb_w = new float[(size_t)K * P * 9];
    memcpy(D.ddfb_w, filters, sizeof(float) * K * P * 9);
    for (int k = 0; k < K; ++k) D.ddfb_gamma[k] = gammas[k];
    D.ddfb_ht = (float)ht;
    *out = den;
    return PNP_OK;
}

extern "C" void pnp_destroy_denoiser(pnp_denoiser* den) {
    if (!den) return;
    DenoiserDev& D = den->dev;
    delete[] D.ddfb_w;
    dfree(D.w32);
    dfree(D.b32);
    dfree(D.wtc);
    dfree(D.wtc_last);
    dfree(D.wtc_first);
    dfree(D.wtc8);
    dfree(D.wtc8_last);
    delete[] D.w8_scale;
    dfree(den->scratch);
    dfree(den->err);
    delete[] D.w32_off;
    delete[] D.b_off;
    delete[] D.hw;
    delete[] D.hb;
    delete den;
}

// ------------------------------------------------------------------ operators

static pnp_status check_blur_args(const void* x, const void* h, int kh, int kw, int ny, int nx,
                                  int nimg, const void* out, const char* who) {
    if (!x || !h || !out) return fail(PNP_EINVAL, std::string(who) + ": NULL pointer");
    if (ny < 1 || nx < 1 || nimg < 1) return fail(PNP_EINVAL, std::string(who) + ": empty image");
    if (kh < 1 || kw < 1 || !(kh & 1) || !(kw & 1) || kh > WIDE_MAXK || kw > WIDE_MAXK)
        return fail(PNP_EINVAL, std::string(who) + ": kernel sizes must be odd and <= 129");
    if (kh > ny || kw > nx)
        return fail(PNP_EINVAL, std::string(who) + ": kernel larger than the image");
    return PNP_OK;
}

extern "C" pnp_status pnp_blur(const float* x, const float* y, const float* h, int kh, int kw,
                               int ny, int nx, int nimg, float* r, void* stream) {
    PNP_TRY(check_blur_args(x, h, kh, kw, ny, nx, nimg, r, "pnp_blur"));
    PNP_CUDA_TRY(launch_blur(x, y, h, kh, kw, ny, nx, nimg, r, (cudaStream_t)stream));
    return PNP_OK;
}

extern "C" pnp_status pnp_blur_adjoint(const float* r, const float* h, int kh, int kw, int ny,
                                       int nx, int nimg, float scale, float* g, void* stream) {
    PNP_TRY(check_blur_args(r, h, kh, kw, ny, nx, nimg, g, "pnp_blur_adjoint"));
    PNP_CUDA_TRY(launch_blur_adjoint(r, h, kh, kw, ny, nx, nimg, scale, g, (cudaStream_t)stream));
    return PNP_OK;
}

// block table for the block + halo mode (floor rule per axis, Eq. 7)
static std::vector<BlockDesc> make_blocks(int ny, int nx, int by, int bx, int nimg, int* maxh,
                                          int* maxw) {
    std::vector<BlockDesc> v;
    *maxh = *maxw = 0;
    for (int img = 0; img < nimg; ++img)
        for (int i = 0; i < by; ++i)
            for (int j = 0; j < bx; ++j) {
                BlockDesc b;
                b.img = img;
                b.r0 = (int)((int64_t)i * ny / by);
                b.r1 = (int)((int64_t)(i + 1) * ny / by);
                b.c0 = (int)((int64_t)j * nx / bx);
                b.c1 = (int)((int64_t)(j + 1) * nx / bx);
                *maxh = std::max(*maxh, b.r1 - b.r0);
                *maxw = std::max(*maxw, b.c1 - b.c0);
                v.push_back(b);
            }
    return v;
}

static size_t denoise_scratch_bytes(const DenoiserDev& D, pnp_precision prec, int ny, int nx,
                                    int nimg) {
    if (prec == PNP_FP32) return denoise_fp32_scratch(D, ny, nx, nimg);
    if (prec == PNP_FP8) return denoise_fp8_scratch(D, ny, nx, nimg);
    return denoise_bf16_scratch(D, ny, nx, nimg);
}

static cudaError_t run_denoise(const DenoiserDev& D, pnp_precision prec, bool residual, const float* x, int ny,
                               int nx, int nimg, const Rect* rects, float* d, void* scratch,
                               cudaStream_t s, int* err) {
    if (prec == PNP_FP32) return denoise_fp32(D, x, ny, nx, nimg, rects, d, (float*)scratch, s);
    if (prec == PNP_FP8) return denoise_fp8(D, x, ny, nx, nimg, rects, d, scratch, s, residual, err);
    return denoise_bf16(D, x, ny, nx, nimg, rects, d, scratch, s, residual, err);
}

static pnp_status check_denoise_args(const pnp_denoiser* den, pnp_precision prec, int ny, int nx,
                                     int nimg, int by, int bx, int halo) {
    if (!den) return fail(PNP_EINVAL, "denoiser is NULL");
    if (ny < 1 || nx < 1 || nimg < 1) return fail(PNP_EINVAL, "empty image");
    if (prec != PNP_FP32 && prec != PNP_BF16 && prec != PNP_FP8)
        return fail(PNP_ENOTSUP, "unknown precision");
    if (den->dev.ddfb && prec != PNP_FP32)
        return fail(PNP_ENOTSUP, "the DDFB denoiser runs in FP32");
    if (den->dev.ddfb && halo > 0)
        return fail(PNP_EINVAL, "the DDFB denoiser uses the direct layout (halo = 0)");
    if (prec != PNP_FP32 && den->dev.F != 64) return fail(PNP_EINVAL, "BF16/FP8 paths need F = 64");
    if (halo < 0) return fail(PNP_EINVAL, "halo must be >= 0");
    if (halo > 0 && (by < 1 || bx < 1 || by > ny || bx > nx))
        return fail(PNP_EINVAL, "blocks must be >= 1 and <= the image size");
    return PNP_OK;
}

extern "C" pnp_status pnp_denoiser_calibrate_fp8(pnp_denoiser* den, const float* x, int ny, int nx,
                                                 int nimg, void* stream) {
    if (!den || !x || ny < 1 || nx < 1 || nimg < 1)
        return fail(PNP_EINVAL, "pnp_denoiser_calibrate_fp8: bad arguments");
    DenoiserDev& D = den->dev;
    if (D.F != 64 || !D.wtc8) return fail(PNP_EINVAL, "FP8 variant needs F = 64");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = denoise_fp32_scratch(D, ny, nx, nimg);
    float* scratch = nullptr;
    float* dtmp = nullptr;
    unsigned* amax = nullptr;
    PNP_TRY(dalloc(&scratch, need / 4));
    pnp_status st = dalloc(&dtmp, (size_t)nimg * ny * nx);
    if (st == PNP_OK) st = dalloc(&amax, (size_t)D.K);
    std::vector<unsigned> h(D.K, 0);
    cudaError_t e = cudaSuccess;
    if (st == PNP_OK) {
        e = denoise_fp32_amax(D, x, ny, nx, nimg, dtmp, scratch, amax, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), amax, 4 * D.K, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    dfree(scratch);
    dfree(dtmp);
    dfree(amax);
    if (st != PNP_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "pnp_denoiser_calibrate_fp8");
    // input of layer k = output of layer k-1; headroom x2 over the calibration maximum
    for (int k = 1; k < D.K; ++k) {
        float m;
        memcpy(&m, &h[k - 1], 4);
        D.a8_scale[k] = (m > 0.f ? 2.f * m : 1.f) / 448.f;
    }
    D.fp8_calibrated = true;
    return PNP_OK;
}

extern "C" pnp_status pnp_denoise(const pnp_denoiser* den, pnp_precision prec, const float* x,
                                  int ny, int nx, int nimg, int blocks_y, int blocks_x, int halo,
                                  float* d, void* stream) {
    PNP_TRY(check_denoise_args(den, prec, ny, nx, nimg, blocks_y, blocks_x, halo));
    if (!x || !d) return fail(PNP_EINVAL, "pnp_denoise: NULL pointer");
    if (prec == PNP_FP8 && !den->dev.fp8_calibrated)
        PNP_TRY(pnp_denoiser_calibrate_fp8(const_cast<pnp_denoiser*>(den), x, ny, nx, nimg, stream));
    pnp_denoiser* dn = const_cast<pnp_denoiser*>(den);
    const DenoiserDev& D = den->dev;
    cudaStream_t s = (cudaStream_t)stream;
    if (halo == 0) {
        const size_t need = denoise_scratch_bytes(D, prec, ny, nx, nimg);
        if (dn->scratch_bytes < need) {
            PNP_CUDA_TRY(cudaStreamSynchronize(s));
            dfree(dn->scratch);
            dn->scratch = nullptr;
            dn->scratch_bytes = 0;
            PNP_TRY(dalloc((uint8_t**)&dn->scratch, need));
            PNP_CUDA_TRY(cudaMemset(dn->scratch, 0, need));
            dn->scratch_bytes = need;
        }
        PNP_CUDA_TRY(run_denoise(D, prec, false, x, ny, nx, nimg, nullptr, d, dn->scratch, s, dn->err));
        return PNP_OK;
    }
    // block + halo: gather extended blocks, run the network per tile, scatter interiors
    int mh, mw;
    std::vector<BlockDesc> bl = make_blocks(ny, nx, blocks_y, blocks_x, nimg, &mh, &mw);
    const int ty = mh + 2 * halo, tx = mw + 2 * halo, nb = (int)bl.size();
    const size_t tile_floats = (size_t)nb * ty * tx;
    const size_t need_net = denoise_scratch_bytes(D, prec, ty, tx, nb);
    const size_t need = need_net + 2 * tile_floats * 4 + nb * sizeof(Rect) + nb * sizeof(BlockDesc) + 1024;
    PNP_CUDA_TRY(cudaStreamSynchronize(s));
    if (dn->scratch_bytes < need) {
        dfree(dn->scratch);
        dn->scratch = nullptr;
        dn->scratch_bytes = 0;
        PNP_TRY(dalloc((uint8_t**)&dn->scratch, need));
        PNP_CUDA_TRY(cudaMemset(dn->scratch, 0, need));
        dn->scratch_bytes = need;
    }
    uint8_t* p = (uint8_t*)dn->scratch;
    void* net_scratch = p;
    p += (need_net + 255) & ~(size_t)255;
    float* tiles = (float*)p;
    p += tile_floats * 4;
    float* dtiles = (float*)p;
    p += tile_floats * 4;
    Rect* rects = (Rect*)p;
    p += nb * sizeof(Rect);
    BlockDesc* blocks = (BlockDesc*)p;
    PNP_CUDA_TRY(cudaMemcpyAsync(blocks, bl.data(), nb * sizeof(BlockDesc), cudaMemcpyHostToDevice, s));
    PNP_CUDA_TRY(launch_gather_blocks(x, ny, nx, blocks, nb, halo, ty, tx, tiles, rects, s));
    PNP_CUDA_TRY(run_denoise(D, prec, false, tiles, ty, tx, nb, rects, dtiles, net_scratch, s, dn->err));
    PNP_CUDA_TRY(launch_scatter_blocks(dtiles, ny, nx, blocks, nb, halo, ty, tx, d, s));
    PNP_CUDA_TRY(cudaStreamSynchronize(s));   // the host block table must outlive the copy
    return PNP_OK;
}

extern "C" pnp_status pnp_denoise_status(const pnp_denoiser* den, void* stream) {
    if (!den) return fail(PNP_EINVAL, "pnp_denoise_status: denoiser is NULL");
    return take_timeout(den->err, (cudaStream_t)stream, "pnp_denoise");
}

extern "C" pnp_status pnp_debug_inject_tc_timeout(int cta, int load_index,
                                                  long long budget_cycles) {
    if (cta < 0 || load_index < 0 || budget_cycles < 1000)
        return fail(PNP_EINVAL, "pnp_debug_inject_tc_timeout: need cta >= 0, load_index >= 0 and "
                                "budget_cycles >= 1000");
    tc_inject_timeout(cta, load_index, budget_cycles);
    return PNP_OK;
}

extern "C" pnp_status pnp_debug_inject_update_timeout(int cta, int tile_index,
                                                      long long budget_cycles) {
    if (cta < 0 || tile_index < 0 || budget_cycles < 1000)
        return fail(PNP_EINVAL, "pnp_debug_inject_update_timeout: need cta >= 0, tile_index >= 0 "
                                "and budget_cycles >= 1000");
    os_inject_timeout(cta, tile_index, budget_cycles);
    return PNP_OK;
}

static pnp_status fill_update_params(UpdateParams& u, float* x, const float* r, const float* d,
                                     const float* h, int kh, int kw, int ny, int nx, int nchain,
                                     double sigma, double alpha, double eps, double lambda,
                                     double gamma, uint64_t seed, int noise) {
    if (!(sigma > 0) || !(gamma > 0)) return fail(PNP_EINVAL, "sigma and gamma must be > 0");
    if (d && !(eps > 0)) return fail(PNP_EINVAL, "eps must be > 0 with a prior term");
    u.x = x;
    u.r = r;
    u.d = d;
    u.h = h;
    u.kh = kh;
    u.kw = kw;
    u.ny = ny;
    u.nx = nx;
    u.nchain = nchain;
    u.inv_s2 = (float)(1.0 / (sigma * sigma));
    u.gamma = (float)gamma;
    u.c_prior = d ? (float)(alpha * gamma / (eps * eps)) : 0.f;
    u.c_proj = lambda > 0 ? (float)(gamma / lambda) : 0.f;
    u.c_noise = noise ? (float)std::sqrt(2.0 * gamma) : 0.f;
    u.key0 = (uint32_t)(seed & 0xffffffffu);
    u.key1 = (uint32_t)(seed >> 32);
    u.t = 0;
    u.t_dev = nullptr;
    u.mean = nullptr;
    u.m2 = nullptr;
    u.inv_n = 0.f;
    u.burn_dev = nullptr;
    u.d_residual = 0;
    u.arrive = nullptr;
    u.tile = -1;
    u.hsep = nullptr;
    u.z2 = nullptr;
    u.c_z2 = 0.f;
    u.wtaps = nullptr;
    u.nwtaps = 0;
    u.qb = nullptr;
    u.x_out = nullptr;
    return PNP_OK;
}

extern "C" pnp_status pnp_langevin_update(float* x, const float* r, const float* d, const float* h,
                                          int kh, int kw, int ny, int nx, int nchain, double sigma,
                                          double alpha, double eps, double lambda, double gamma,
                                          uint64_t seed, uint32_t t, int noise, float* mean,
                                          float* m2, int64_t n_kept, void* stream) {
    PNP_TRY(check_blur_args(x, h, kh, kw, ny, nx, nchain, r, "pnp_langevin_update"));
    if (n_kept > 0 && (!mean || !m2)) return fail(PNP_EINVAL, "moments requested without buffers");
    UpdateParams u;
    PNP_TRY(fill_update_params(u, x, r, d, h, kh, kw, ny, nx, nchain, sigma, alpha, eps, lambda,
                               gamma, seed, noise));
    u.t = t;
    u.mean = mean;
    u.m2 = m2;
    u.inv_n = n_kept > 0 ? (float)(1.0 / (double)n_kept) : 0.f;
    PNP_CUDA_TRY(launch_langevin_update(u, (cudaStream_t)stream));
    return PNP_OK;
}

extern "C" pnp_status pnp_inpaint_update(float* x, const float* y_obs, const float* d, int ny,
                                         int nx, int nchain, double sigma, double alpha,
                                         double eps, double lambda, double gamma, uint64_t seed,
                                         uint32_t t, int noise, float* mean, float* m2,
                                         int64_t n_kept, void* stream) {
    if (!x || !y_obs || ny < 1 || nx < 1 || nchain < 1)
        return fail(PNP_EINVAL, "pnp_inpaint_update: need x, y_obs and positive sizes");
    if (n_kept > 0 && (!mean || !m2)) return fail(PNP_EINVAL, "moments requested without buffers");
    UpdateParams u;
    PNP_TRY(fill_update_params(u, x, y_obs, d, nullptr, 1, 1, ny, nx, nchain, sigma, alpha, eps,
                               lambda, gamma, seed, noise));
    u.t = t;
    u.mean = mean;
    u.m2 = m2;
    u.inv_n = n_kept > 0 ? (float)(1.0 / (double)n_kept) : 0.f;
    PNP_CUDA_TRY(launch_update_mask(u, (cudaStream_t)stream));
    return PNP_OK;
}

extern "C" pnp_status pnp_finalize_moments(const float* mean, const float* m2, int64_t npix,
                                           int64_t n_kept, int want_var, double* mmse,
                                           double* out2, void* stream) {
    if (!mean || !m2 || !mmse || !out2 || npix < 1)
        return fail(PNP_EINVAL, "pnp_finalize_moments: bad arguments");
    PNP_CUDA_TRY(launch_finalize_moments(mean, m2, npix, n_kept, want_var, mmse, out2,
                                         (cudaStream_t)stream));
    return PNP_OK;
}

// ------------------------------------------------------------------ problem

extern "C" void pnp_destroy_problem(pnp_problem* p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (int k = 0; k < 2; ++k) {
        if (p->graph[k]) cudaGraphExecDestroy(p->graph[k]);
        if (p->graph_batch[k]) cudaGraphExecDestroy(p->graph_batch[k]);
    }
    // the state buffers are xb[0] and, for the one-pass gradient, the residual
    // plane r; x points at one of them
    for (void* q : {(void*)p->y, (void*)p->h, (void*)p->xb[0], (void*)p->r, (void*)p->d,
                    (void*)p->mean, (void*)p->m2, (void*)p->blocks, (void*)p->tiles,
                    (void*)p->dtiles, (void*)p->rects, p->scratch, (void*)p->st,
                    (void*)p->hsep, (void*)p->z1, (void*)p->z2, (void*)p->wt_fwd,
                    (void*)p->wt_adj, (void*)p->err, (void*)p->qb, (void*)p->qsep})
        dfree(q);
    pnp::spectral_free(p->sp);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

namespace pnp {

// Poisson: r = eta H x - z1 for the current state. The z-update of every
// iteration writes it for the next one (it has eta H x+ at hand), so an
// iteration launches no blur; this refresh runs only when the host changes x
// or z1 (creation, pnp_set_state, pnp_set_aux_state).
static pnp_status poisson_refresh_r(pnp_problem* p) {
    PNP_CUDA_TRY(launch_blur(p->x, p->z1, p->h, p->kh, p->kw, p->ny, p->nx, p->nchain, p->r,
                             p->stream, p->blur_tile, p->hsep, (float)p->eta, p->N));
    return PNP_OK;
}

pnp_status problem_pre(pnp_problem* p, cudaStream_t s) {
    if (p->inpaint) return PNP_OK;   // H = diag(mask): the update forms x - y itself
    if (p->fused) return PNP_OK;     // the update forms (H^T H) x - H^T y from x itself
    if (p->sp) {
        // P F(x) for every chain; the update's inverse row FFTs finish F^-1
        PNP_CUDA_TRY(spectral_pre(*p->sp, p->x, p->nchain, s));
        return PNP_OK;
    }
    if (p->poisson) {
        return PNP_OK;               // r = eta H x - z1 was written by the last z-update
    } else {
        PNP_CUDA_TRY(launch_blur(p->x, p->y, p->h, p->kh, p->kw, p->ny, p->nx, p->nchain, p->r, s,
                                 p->blur_tile, p->hsep, 1.0f, 0, p->wt_fwd, p->nwt));
    }
    return PNP_OK;
}

// The update of one iteration on the problem's buffers; the kernel reads the
// step counter from the device and its last block advances it.
pnp_status problem_update_params(const pnp_problem* p, UpdateParams& u) {
    const bool prior = p->D && p->alpha != 0.0;
    // Poisson: the H^T r coefficient eta / rho1 takes the place of 1 / sigma^2
    const double sig = p->poisson ? std::sqrt(p->rho1 / p->eta) : p->sigma;
    PNP_TRY(fill_update_params(u, p->x, p->inpaint ? p->y : p->r, prior ? p->d : nullptr, p->h,
                               p->kh, p->kw, p->ny,
                               p->nx, p->nchain, sig, p->alpha, p->eps, p->lambda, p->gamma,
                               p->seed, 1));
    u.t_dev = &p->st->t;
    u.burn_dev = &p->st->burn_in;
    u.arrive = &p->st->arrive;
    u.mean = p->mean;
    u.m2 = p->m2;
    u.d_residual = p->prec != PNP_FP32;   // the tensor-core denoisers hand over G = x - D(x)
    u.tile = p->update_tile;
    u.hsep = p->hsep;
    u.wtaps = p->wt_adj;
    u.nwtaps = p->nwt;
    if (p->fused) {
        // one pass over the current state with the taps of H^T H, x+ to the other buffer
        u.r = p->x;
        u.x_out = p->xb[p->par ^ 1];
        u.qb = p->qb;
        u.hsep = p->qsep;
        u.h = nullptr;
        u.kh = 2 * p->kh - 1;
        u.kw = 2 * p->kw - 1;
        u.os = 1;
        u.err = p->err;
    }
    if (p->sp) u.qb = p->qb;   // spectral gradient: g = Re(F^-1(P F x)) - H^T y
    if (p->poisson) {
        u.inv_s2 = (float)(p->eta / p->rho1);
        u.z2 = p->z2;
        u.c_z2 = (float)(p->gamma / p->rho2);
        u.arrive = nullptr;   // the z-update, the iteration's last kernel, advances t
    }
    return PNP_OK;
}

ZParams problem_z_params(const pnp_problem* p) {
    ZParams z;
    z.x = p->x;
    z.z1 = p->z1;
    z.z2 = p->z2;
    z.y = p->y;
    z.h = p->h;
    z.hsep = p->hsep;
    z.kh = p->kh;
    z.kw = p->kw;
    z.ny = p->ny;
    z.nx = p->nx;
    z.nchain = p->nchain;
    z.eta = (float)p->eta;
    z.a1 = (float)(p->kappa1 / p->rho1);
    z.a2 = (float)(p->kappa2 / p->rho2);
    z.s1 = (float)std::sqrt(2.0 * p->kappa1);
    z.s2 = (float)std::sqrt(2.0 * p->kappa2);
    z.kappa1 = (float)p->kappa1;
    z.noise = 1;
    z.key0 = (uint32_t)(p->seed & 0xffffffffu);
    z.key1 = (uint32_t)(p->seed >> 32);
    z.t = 0;
    z.t_dev = &p->st->t;
    z.arrive = &p->st->arrive;
    z.tile = p->update_tile;
    z.r_out = p->r;
    return z;
}

pnp_status problem_post(pnp_problem* p, cudaStream_t s) {
    UpdateParams u;
    PNP_TRY(problem_update_params(p, u));
    if (p->inpaint) PNP_CUDA_TRY(launch_update_mask(u, s));
    else if (p->sp) PNP_CUDA_TRY(spectral_update(*p->sp, u, s));
    else PNP_CUDA_TRY(launch_langevin_update(u, s));
    if (p->poisson) PNP_CUDA_TRY(launch_zupdate(problem_z_params(p), s));
    problem_flip(p);
    return PNP_OK;
}

}  // namespace pnp

static pnp_status enqueue_iteration(pnp_problem* p) {
    cudaStream_t s = p->stream;
    PNP_TRY(problem_pre(p, s));
    const bool prior = p->D && p->alpha != 0.0;
    if (prior) {
        const DenoiserDev& D = p->D->dev;
        if (p->halo == 0) {
            PNP_CUDA_TRY(run_denoise(D, p->prec, p->prec != PNP_FP32, p->x, p->ny, p->nx, p->nchain, nullptr, p->d,
                                     p->scratch, s, p->err));
        } else {
            PNP_CUDA_TRY(launch_gather_blocks(p->x, p->ny, p->nx, p->blocks, p->nblocks, p->halo,
                                              p->ty, p->tx, p->tiles, p->rects, s));
            PNP_CUDA_TRY(run_denoise(D, p->prec, p->prec != PNP_FP32, p->tiles, p->ty, p->tx, p->nblocks, p->rects,
                                     p->dtiles, p->scratch, s, p->err));
            PNP_CUDA_TRY(launch_scatter_blocks(p->dtiles, p->ny, p->nx, p->blocks, p->nblocks,
                                               p->halo, p->ty, p->tx, p->d, s));
        }
    }
    return problem_post(p, s);
}

// Rank-one split of the blur kernel: h = u v^T up to FP32 rounding
// (|h - u v^T|_F <= 1e-7 |h|_F; Gaussian and uniform kernels are rank one, a
// motion kernel is not). The top singular pair comes from power iteration in
// FP64. out = [u (kh) | v (kw) | u reversed | v reversed], the reversed pair
// being the taps of the flipped kernel used by the forward operator.
static bool separable_taps(const float* h, int kh, int kw, std::vector<float>& out) {
    if (kh < 2 || kw < 2) return false;
    std::vector<double> u(kh, 0.0), v(kw, 1.0 / std::sqrt((double)kw));
    double sig = 0.0, hn = 0.0;
    for (int i = 0; i < kh * kw; ++i) hn += (double)h[i] * h[i];
    if (!(hn > 0)) return false;
    for (int it = 0; it < 200; ++it) {
        double nu = 0.0;
        for (int a = 0; a < kh; ++a) {
            double s = 0.0;
            for (int b = 0; b < kw; ++b) s += (double)h[a * kw + b] * v[b];
            u[a] = s;
            nu += s * s;
        }
        nu = std::sqrt(nu);
        if (!(nu > 0)) return false;
        for (double& x : u) x /= nu;
        double nv = 0.0;
        for (int b = 0; b < kw; ++b) {
            double s = 0.0;
            for (int a = 0; a < kh; ++a) s += (double)h[a * kw + b] * u[a];
            v[b] = s;
            nv += s * s;
        }
        sig = std::sqrt(nv);
        if (!(sig > 0)) return false;
        for (double& x : v) x /= sig;
    }
    double res = 0.0, su = 0.0;
    for (int a = 0; a < kh; ++a)
        for (int b = 0; b < kw; ++b) {
            const double d = (double)h[a * kw + b] - sig * u[a] * v[b];
            res += d * d;
        }
    if (res > 1e-14 * hn) return false;
    for (double x : u) su += x;
    const double sgn = su < 0 ? -1.0 : 1.0, rs = std::sqrt(sig);
    out.assign(2 * (kh + kw), 0.f);
    for (int a = 0; a < kh; ++a) {
        out[a] = (float)(sgn * rs * u[a]);
        out[kh + kw + a] = (float)(sgn * rs * u[kh - 1 - a]);
    }
    for (int b = 0; b < kw; ++b) {
        out[kh + b] = (float)(sgn * rs * v[b]);
        out[2 * kh + kw + b] = (float)(sgn * rs * v[kw - 1 - b]);
    }
    return true;
}

extern "C" pnp_status pnp_create_problem(const pnp_problem_desc* dsc, pnp_problem** out) {
    if (!dsc || !out) return fail(PNP_EINVAL, "pnp_create_problem: NULL argument");
    *out = nullptr;
    pnp_problem_desc q = *dsc;
    const bool inpaint = q.mask != nullptr;
    static const float unit_tap = 1.0f;
    if (inpaint) {
        // H = diag(mask): h is not used; a 1 x 1 unit tap keeps the blur fields valid
        q.h = &unit_tap;
        q.kh = q.kw = 1;
        if (!(q.hnorm > 0)) q.hnorm = 1.0;
        if (q.noise_model != PNP_GAUSSIAN)
            return fail(PNP_EINVAL, "inpainting takes the Gaussian noise model");
    }
    if (q.ny < 1 || q.nx < 1 || !q.y || !q.h) return fail(PNP_EINVAL, "need ny, nx >= 1, y and h");
    PNP_TRY(check_blur_args(q.y, q.h, q.kh, q.kw, q.ny, q.nx, 1, q.y, "pnp_create_problem"));
    const bool poisson = q.noise_model == PNP_POISSON;
    if (q.noise_model != PNP_GAUSSIAN && !poisson) return fail(PNP_EINVAL, "unknown noise model");
    if (!poisson && (!(q.sigma > 0) || !std::isfinite(q.sigma)))
        return fail(PNP_EINVAL, "sigma must be > 0");
    if (poisson && is_wide(q.kh, q.kw))
        return fail(PNP_ENOTSUP, "Poisson model: blur kernels up to 31 x 31");
    if (poisson) {
        if (!(q.eta > 0) || !(q.rho1 > 0) || !(q.rho2 > 0) || !std::isfinite(q.eta) ||
            !std::isfinite(q.rho1) || !std::isfinite(q.rho2))
            return fail(PNP_EINVAL, "Poisson model: need eta, rho1, rho2 > 0");
        if ((q.kappa1 > 0 && !(q.kappa1 < q.rho1)) || (q.kappa2 > 0 && !(q.kappa2 < q.rho2)))
            return fail(PNP_EINVAL, "Poisson model: need kappa_i in (0, rho_i)");
    }
    if (q.nchain < 1) return fail(PNP_EINVAL, "nchain must be >= 1");
    if (q.blocks_y < 1 || q.blocks_x < 1 || q.blocks_y > q.ny || q.blocks_x > q.nx)
        return fail(PNP_EINVAL, "blocks must be in [1, image size]");
    if (q.halo < 0) return fail(PNP_EINVAL, "halo must be >= 0");
    if (q.D && q.halo > 0 && q.halo < q.D->dev.K)
        return fail(PNP_EINVAL, "halo must cover the receptive field (halo >= K)");
    if (q.precision != PNP_FP32 && q.precision != PNP_BF16 && q.precision != PNP_FP8)
        return fail(PNP_ENOTSUP, "unknown precision");
    if (q.D && q.D->dev.ddfb && q.precision != PNP_FP32)
        return fail(PNP_ENOTSUP, "the DDFB denoiser runs in FP32");
    if (q.D && q.D->dev.ddfb && q.halo > 0)
        return fail(PNP_EINVAL, "the DDFB denoiser uses the direct layout (halo = 0)");
    if (q.D && q.precision != PNP_FP32 && q.D->dev.F != 64)
        return fail(PNP_EINVAL, "BF16/FP8 denoiser needs F = 64");
    const int64_t N = (int64_t)q.ny * q.nx;
    for (int64_t i = 0; i < N; ++i) {
        if (inpaint && q.mask[i] != 0.f && q.mask[i] != 1.f)
            return fail(PNP_EINVAL, "mask entries must be 0 or 1");
        if (inpaint && q.mask[i] == 0.f) continue;   // y is not read at missing pixels
        if (!std::isfinite(q.y[i])) return fail(PNP_EINVAL, "y contains NaN or Inf");
        if (poisson && q.y[i] < 0) return fail(PNP_EINVAL, "Poisson counts y must be >= 0");
    }
    double hsum = 0.0;
    for (int i = 0; i < q.kh * q.kw; ++i) {
        if (!std::isfinite(q.h[i])) return fail(PNP_EINVAL, "h contains NaN or Inf");
        hsum += std::fabs(q.h[i]);
    }
    pnp_problem* p = new pnp_problem();
    cudaGetDevice(&p->device);
    p->ny = q.ny;
    p->nx = q.nx;
    p->N = N;
    p->nchain = q.nchain;
    p->kh = q.kh;
    p->kw = q.kw;
    p->sigma = poisson ? 0.0 : q.sigma;
    p->poisson = poisson;
    p->inpaint = inpaint;
    if (poisson) {
        p->eta = q.eta;
        p->rho1 = q.rho1;
        p->rho2 = q.rho2;
        p->kappa1 = q.kappa1 > 0 ? q.kappa1 : 0.99 * q.rho1;
        p->kappa2 = q.kappa2 > 0 ? q.kappa2 : 0.99 * q.rho2;
    }
    p->alpha = q.alpha < 0 ? 1.0 : q.alpha;
    // the paper's Poisson setting takes eps = 0.05; the Gaussian one eps = sigma
    p->eps = q.eps > 0 ? q.eps : (poisson ? 0.05 : q.sigma);
    p->hnorm = q.hnorm > 0 ? q.hnorm : hsum;
    p->seed = q.seed;
    p->burn_in = q.burn_in;
    p->prec = q.precision;
    p->D = q.D;
    p->by = q.blocks_y;
    p->bx = q.blocks_x;
    p->halo = q.halo;
    const double lip = q.D ? q.D->dev.lip : 0.0;
    const double alpha_eff = q.D ? p->alpha : 0.0;
    double lam = q.lambda, gam = q.gamma;
    if (!(lam > 0) || !(gam > 0)) {
        double l2, g2, k1, k2;
        pnp_status st = poisson
            ? pnp_stepsizes_poisson(p->hnorm, p->eta, p->rho1, p->rho2, alpha_eff, p->eps, lip,
                                    q.step_c > 0 ? q.step_c : 0.99, &l2, &g2, &k1, &k2)
            : pnp_stepsizes(p->hnorm, p->sigma, alpha_eff, p->eps, lip,
                            q.step_c > 0 ? q.step_c : 0.99, &l2, &g2);
        if (st != PNP_OK) {
            delete p;
            return st;
        }
        if (!(lam > 0)) lam = l2;
        if (!(gam > 0)) gam = g2;
    }
    p->lambda = lam;
    p->gamma = gam;
    // Eq. 12 must hold for the parameters actually used: Gaussian L = ||H||^2 /
    // sigma^2 and H_2 = 0; Poisson f1 = 0 and ||H_2||^2 = ||eta H||^2 / rho1 + 1 / rho2
    {
        const double L = poisson ? 0.0 : p->hnorm * p->hnorm / (p->sigma * p->sigma);
        const double h2 = poisson ? p->eta * p->hnorm * p->eta * p->hnorm / p->rho1 + 1.0 / p->rho2
                                  : 0.0;
        const double prior = alpha_eff * lip / (p->eps * p->eps);
        if (!(3.0 * gam * (L + h2 + 1.0 / lam + prior) < 1.0) ||
            !(2.0 * (L + h2) + prior <= 0.5 / lam * (1 + 1e-12))) {
            delete p;
            return fail(PNP_EINVAL, "step sizes violate the conditions of Eq. 10");
        }
    }
    pnp_status st = PNP_OK;
#define ALLOC(ptr, n)                               \
    if ((st = dalloc(&(ptr), (n))) != PNP_OK) {     \
        pnp_destroy_problem(p);                     \
        return st;                                  \
    }
    const size_t NC = (size_t)N * q.nchain;
    ALLOC(p->y, N);
    ALLOC(p->h, (size_t)q.kh * q.kw);
    ALLOC(p->x, NC);
    p->xb[0] = p->xb[1] = p->x;
    ALLOC(p->r, NC);
    ALLOC(p->d, NC);
    ALLOC(p->mean, NC);
    ALLOC(p->m2, NC);
    ALLOC(p->st, 1);
    ALLOC(p->err, 1);
    cudaMemset(p->err, 0, sizeof(int));
    if (poisson) {
        ALLOC(p->z1, NC);
        ALLOC(p->z2, NC);
    }
    if (q.stream) {
        p->stream = (cudaStream_t)q.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            pnp_destroy_problem(p);
            return cuda_fail(e, "cudaStreamCreate");
        }
        p->own_stream = true;
    }
    if (q.D) {
        const DenoiserDev& D = q.D->dev;
        if (q.halo == 0) {
            p->scratch_bytes = denoise_scratch_bytes(D, q.precision, q.ny, q.nx, q.nchain);
        } else {
            int mh, mw;
            std::vector<BlockDesc> bl = make_blocks(q.ny, q.nx, q.blocks_y, q.blocks_x, q.nchain, &mh, &mw);
            p->nblocks = (int)bl.size();
            p->ty = mh + 2 * q.halo;
            p->tx = mw + 2 * q.halo;
            const size_t tf = (size_t)p->nblocks * p->ty * p->tx;
            ALLOC(p->blocks, (size_t)p->nblocks);
            ALLOC(p->tiles, tf);
            ALLOC(p->dtiles, tf);
            ALLOC(p->rects, (size_t)p->nblocks);
            cudaMemcpy(p->blocks, bl.data(), bl.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice);
            p->scratch_bytes = denoise_scratch_bytes(D, q.precision, p->ty, p->tx, p->nblocks);
        }
        uint8_t* sc = nullptr;
        ALLOC(sc, p->scratch_bytes);
        p->scratch = sc;
        cudaMemset(p->scratch, 0, p->scratch_bytes);
    }
#undef ALLOC
    if (inpaint) {
        // missing pixels hold NaN: the masked update reads the mask from y
        std::vector<float> yo(q.y, q.y + N);
        for (int64_t i = 0; i < N; ++i)
            if (q.mask[i] == 0.f) yo[i] = std::numeric_limits<float>::quiet_NaN();
        cudaMemcpy(p->y, yo.data(), N * 4, cudaMemcpyHostToDevice);
    } else {
        cudaMemcpy(p->y, q.y, N * 4, cudaMemcpyHostToDevice);
    }
    cudaMemcpy(p->h, q.h, (size_t)q.kh * q.kw * 4, cudaMemcpyHostToDevice);
    if (is_wide(q.kh, q.kw)) {
        // large kernel: nonzero taps as window offsets, forward and adjoint
        const std::vector<WTap> f = wide_taps(q.h, q.kh, q.kw, false);
        const std::vector<WTap> a = wide_taps(q.h, q.kh, q.kw, true);
        p->nwt = (int)f.size();
        const size_t nt = std::max<size_t>(f.size(), 1);
        if ((st = dalloc(&p->wt_fwd, nt)) != PNP_OK || (st = dalloc(&p->wt_adj, nt)) != PNP_OK) {
            pnp_destroy_problem(p);
            return st;
        }
        cudaMemcpy(p->wt_fwd, f.data(), f.size() * sizeof(WTap), cudaMemcpyHostToDevice);
        cudaMemcpy(p->wt_adj, a.data(), a.size() * sizeof(WTap), cudaMemcpyHostToDevice);
    }
    {
        std::vector<float> sep;
        if (!is_wide(q.kh, q.kw) && separable_taps(q.h, q.kh, q.kw, sep)) {
            if ((st = dalloc(&p->hsep, sep.size())) != PNP_OK) {
                pnp_destroy_problem(p);
                return st;
            }
            cudaMemcpy(p->hsep, sep.data(), sep.size() * 4, cudaMemcpyHostToDevice);
            // One-pass gradient for a separable blur under Gaussian noise:
            // H^T (H x - y) = (H^T H) x - H^T y. H^T H is the correlation with
            // the autocorrelation q of h (symmetric, 2 L - 1 taps per axis),
            // separable as qu qv^T when h = u v^T.
            if (!poisson && !inpaint && 2 * q.kh - 1 <= STENCIL_MAXK && 2 * q.kw - 1 <= STENCIL_MAXK) {
                const int qh = 2 * q.kh - 1, qw = 2 * q.kw - 1;
                auto autocorr = [](const float* v, int L, std::vector<double>& out) {
                    out.assign(2 * L - 1, 0.0);
                    for (int k = -(L - 1); k <= L - 1; ++k)
                        for (int a = 0; a < L; ++a)
                            if (a + k >= 0 && a + k < L) out[k + L - 1] += (double)v[a + k] * v[a];
                };
                std::vector<double> qu, qv;
                autocorr(sep.data(), q.kh, qu);
                autocorr(sep.data() + q.kh, q.kw, qv);
                std::vector<float> qs(2 * (qh + qw));
                for (int a = 0; a < qh; ++a) {
                    qs[a] = (float)qu[a];
                    qs[qh + qw + a] = (float)qu[qh - 1 - a];
                }
                for (int b = 0; b < qw; ++b) {
                    qs[qh + b] = (float)qv[b];
                    qs[2 * qh + qw + b] = (float)qv[qw - 1 - b];
                }
                if ((st = dalloc(&p->qsep, qs.size())) != PNP_OK ||
                    (st = dalloc(&p->qb, (size_t)N)) != PNP_OK) {
                    pnp_destroy_problem(p);
                    return st;
                }
                cudaMemcpy(p->qsep, qs.data(), qs.size() * 4, cudaMemcpyHostToDevice);
                // H^T y, formed once for the whole chain
                cudaError_t e = launch_blur_adjoint(p->y, p->h, q.kh, q.kw, q.ny, q.nx, 1, 1.0f,
                                                    p->qb, p->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
                if (e != cudaSuccess) {
                    pnp_destroy_problem(p);
                    return cuda_fail(e, "pnp_create_problem: H^T y");
                }
                p->fused = true;
                p->xb[1] = p->r;   // the residual plane is not needed: second state buffer
            }
        }
        // Spectral gradient for wide blurs under Gaussian noise on power-of-two
        // images: g = F^-1(|H^|^2 F(x)) - H^T y; H^T y by the direct adjoint
        if (g_spectral.load() && !poisson && !inpaint && is_wide(q.kh, q.kw) &&
            spectral_eligible(q.ny, q.nx, q.kh, q.kw)) {
            if ((st = dalloc(&p->qb, (size_t)N)) != PNP_OK) {
                pnp_destroy_problem(p);
                return st;
            }
            cudaError_t e = launch_blur_adjoint(p->y, p->h, q.kh, q.kw, q.ny, q.nx, 1, 1.0f, p->qb,
                                                p->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
            if (e == cudaSuccess)
                e = spectral_setup(p->h, q.kh, q.kw, q.ny, q.nx, p->nchain, p->stream, &p->sp);
            if (e != cudaSuccess && e != cudaErrorNotSupported) {
                pnp_destroy_problem(p);
                return cuda_fail(e, "pnp_create_problem: spectral gradient");
            }
        }
    }
    {
        // stencil tile shapes, timed on this problem's buffers before they are initialised
        cudaMemset(p->x, 0, NC * 4);
        cudaMemset(p->r, 0, NC * 4);
        cudaMemset(p->d, 0, NC * 4);
        cudaMemset(p->mean, 0, NC * 4);
        cudaMemset(p->m2, 0, NC * 4);
        UpdateParams u;
        pnp_status us = problem_update_params(p, u);
        if (us == PNP_OK && !inpaint && !is_wide(q.kh, q.kw)) {
            u.t_dev = nullptr;
            u.burn_dev = nullptr;
            u.arrive = nullptr;
            u.inv_n = 1.0f;   // time the sampling form (Welford traffic included)
            cudaError_t e = p->fused
                ? stencil_autotune(p->x, p->y, p->h, p->qsep, 2 * p->kh - 1, 2 * p->kw - 1, p->ny,
                                   p->nx, p->nchain, p->r, u, p->stream, &p->blur_tile,
                                   &p->update_tile)
                : stencil_autotune(p->x, p->y, p->h, p->hsep, p->kh, p->kw, p->ny,
                                   p->nx, p->nchain, p->r, u, p->stream,
                                   &p->blur_tile, &p->update_tile);
            if (e != cudaSuccess) us = cuda_fail(e, "stencil autotune");
        }
        if (us != PNP_OK) {
            pnp_destroy_problem(p);
            return us;
        }
    }
    if (q.x0) cudaMemcpy(p->x, q.x0, NC * 4, cudaMemcpyHostToDevice);
    else cudaMemset(p->x, 0, NC * 4);
    cudaMemset(p->mean, 0, NC * 4);
    cudaMemset(p->m2, 0, NC * 4);
    cudaMemset(p->r, 0, NC * 4);
    cudaMemset(p->d, 0, NC * 4);
    if (poisson) {
        // auxiliary variables start at zero (Sec. IV-B)
        cudaMemset(p->z1, 0, NC * 4);
        cudaMemset(p->z2, 0, NC * 4);
    }
    StepState s0{0u, (int32_t)q.burn_in, 0u};
    cudaMemcpy(p->st, &s0, sizeof(s0), cudaMemcpyHostToDevice);
    if (q.D && q.precision == PNP_FP8 && !q.D->dev.fp8_calibrated) {
        // static activation scales from an image of the signal's range: the
        // observation y (x = y), the counts over eta (Poisson), or the
        // initial state (inpainting: y is zero at 70 % of the pixels)
        const float* src = p->y;
        if (poisson || (inpaint && q.x0)) {
            std::vector<float> c(N);
            for (int64_t i = 0; i < N; ++i) c[i] = poisson ? (float)(q.y[i] / q.eta) : q.x0[i];
            cudaMemcpy(p->r, c.data(), N * 4, cudaMemcpyHostToDevice);
            src = p->r;
        }
        pnp_status cs = pnp_denoiser_calibrate_fp8(const_cast<pnp_denoiser*>(q.D), src, q.ny, q.nx, 1,
                                                   p->stream);
        if (src != p->y) cudaMemsetAsync(p->r, 0, NC * 4, p->stream);
        if (cs != PNP_OK) {
            pnp_destroy_problem(p);
            return cs;
        }
    }
    if (poisson) {
        pnp_status rs = poisson_refresh_r(p);
        if (rs != PNP_OK) {
            pnp_destroy_problem(p);
            return rs;
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        pnp_destroy_problem(p);
        return cuda_fail(e, "pnp_create_problem");
    }
    *out = p;
    return PNP_OK;
}

extern "C" pnp_status pnp_problem_params(const pnp_problem* p, double* lambda, double* gamma,
                                         double* alpha, double* eps) {
    if (!p) return fail(PNP_EINVAL, "problem is NULL");
    if (lambda) *lambda = p->lambda;
    if (gamma) *gamma = p->gamma;
    if (alpha) *alpha = p->alpha;
    if (eps) *eps = p->eps;
    return PNP_OK;
}

// Captures `iters` iterations of the problem, starting from its current state
// buffer, into one executable graph. Capturing executes nothing, so the
// host-side state buffer is restored afterwards.
static pnp_status capture_graph(pnp_problem* p, int iters, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    const int par0 = p->par;
    PNP_CUDA_TRY(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    pnp_status st = PNP_OK;
    for (int i = 0; i < iters && st == PNP_OK; ++i) st = enqueue_iteration(p);
    cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    p->par = par0;
    p->x = p->xb[par0];
    if (st != PNP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    return PNP_OK;
}

static bool g_use_graph = true;

extern "C" pnp_status pnp_kernel_timer(int enable) {
    PNP_CUDA_TRY(cudaDeviceSynchronize());
    for (auto& t : g_timers) t.used = 0;
    g_timing = enable != 0;
    return PNP_OK;
}

extern "C" pnp_status pnp_kernel_timer_read(const char* name, double* total_ms, int64_t* launches) {
    if (!name || !total_ms || !launches) return fail(PNP_EINVAL, "pnp_kernel_timer_read: NULL");
    for (int i = 0; i < T_COUNT; ++i) {
        if (strcmp(name, g_timer_names[i]) != 0) continue;
        PNP_CUDA_TRY(cudaDeviceSynchronize());
        double tot = 0.0;
        for (size_t k = 0; k < g_timers[i].used; ++k) {
            float ms = 0.f;
            PNP_CUDA_TRY(cudaEventElapsedTime(&ms, g_timers[i].begin[k], g_timers[i].end[k]));
            tot += ms;
        }
        *total_ms = tot;
        *launches = (int64_t)g_timers[i].used;
        return PNP_OK;
    }
    return fail(PNP_EINVAL, std::string("unknown kernel timer ") + name);
}

extern "C" int64_t pnp_launch_count(void) { return g_launches.load(); }

extern "C" pnp_status pnp_set_graph_mode(int enable) {
    g_use_graph = enable != 0;
    return PNP_OK;
}

extern "C" pnp_status pnp_set_pdl(int enable) {
    g_pdl = enable != 0;
    return PNP_OK;
}

extern "C" pnp_status pnp_set_spectral(int enable) {
    g_spectral = enable != 0;
    return PNP_OK;
}

extern "C" int pnp_stencil_tile_count(void) { return stencil_tile_count(); }

extern "C" pnp_status pnp_set_stencil_tile(int tile) {
    if (!set_forced_stencil_tile(tile))
        return fail(PNP_EINVAL, "pnp_set_stencil_tile: tile must be -1 or in [0, count)");
    return PNP_OK;
}

extern "C" pnp_status pnp_problem_stencil_tiles(const pnp_problem* p, int* blur_tile,
                                                int* update_tile, int* separable) {
    if (!p) return fail(PNP_EINVAL, "problem is NULL");
    if (blur_tile) *blur_tile = p->blur_tile;
    if (update_tile) *update_tile = p->update_tile;
    if (separable) *separable = p->hsep != nullptr;
    return PNP_OK;
}

extern "C" pnp_status pnp_step(pnp_problem* p, int n_iters) {
    if (!p || n_iters < 0) return fail(PNP_EINVAL, "pnp_step: bad arguments");
    if (n_iters == 0) return PNP_OK;
    if (g_use_graph && !g_timing) {
        if (!p->eager_done) {
            // one eager iteration first performs the lazy per-kernel setup
            PNP_TRY(enqueue_iteration(p));
            p->eager_done = true;
            p->t += 1;
            --n_iters;
            if (n_iters == 0) return PNP_OK;
        }
        // graphs per start parity of the state buffers (one pair when the
        // state is updated in place); a kGraphBatch-iteration graph ends on
        // the parity it started from
        int left = n_iters;
        while (left > 0) {
            const int gi = p->xb[0] == p->xb[1] ? 0 : p->par;
            if (left >= kGraphBatch) {
                if (!p->graph_batch[gi]) PNP_TRY(capture_graph(p, kGraphBatch, &p->graph_batch[gi]));
                PNP_CUDA_TRY(cudaGraphLaunch(p->graph_batch[gi], p->stream));
                left -= kGraphBatch;
                if (kGraphBatch % 2) problem_flip(p);
            } else {
                if (!p->graph[gi]) PNP_TRY(capture_graph(p, 1, &p->graph[gi]));
                PNP_CUDA_TRY(cudaGraphLaunch(p->graph[gi], p->stream));
                left -= 1;
                problem_flip(p);
            }
        }
    } else {
        for (int i = 0; i < n_iters; ++i) PNP_TRY(enqueue_iteration(p));
    }
    p->t += n_iters;
    return PNP_OK;
}

extern "C" pnp_status pnp_prepare_graphs(pnp_problem* p) {
    if (!p) return fail(PNP_EINVAL, "problem is NULL");
    if (!g_use_graph || g_timing) return PNP_OK;
    if (!p->eager_done)
        return fail(PNP_ESTATE, "pnp_prepare_graphs: step the problem once first (its first "
                                "iteration runs eagerly and performs the lazy kernel setup)");
    const int par0 = p->par;
    const int npar = p->xb[0] == p->xb[1] ? 1 : 2;
    pnp_status st = PNP_OK;
    for (int k = 0; k < npar && st == PNP_OK; ++k) {
        p->par = k;
        p->x = p->xb[k];
        if (!p->graph[k]) st = capture_graph(p, 1, &p->graph[k]);
        if (st == PNP_OK && !p->graph_batch[k]) st = capture_graph(p, kGraphBatch, &p->graph_batch[k]);
    }
    p->par = par0;
    p->x = p->xb[par0];
    return st;
}

extern "C" pnp_status pnp_sync(pnp_problem* p) {
    if (!p) return fail(PNP_EINVAL, "problem is NULL");
    PNP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return take_timeout(p->err, p->stream, "pnp_sync");
}

extern "C" pnp_status pnp_run_chain(pnp_problem* p, int T, int burn_in) {
    if (!p || T < 0 || burn_in < 0) return fail(PNP_EINVAL, "pnp_run_chain: bad arguments");
    if (burn_in != p->burn_in) {
        p->burn_in = burn_in;
        PNP_CUDA_TRY(cudaMemcpyAsync(&p->st->burn_in, &burn_in, 4, cudaMemcpyHostToDevice, p->stream));
        PNP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    }
    PNP_TRY(pnp_step(p, T));
    return pnp_sync(p);
}

extern "C" pnp_status pnp_get_moments(pnp_problem* p, int chain, double* mmse, double* std_or_var,
                                      int64_t* n_kept, int want_var) {
    if (!p || !mmse || !std_or_var || chain < 0 || chain >= p->nchain)
        return fail(PNP_EINVAL, "pnp_get_moments: bad arguments");
    PNP_TRY(take_timeout(p->err, p->stream, "pnp_get_moments"));
    const int64_t n = std::max<int64_t>(0, p->t - p->burn_in);
    double* dm = nullptr;
    PNP_TRY(dalloc(&dm, (size_t)2 * p->N));
    PNP_CUDA_TRY(launch_finalize_moments(p->mean + chain * p->N, p->m2 + chain * p->N, p->N, n,
                                         want_var, dm, dm + p->N, p->stream));
    cudaError_t e = cudaMemcpyAsync(mmse, dm, p->N * 8, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(std_or_var, dm + p->N, p->N * 8, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cudaFree(dm);
    if (e != cudaSuccess) return cuda_fail(e, "pnp_get_moments");
    if (n_kept) *n_kept = n;
    return PNP_OK;
}

extern "C" pnp_status pnp_get_state(pnp_problem* p, float* x, int64_t* t) {
    if (!p) return fail(PNP_EINVAL, "problem is NULL");
    PNP_TRY(take_timeout(p->err, p->stream, "pnp_get_state"));
    if (x) {
        PNP_CUDA_TRY(cudaMemcpyAsync(x, p->x, (size_t)p->N * p->nchain * 4, cudaMemcpyDeviceToHost, p->stream));
    }
    PNP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    if (t) *t = p->t;
    return PNP_OK;
}

extern "C" pnp_status pnp_set_state(pnp_problem* p, const float* x, int64_t t) {
    if (!p || t < 0 || t > 0xffffffffLL) return fail(PNP_EINVAL, "pnp_set_state: bad arguments");
    if (x) {
        PNP_CUDA_TRY(cudaMemcpyAsync(p->x, x, (size_t)p->N * p->nchain * 4, cudaMemcpyHostToDevice, p->stream));
    }
    StepState s0{(uint32_t)t, (int32_t)p->burn_in, 0u};
    PNP_CUDA_TRY(cudaMemcpyAsync(p->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, p->stream));
    if (p->poisson && x) PNP_TRY(poisson_refresh_r(p));
    PNP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    p->t = t;
    return PNP_OK;
}

extern "C" pnp_status pnp_get_aux_state(pnp_problem* p, float* z1, float* z2) {
    if (!p || !p->poisson) return fail(PNP_EINVAL, "pnp_get_aux_state: not a Poisson problem");
    const size_t bytes = (size_t)p->N * p->nchain * 4;
    if (z1) PNP_CUDA_TRY(cudaMemcpyAsync(z1, p->z1, bytes, cudaMemcpyDeviceToHost, p->stream));
    if (z2) PNP_CUDA_TRY(cudaMemcpyAsync(z2, p->z2, bytes, cudaMemcpyDeviceToHost, p->stream));
    PNP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return PNP_OK;
}

extern "C" pnp_status pnp_set_aux_state(pnp_problem* p, const float* z1, const float* z2) {
    if (!p || !p->poisson) return fail(PNP_EINVAL, "pnp_set_aux_state: not a Poisson problem");
    const size_t bytes = (size_t)p->N * p->nchain * 4;
    if (z1) PNP_CUDA_TRY(cudaMemcpyAsync(p->z1, z1, bytes, cudaMemcpyHostToDevice, p->stream));
    if (z2) PNP_CUDA_TRY(cudaMemcpyAsync(p->z2, z2, bytes, cudaMemcpyHostToDevice, p->stream));
    if (z1) PNP_TRY(poisson_refresh_r(p));
    PNP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return PNP_OK;
}

extern "C" float* pnp_problem_x_device(pnp_problem* p) { return p ? p->x : nullptr; }
