/*
 * FP64 CPU oracle for the PnP-ULA Gaussian-deconvolution sampler.
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, plainly written
 * reference that the CUDA path is checked against. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never calls it and shares no code with it.
 *
 * Every routine follows the paper's definitions directly, with no blocking,
 * fusion or reordering beyond what the definition states:
 *   - circular blur H and its adjoint H^T           (Sec. III-A2, Eq. 12 likelihood)
 *   - multichannel "half-padding" 3x3 convolution    (Sec. II-B, Eqs. 5-6)
 *   - DnCNN-form denoiser D = Id - G, G = T_K o ... o T_1 (Sec. II-B, Example 1)
 *   - block-wise denoiser with a halo (Defs. 1-2, Sec. II-B2, receptive-field variant)
 *   - Philox4x32-10 (Salmon et al., SC'11) + Box-Muller normals
 *   - one PnP-ULA transition (Eq. 8 / Algorithm 1, x-update), f2 = 0
 *   - step sizes (Eq. 10 conditions, Sec. III-B Gaussian-noise setting)
 *   - online (Welford) and two-pass moments (Sec. III-C, footnote on variance)
 *
 * Parity pins live in tests/test_oracle_*.py. Status of each function:
 *   ora_philox4x32_10      pinned (library Philox, statistics)
 *   ora_normals            pinned (moments, KS, Box-Muller identity)
 *   ora_blur / ora_blur_adj pinned (DFT convolution theorem, adjoint identity)
 *   ora_conv_layer         pinned (library conv2d)
 *   ora_denoise            pinned (layer composition vs library, Id - G form)
 *   ora_denoise_blockwise  pinned (equals whole image iff halo >= K)
 *   ora_langevin_step      pinned (closed-form Gaussian recursion and stationary
 *                          law; projection and linear-prior fixed points)
 *   ora_langevin_step_window pinned (equals ora_langevin_step bitwise on every
 *                          window of small images: corners, edges, interior)
 *   ora_run_chain moments  pinned (two-pass vs Welford, stored samples)
 *   ora_stepsizes          pinned (Eq. 10 inequalities)
 *   mask operator (inpainting) pinned (per-pixel closed form and stationary law,
 *                          masked linear-prior fixed point)
 *   ora_kl_prox, ora_normals_stream, ora_poisson_stepsizes, ora_poisson_step
 *                          pinned (scalar minimisation, stream statistics, Eq. 12,
 *                          augmented-objective fixed point)
 *   ora_ddfb_W / ora_ddfb_Wt pinned (library conv2d / conv_transpose2d)
 *   ora_ddfb_denoise       pinned (linear regime vs dense library operators;
 *                          identity analysis operator -> clip(soft(v, ht), 0, 1))
 */
#ifndef PNP_ORACLE_H
#define PNP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* DnCNN-form network: K layers of ks x ks cross-correlations, layer k maps
 * cin[k] -> cout[k] channels, weights OIHW concatenated over layers, biases
 * concatenated. ReLU after every layer but the last. */
typedef struct {
    int K;
    const int* cin;
    const int* cout;
    int ks;
    const double* w;
    const double* b;
} ora_net;

typedef struct {
    int ny, nx;              /* image size (one channel)                      */
    const double* y;         /* observation [ny*nx]                           */
    const double* h;         /* blur kernel [kh*kw], anchored at (kh/2, kw/2) */
    int kh, kw;
    double sigma;            /* noise std: f1(Hx) = ||y - Hx||^2 / (2 sigma^2) */
    double alpha, eps;       /* prior weight and denoiser noise level         */
    double lambda;           /* Moreau-Yosida parameter of iota_C; <= 0: term off */
    double gamma;            /* step size                                     */
    uint64_t seed;           /* Philox key                                    */
    const ora_net* net;      /* NULL: no denoiser term                        */
    int noise;               /* 0: xi := 0 (deterministic recursion)          */
    const struct ora_ddfb_s* ddfb;   /* DDFB denoiser (used when net is NULL)  */
    const double* mask;      /* NULL: H is the blur h; else H = diag(mask),
                                mask[n] in {0, 1} (inpainting, Sec. IV-A)     */
} ora_problem;

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void ora_normals(uint64_t seed, uint32_t t, uint32_t chain, int64_t n, double* xi);

void ora_blur(const double* x, int ny, int nx, const double* h, int kh, int kw, double* out);
void ora_blur_adj(const double* r, int ny, int nx, const double* h, int kh, int kw, double* out);

void ora_conv_layer(const double* in, int cin, int ny, int nx, const double* w,
                    const double* b, int cout, int ks, int relu, double* out);
void ora_denoise(const double* v, int ny, int nx, const ora_net* net, double* out);
int  ora_denoise_blockwise(const double* v, int ny, int nx, const ora_net* net,
                           int by, int bx, int halo, double* out);

void ora_stepsizes(double hnorm, double sigma, double alpha, double eps, double lip_eps,
                   double c, double* lambda, double* gamma);

void ora_langevin_step(const ora_problem* p, const double* x, uint32_t t, uint32_t chain,
                       double* xnew);
/* ora_langevin_step at the output pixels of the window [i0, i0+wy) x
 * [j0, j0+wx) only (whole-image x in, out [wy][wx]); for images too large to
 * step whole. Equal to the corresponding part of ora_langevin_step. Returns
 * 0, or -1 for a window outside the image or a DDFB denoiser. */
int ora_langevin_step_window(const ora_problem* p, const double* x, uint32_t t, uint32_t chain,
                             int i0, int j0, int wy, int wx, double* out);
/* Runs iterations t = t0 .. t0+T-1 from x (updated in place). Samples
 * x^(t+1) with t+1 > burn_in enter the FP64 Welford moments (mean, m2, *n).
 * samples (optional) receives every kept sample, [n_kept][ny*nx]. */
void ora_run_chain(const ora_problem* p, double* x, int t0, int T, int burn_in,
                   uint32_t chain, double* mean, double* m2, int64_t* n_kept,
                   double* samples);
void ora_moments_two_pass(const double* samples, int64_t n, int64_t npix,
                          double* mean, double* var);

/* ---------------------------------------------------------------------------
 * Deconvolution under Poisson noise (Sec. IV-A, Poisson case), sampled with
 * the AXDA-split PnP-ULA / PSGLA scheme (Eqs. 13-14, Algorithm 1):
 *   y ~ Poisson(eta H xbar),  f1 = 0,
 *   f2(H2 x) = KL(y || eta H x) + iota_{R+}(x),  H2 x = (eta H x, x),
 *   z = (z1, z2) coupled to (eta H x, x) with rho1, rho2,
 *   KL(y || u) = sum_n u_n - y_n + y_n log(y_n / u_n).
 * ------------------------------------------------------------------------- */
typedef struct {
    int ny, nx;
    const double* y;         /* photon counts [ny*nx]                         */
    const double* h;         /* blur kernel [kh*kw], anchored at (kh/2, kw/2) */
    int kh, kw;
    double eta;              /* y ~ Poisson(eta H x)                          */
    double rho1, rho2;       /* AXDA coupling of z1 ~ eta H x and z2 ~ x      */
    double kappa1, kappa2;   /* PSGLA step sizes of z1, z2                    */
    double alpha, eps;       /* prior weight and denoiser noise level         */
    double lambda;           /* Moreau-Yosida parameter of iota_[0,1]; <= 0: off */
    double gamma;            /* x step size                                   */
    uint64_t seed;           /* Philox key                                    */
    const ora_net* net;      /* NULL: no denoiser term                        */
    int noise;               /* 0: xi, zeta := 0                              */
} ora_poisson;

/* Normals of Philox stream `stream` (counter word 3): stream 0 drives xi,
 * streams 1 and 2 drive zeta_1 and zeta_2; ora_normals is stream 0. */
void ora_normals_stream(uint64_t seed, uint32_t t, uint32_t chain, uint32_t stream, int64_t n,
                        double* xi);
/* prox of kappa KL(y || .) at v, one pixel: the positive root of
 * u^2 + (kappa - v) u - kappa y = 0. */
double ora_kl_prox(double v, double y, double kappa);
/* Step sizes of the Poisson setting (Sec. IV-B (ii)), c = 0.99 in the paper:
 *   lambda = 0.99 / (4 ||eta H||^2 / rho1 + 4 / rho2 + 2 alpha L_eps / eps^2)
 *   gamma  = c / (3 (alpha L_eps / eps^2 + ||eta H||^2 / rho1 + 1 / rho2 + 1 / lambda))
 *   kappa_i = 0.99 rho_i */
void ora_poisson_stepsizes(double hnorm, double eta, double rho1, double rho2, double alpha,
                           double eps, double lip_eps, double c, double* lambda, double* gamma,
                           double* kappa1, double* kappa2);
/* One transition t -> t + 1: x by Eq. 13, then z by Eq. 14 from the new x. */
void ora_poisson_step(const ora_poisson* p, const double* x, const double* z1, const double* z2,
                      uint32_t t, uint32_t chain, double* xnew, double* z1new, double* z2new);

/* DDFB denoiser (Sec. II-B, Example 2): an unrolled dual forward-backward
 * algorithm with K layers. W_k maps the image to P feature channels (a ks x ks
 * cross-correlation with zero padding), W_k^* is its adjoint, gamma_k its step
 * and HT the hard-tanh (clip to [-ht, ht]):
 *   D(v) = proj_[0,1]( v - gamma_K W_K^* G(W_K v) ),  G = T_{K-1} o ... o T_1,
 *   T_k(u) = HT( u + gamma_k W_k proj_[0,1](v - W_k^* u) ). */
typedef struct ora_ddfb_s {
    int K, P, ks;
    const double* w;         /* [K][P][ks*ks]                                 */
    const double* gamma;     /* [K]                                           */
    double ht;               /* hard-tanh threshold                           */
} ora_ddfb;

void ora_ddfb_W(const double* v, int ny, int nx, const double* wk, int P, int ks, double* u);
void ora_ddfb_Wt(const double* u, int ny, int nx, const double* wk, int P, int ks, double* v);
void ora_ddfb_denoise(const double* v, int ny, int nx, const ora_ddfb* net, double* out);

#ifdef __cplusplus
}
#endif
#endif
