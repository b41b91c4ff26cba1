/*
 * FP64 CPU oracle for the PnP-ULA Gaussian-deconvolution sampler.
 * TEST INFRASTRUCTURE ONLY: see oracle.h. Plain loops, written to be read
 * against the paper; OpenMP only splits independent output pixels.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static inline int wrap(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers:
 * as easy as 1, 2, 3"). One round: the two even counter words are multiplied
 * by the round multipliers; the high halves are xored with the odd words and
 * the key, the words are permuted; the key is bumped by the Weyl constants
 * between rounds.
 * ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normals xi[n], n = 0..N-1, for iteration t and chain `chain`.
 * Philox counter (floor(n/4), t, chain, 0), key (seed_lo, seed_hi); each
 * 32-bit word k -> u = ((k >> 8) + 1/2) 2^-24 in (0,1); Box-Muller maps
 * (u0,u1) -> xi[4m], xi[4m+1] and (u2,u3) -> xi[4m+2], xi[4m+3]. */
void ora_normals(uint64_t seed, uint32_t t, uint32_t chain, int64_t n, double* xi) {
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    const double two_pi = 6.283185307179586476925286766559;
    int64_t groups = (n + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < groups; ++m) {
        uint32_t ctr[4] = {(uint32_t)m, t, chain, 0u};
        uint32_t r[4];
        ora_philox4x32_10(ctr, key, r);
        double u[4];
        for (int k = 0; k < 4; ++k) u[k] = ((double)(r[k] >> 8) + 0.5) * (1.0 / 16777216.0);
        double z[4];
        for (int pair = 0; pair < 2; ++pair) {
            double rad = sqrt(-2.0 * log(u[2 * pair]));
            double ang = two_pi * u[2 * pair + 1];
            z[2 * pair] = rad * cos(ang);
            z[2 * pair + 1] = rad * sin(ang);
        }
        for (int k = 0; k < 4; ++k)
            if (4 * m + k < n) xi[4 * m + k] = z[k];
    }
}

/* ---------------------------------------------------------------------------
 * Blur operator H of the Gaussian-deconvolution likelihood, circular boundary:
 *   (h * x)[i,j] = sum_{a,b} h[a,b] x[(i - (a - kh/2)) mod ny, (j - (b - kw/2)) mod nx]
 * and its adjoint (correlation with h):
 *   (H^T r)[i,j] = sum_{a,b} h[a,b] r[(i + a - kh/2) mod ny, (j + b - kw/2) mod nx]
 * ------------------------------------------------------------------------- */
void ora_blur(const double* x, int ny, int nx, const double* h, int kh, int kw, double* out) {
    const int ry = kh / 2, rx = kw / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double s = 0.0;
            for (int a = 0; a < kh; ++a)
                for (int b = 0; b < kw; ++b)
                    s += h[a * kw + b] * x[(int64_t)wrap(i - (a - ry), ny) * nx + wrap(j - (b - rx), nx)];
            out[(int64_t)i * nx + j] = s;
        }
}

void ora_blur_adj(const double* r, int ny, int nx, const double* h, int kh, int kw, double* out) {
    const int ry = kh / 2, rx = kw / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double s = 0.0;
            for (int a = 0; a < kh; ++a)
                for (int b = 0; b < kw; ++b)
                    s += h[a * kw + b] * r[(int64_t)wrap(i + (a - ry), ny) * nx + wrap(j + (b - rx), nx)];
            out[(int64_t)i * nx + j] = s;
        }
}

/* ---------------------------------------------------------------------------
 * One CNN layer T(v) = eta(W v + b) with W a multichannel half-padding
 * (zero "same") ks x ks filter bank, written as a cross-correlation (the
 * convention of the deep-learning frameworks the denoisers are defined in):
 *   out[co,i,j] = b[co] + sum_ci sum_{p,q} w[co,ci,p,q] in[ci, i+p-ks/2, j+q-ks/2]
 * with in = 0 outside the image; eta = ReLU when relu != 0.
 * ------------------------------------------------------------------------- */
void ora_conv_layer(const double* in, int cin, int ny, int nx, const double* w,
                    const double* b, int cout, int ks, int relu, double* out) {
    const int r = ks / 2;
    const int64_t plane = (int64_t)ny * nx;
#pragma omp parallel for collapse(2) schedule(static)
    for (int co = 0; co < cout; ++co)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                double s = b ? b[co] : 0.0;
                for (int ci = 0; ci < cin; ++ci)
                    for (int p = 0; p < ks; ++p) {
                        int ii = i + p - r;
                        if (ii < 0 || ii >= ny) continue;
                        for (int q = 0; q < ks; ++q) {
                            int jj = j + q - r;
                            if (jj < 0 || jj >= nx) continue;
                            s += w[(((int64_t)co * cin + ci) * ks + p) * ks + q] *
                                 in[ci * plane + (int64_t)ii * nx + jj];
                        }
                    }
                if (relu && s < 0.0) s = 0.0;
                out[co * plane + (int64_t)i * nx + j] = s;
            }
}

static int64_t net_max_channels(const ora_net* net) {
    int64_t m = 1;
    for (int k = 0; k < net->K; ++k) {
        if (net->cin[k] > m) m = net->cin[k];
        if (net->cout[k] > m) m = net->cout[k];
    }
    return m;
}

/* G(v) = T_K o ... o T_1 (v), result (one channel) written to g. */
static void ora_cnn_forward(const double* v, int ny, int nx, const ora_net* net, double* g,
                            const unsigned char* keep /* optional mask: zero where 0 */) {
    const int64_t plane = (int64_t)ny * nx;
    const int64_t cmax = net_max_channels(net);
    double* a = (double*)malloc(sizeof(double) * cmax * plane);
    double* bb = (double*)malloc(sizeof(double) * cmax * plane);
    memcpy(a, v, sizeof(double) * plane);
    const double* w = net->w;
    const double* b = net->b;
    for (int k = 0; k < net->K; ++k) {
        int relu = (k < net->K - 1);
        ora_conv_layer(a, net->cin[k], ny, nx, w, b, net->cout[k], net->ks, relu, bb);
        if (keep)
            for (int c = 0; c < net->cout[k]; ++c)
                for (int64_t n = 0; n < plane; ++n)
                    if (!keep[n]) bb[c * plane + n] = 0.0;
        w += (int64_t)net->cout[k] * net->cin[k] * net->ks * net->ks;
        b += net->cout[k];
        double* t = a; a = bb; bb = t;
    }
    memcpy(g, a, sizeof(double) * plane);
    free(a);
    free(bb);
}

/* DnCNN form: D(v) = (Id - G)(v). */
void ora_denoise(const double* v, int ny, int nx, const ora_net* net, double* out) {
    const int64_t plane = (int64_t)ny * nx;
    double* g = (double*)malloc(sizeof(double) * plane);
    ora_cnn_forward(v, ny, nx, net, g, NULL);
    for (int64_t n = 0; n < plane; ++n) out[n] = v[n] - g[n];
    free(g);
}

/* Block-wise denoiser (Defs. 1-2 with the receptive-field halo variant of
 * Sec. II-B2): the image is split into by x bx blocks by the floor rule
 * rows floor(b ny / by) .. floor((b+1) ny / by) - 1 (same per column axis);
 * each block is extended by `halo` pixels on every side (the ghost region),
 * the network runs on the extended tile alone with positions outside the
 * image held at zero after every layer (they are padding in the whole-image
 * network), and only the block interior is kept. Equals ora_denoise when
 * halo >= K (3x3 layers). Returns 0, or -1 on bad arguments. */
int ora_denoise_blockwise(const double* v, int ny, int nx, const ora_net* net,
                          int by, int bx, int halo, double* out) {
    if (by < 1 || bx < 1 || by > ny || bx > nx || halo < 0) return -1;
    for (int bi = 0; bi < by; ++bi) {
        int r0 = (int)(((int64_t)bi * ny) / by), r1 = (int)(((int64_t)(bi + 1) * ny) / by);
        for (int bj = 0; bj < bx; ++bj) {
            int c0 = (int)(((int64_t)bj * nx) / bx), c1 = (int)(((int64_t)(bj + 1) * nx) / bx);
            int ty = r1 - r0 + 2 * halo, tx = c1 - c0 + 2 * halo;
            int64_t tp = (int64_t)ty * tx;
            double* tile = (double*)calloc(tp, sizeof(double));
            unsigned char* keep = (unsigned char*)calloc(tp, 1);
            double* g = (double*)malloc(sizeof(double) * tp);
            for (int i = 0; i < ty; ++i)
                for (int j = 0; j < tx; ++j) {
                    int gi = r0 - halo + i, gj = c0 - halo + j;
                    if (gi >= 0 && gi < ny && gj >= 0 && gj < nx) {
                        tile[(int64_t)i * tx + j] = v[(int64_t)gi * nx + gj];
                        keep[(int64_t)i * tx + j] = 1;
                    }
                }
            ora_cnn_forward(tile, ty, tx, net, g, keep);
            for (int i = r0; i < r1; ++i)
                for (int j = c0; j < c1; ++j) {
                    int64_t ti = (int64_t)(i - r0 + halo) * tx + (j - c0 + halo);
                    out[(int64_t)i * nx + j] = v[(int64_t)i * nx + j] - g[ti];
                }
            free(tile);
            free(keep);
            free(g);
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Step sizes, Gaussian-noise setting with f2 = 0 (so H_2 = 0 in Eq. 10):
 *   L      = ||H||^2 / sigma^2                  (Lipschitz constant of grad f1 o H1)
 *   lambda = 0.99 / (4 L + 2 alpha L_eps / eps^2)
 *   gamma  = c / (3 (L + alpha L_eps / eps^2 + 1/lambda))
 * The paper's printed gamma carries a Poisson-case term; with H_2 = 0 it
 * reduces to the expression above, which satisfies Eq. 10 for c < 1.
 * ------------------------------------------------------------------------- */
void ora_stepsizes(double hnorm, double sigma, double alpha, double eps, double lip_eps,
                   double c, double* lambda, double* gamma) {
    double L = hnorm * hnorm / (sigma * sigma);
    double prior = alpha * lip_eps / (eps * eps);
    double lam = 0.99 / (4.0 * L + 2.0 * prior);
    *lambda = lam;
    *gamma = c / (3.0 * (L + prior + 1.0 / lam));
}

/* ---------------------------------------------------------------------------
 * One PnP-ULA transition (Eq. 8, x-update of Algorithm 1 with f2 = 0):
 *   x+ = x - gamma H^T (H x - y) / sigma^2
 * (H the circular blur h, or for inpainting the diagonal selection mask,
 * H = H^T = diag(mask), Sec. IV-A)
 *          + (alpha gamma / eps^2) (D(x) - x)
 *          + (gamma / lambda) (proj_[0,1](x) - x)
 *          + sqrt(2 gamma) xi,     xi = normals(seed, t, chain)
 * ------------------------------------------------------------------------- */
void ora_langevin_step(const ora_problem* p, const double* x, uint32_t t, uint32_t chain,
                       double* xnew) {
    const int64_t N = (int64_t)p->ny * p->nx;
    double* r = (double*)malloc(sizeof(double) * N);
    double* g = (double*)malloc(sizeof(double) * N);
    double* d = (p->net || p->ddfb) ? (double*)malloc(sizeof(double) * N) : NULL;
    double* xi = (double*)calloc(N, sizeof(double));
    if (p->mask) {
        for (int64_t n = 0; n < N; ++n) r[n] = p->mask[n] * x[n] - p->y[n];
        for (int64_t n = 0; n < N; ++n) g[n] = p->mask[n] * r[n];
    } else {
        ora_blur(x, p->ny, p->nx, p->h, p->kh, p->kw, r);
        for (int64_t n = 0; n < N; ++n) r[n] -= p->y[n];
        ora_blur_adj(r, p->ny, p->nx, p->h, p->kh, p->kw, g);
    }
    if (d && p->net) ora_denoise(x, p->ny, p->nx, p->net, d);
    else if (d) ora_ddfb_denoise(x, p->ny, p->nx, p->ddfb, d);
    if (p->noise) ora_normals(p->seed, t, chain, N, xi);
    const double gam = p->gamma;
    const double s2 = p->sigma * p->sigma;
    const double cprior = p->alpha * gam / (p->eps * p->eps);
    const double cproj = p->lambda > 0.0 ? gam / p->lambda : 0.0;
    const double cnoise = sqrt(2.0 * gam);
    for (int64_t n = 0; n < N; ++n) {
        double xv = x[n];
        double v = xv - gam * g[n] / s2;
        if (d) v += cprior * (d[n] - xv);
        double pr = xv < 0.0 ? 0.0 : (xv > 1.0 ? 1.0 : xv);
        v += cproj * (pr - xv);
        v += cnoise * xi[n];
        xnew[n] = v;
    }
    free(r);
    free(g);
    free(d);
    free(xi);
}

/* Standard normal xi[n] of ora_normals for one flat index n: Philox group
 * floor(n/4), word n mod 4, Box-Muller on the word pair holding it. */
static double normal_at(uint64_t seed, uint32_t t, uint32_t chain, int64_t n) {
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t ctr[4] = {(uint32_t)(n / 4), t, chain, 0u};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    const int k = (int)(n % 4), pair = k / 2;
    double u0 = ((double)(r[2 * pair] >> 8) + 0.5) * (1.0 / 16777216.0);
    double u1 = ((double)(r[2 * pair + 1] >> 8) + 0.5) * (1.0 / 16777216.0);
    double rad = sqrt(-2.0 * log(u0));
    double ang = two_pi * u1;
    return (k % 2 == 0) ? rad * cos(ang) : rad * sin(ang);
}

/* ---------------------------------------------------------------------------
 * The transition of ora_langevin_step evaluated only at the output pixels of
 * the window [i0, i0 + wy) x [j0, j0 + wx) of the image (for images too large
 * to step whole in FP64). Each term is its definition restricted to the
 * window: the residual r = h * x - y on the window grown by the blur radius
 * (circular indices into the whole x), g = H^T r on the window, the
 * denoiser on the crop of x that extends the window by the network's
 * receptive radius K (ks / 2) (clipped at the image border, where its zero
 * padding is the image's own), and xi at the pixels' global flat indices.
 * Sums run in the same order as the whole-image routines, so the window
 * equals the corresponding part of ora_langevin_step exactly. out: [wy][wx].
 * Returns 0, or -1 for a window outside the image or a DDFB denoiser.
 * ------------------------------------------------------------------------- */
int ora_langevin_step_window(const ora_problem* p, const double* x, uint32_t t, uint32_t chain,
                             int i0, int j0, int wy, int wx, double* out) {
    const int ny = p->ny, nx = p->nx;
    if (wy < 1 || wx < 1 || i0 < 0 || j0 < 0 || i0 + wy > ny || j0 + wx > nx) return -1;
    if (!p->net && p->ddfb) return -1;
    const int ry = p->mask ? 0 : p->kh / 2, rx = p->mask ? 0 : p->kw / 2;
    /* residual on the window grown by (ry, rx): rows i0 - ry .. i0 + wy - 1 + ry */
    const int ey = wy + 2 * ry, ex = wx + 2 * rx;
    double* r = (double*)malloc(sizeof(double) * (int64_t)ey * ex);
    for (int u = 0; u < ey; ++u)
        for (int v = 0; v < ex; ++v) {
            const int qi = wrap(i0 - ry + u, ny), qj = wrap(j0 - rx + v, nx);
            const int64_t q = (int64_t)qi * nx + qj;
            double s;
            if (p->mask) {
                s = p->mask[q] * x[q];
            } else {
                s = 0.0;
                for (int a = 0; a < p->kh; ++a)
                    for (int b = 0; b < p->kw; ++b)
                        s += p->h[a * p->kw + b] *
                             x[(int64_t)wrap(qi - (a - ry), ny) * nx + wrap(qj - (b - rx), nx)];
            }
            r[(int64_t)u * ex + v] = s - p->y[q];
        }
    /* denoiser on the crop that covers the window's receptive field */
    double* d = NULL;
    int ci0 = 0, cj0 = 0, cy = 0, cx = 0;
    if (p->net) {
        const int R = p->net->K * (p->net->ks / 2);
        ci0 = i0 - R < 0 ? 0 : i0 - R;
        cj0 = j0 - R < 0 ? 0 : j0 - R;
        const int ci1 = i0 + wy + R > ny ? ny : i0 + wy + R;
        const int cj1 = j0 + wx + R > nx ? nx : j0 + wx + R;
        cy = ci1 - ci0;
        cx = cj1 - cj0;
        double* crop = (double*)malloc(sizeof(double) * (int64_t)cy * cx);
        d = (double*)malloc(sizeof(double) * (int64_t)cy * cx);
        for (int u = 0; u < cy; ++u)
            memcpy(crop + (int64_t)u * cx, x + (int64_t)(ci0 + u) * nx + cj0, sizeof(double) * cx);
        ora_denoise(crop, cy, cx, p->net, d);
        free(crop);
    }
    const double gam = p->gamma;
    const double s2 = p->sigma * p->sigma;
    const double cprior = p->alpha * gam / (p->eps * p->eps);
    const double cproj = p->lambda > 0.0 ? gam / p->lambda : 0.0;
    const double cnoise = sqrt(2.0 * gam);
    for (int u = 0; u < wy; ++u)
        for (int v = 0; v < wx; ++v) {
            const int i = i0 + u, j = j0 + v;
            const int64_t n = (int64_t)i * nx + j;
            double g;
            if (p->mask) {
                g = p->mask[n] * r[(int64_t)u * ex + v];
            } else {
                g = 0.0;
                for (int a = 0; a < p->kh; ++a)
                    for (int b = 0; b < p->kw; ++b)
                        g += p->h[a * p->kw + b] * r[(int64_t)(u + a) * ex + (v + b)];
            }
            const double xv = x[n];
            double val = xv - gam * g / s2;
            if (d) val += cprior * (d[(int64_t)(i - ci0) * cx + (j - cj0)] - xv);
            const double pr = xv < 0.0 ? 0.0 : (xv > 1.0 ? 1.0 : xv);
            val += cproj * (pr - xv);
            val += cnoise * (p->noise ? normal_at(p->seed, t, chain, n) : 0.0);
            out[(int64_t)u * wx + v] = val;
        }
    free(r);
    free(d);
    return 0;
}

void ora_run_chain(const ora_problem* p, double* x, int t0, int T, int burn_in,
                   uint32_t chain, double* mean, double* m2, int64_t* n_kept,
                   double* samples) {
    const int64_t N = (int64_t)p->ny * p->nx;
    double* xn = (double*)malloc(sizeof(double) * N);
    for (int t = t0; t < t0 + T; ++t) {
        ora_langevin_step(p, x, (uint32_t)t, chain, xn);
        memcpy(x, xn, sizeof(double) * N);
        if (t + 1 > burn_in) {
            int64_t k = ++(*n_kept);
            for (int64_t n = 0; n < N; ++n) {
                double delta = x[n] - mean[n];
                mean[n] += delta / (double)k;
                m2[n] += delta * (x[n] - mean[n]);
            }
            if (samples) memcpy(samples + (k - 1) * N, x, sizeof(double) * N);
        }
    }
    free(xn);
}

void ora_normals_stream(uint64_t seed, uint32_t t, uint32_t chain, uint32_t stream, int64_t n,
                        double* xi) {
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    const double two_pi = 6.283185307179586476925286766559;
    int64_t groups = (n + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < groups; ++m) {
        uint32_t ctr[4] = {(uint32_t)m, t, chain, stream};
        uint32_t w[4];
        ora_philox4x32_10(ctr, key, w);
        double u[4];
        for (int k = 0; k < 4; ++k) u[k] = ((double)(w[k] >> 8) + 0.5) * 5.9604644775390625e-08;
        double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
        double z[4] = {r0 * cos(two_pi * u[1]), r0 * sin(two_pi * u[1]),
                       r1 * cos(two_pi * u[3]), r1 * sin(two_pi * u[3])};
        for (int k = 0; k < 4; ++k)
            if (4 * m + k < n) xi[4 * m + k] = z[k];
    }
}

double ora_kl_prox(double v, double y, double kappa) {
    /* minimiser of kappa (u - y log u) + (u - v)^2 / 2 over u > 0 (u >= 0 when y = 0) */
    double a = v - kappa;
    return 0.5 * (a + sqrt(a * a + 4.0 * kappa * y));
}

void ora_poisson_stepsizes(double hnorm, double eta, double rho1, double rho2, double alpha,
                           double eps, double lip_eps, double c, double* lambda, double* gamma,
                           double* kappa1, double* kappa2) {
    double c1 = eta * hnorm * eta * hnorm / rho1; /* ||eta H||^2 / rho1 */
    double c2 = 1.0 / rho2;
    double prior = alpha * lip_eps / (eps * eps);
    double lam = 0.99 / (4.0 * c1 + 4.0 * c2 + 2.0 * prior);
    *lambda = lam;
    *gamma = c / (3.0 * (prior + c1 + c2 + 1.0 / lam));
    *kappa1 = 0.99 * rho1;
    *kappa2 = 0.99 * rho2;
}

/* ---------------------------------------------------------------------------
 * One transition of the Poisson sampler (Eqs. 13-14 with f1 = 0 and the two
 * AXDA blocks):
 *   x+  = x - gamma [ (eta/rho1) H^T (eta H x - z1) + (x - z2)/rho2 ]
 *           + (alpha gamma / eps^2)(D(x) - x) + (gamma / lambda)(proj_[0,1](x) - x)
 *           + sqrt(2 gamma) xi                                   (xi: stream 0)
 *   z1+ = prox_{kappa1 KL(y||.)}( z1 - (kappa1/rho1)(z1 - eta H x+) + sqrt(2 kappa1) zeta1 )
 *   z2+ = max( z2 - (kappa2/rho2)(z2 - x+) + sqrt(2 kappa2) zeta2, 0 )
 * ------------------------------------------------------------------------- */
void ora_poisson_step(const ora_poisson* p, const double* x, const double* z1, const double* z2,
                      uint32_t t, uint32_t chain, double* xnew, double* z1new, double* z2new) {
    const int64_t N = (int64_t)p->ny * p->nx;
    double* r = (double*)malloc(sizeof(double) * N);
    double* g = (double*)malloc(sizeof(double) * N);
    double* d = p->net ? (double*)malloc(sizeof(double) * N) : NULL;
    double* xi = (double*)calloc(N, sizeof(double));
    double* ze1 = (double*)calloc(N, sizeof(double));
    double* ze2 = (double*)calloc(N, sizeof(double));
    /* x-update */
    ora_blur(x, p->ny, p->nx, p->h, p->kh, p->kw, r);
    for (int64_t n = 0; n < N; ++n) r[n] = p->eta * r[n] - z1[n];
    ora_blur_adj(r, p->ny, p->nx, p->h, p->kh, p->kw, g);
    if (d) ora_denoise(x, p->ny, p->nx, p->net, d);
    if (p->noise) {
        ora_normals_stream(p->seed, t, chain, 0, N, xi);
        ora_normals_stream(p->seed, t, chain, 1, N, ze1);
        ora_normals_stream(p->seed, t, chain, 2, N, ze2);
    }
    const double gam = p->gamma;
    const double cprior = p->alpha * gam / (p->eps * p->eps);
    const double cproj = p->lambda > 0.0 ? gam / p->lambda : 0.0;
    for (int64_t n = 0; n < N; ++n) {
        double xv = x[n];
        double grad = (p->eta / p->rho1) * g[n] + (xv - z2[n]) / p->rho2;
        double v = xv - gam * grad;
        if (d) v += cprior * (d[n] - xv);
        double pr = xv < 0.0 ? 0.0 : (xv > 1.0 ? 1.0 : xv);
        v += cproj * (pr - xv);
        v += sqrt(2.0 * gam) * xi[n];
        xnew[n] = v;
    }
    /* z-update from the new x */
    ora_blur(xnew, p->ny, p->nx, p->h, p->kh, p->kw, r);
    for (int64_t n = 0; n < N; ++n) {
        double w1 = z1[n] - (p->kappa1 / p->rho1) * (z1[n] - p->eta * r[n]) +
                    sqrt(2.0 * p->kappa1) * ze1[n];
        z1new[n] = ora_kl_prox(w1, p->y[n], p->kappa1);
        double w2 = z2[n] - (p->kappa2 / p->rho2) * (z2[n] - xnew[n]) +
                    sqrt(2.0 * p->kappa2) * ze2[n];
        z2new[n] = w2 > 0.0 ? w2 : 0.0;
    }
    free(r);
    free(g);
    free(d);
    free(xi);
    free(ze1);
    free(ze2);
}

/* Two-pass moments of stored samples: mean, then unbiased variance. */
void ora_moments_two_pass(const double* samples, int64_t n, int64_t npix,
                          double* mean, double* var) {
    for (int64_t j = 0; j < npix; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s += samples[k * npix + j];
        double m = s / (double)n;
        double q = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double dlt = samples[k * npix + j] - m;
            q += dlt * dlt;
        }
        mean[j] = m;
        var[j] = n > 1 ? q / (double)(n - 1) : 0.0;
    }
}

/* ---------------------------------------------------------------------------
 * DDFB denoiser (Sec. II-B, Example 2).
 *   W_k v:    u_p(i,j) = sum_{a,b} w_k[p][a][b] v(i + a - r, j + b - r)
 *   W_k^* u:  v(i,j)   = sum_p sum_{a,b} w_k[p][a][b] u_p(i - a + r, j - b + r)
 * (r = ks / 2, zero outside the image), the exact adjoint of the first.
 * ------------------------------------------------------------------------- */
void ora_ddfb_W(const double* v, int ny, int nx, const double* wk, int P, int ks, double* u) {
    const int r = ks / 2;
    const int64_t plane = (int64_t)ny * nx;
    for (int p = 0; p < P; ++p)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j) {
                double s = 0.0;
                for (int a = 0; a < ks; ++a)
                    for (int b = 0; b < ks; ++b) {
                        const int ii = i + a - r, jj = j + b - r;
                        if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
                        s += wk[(p * ks + a) * ks + b] * v[(int64_t)ii * nx + jj];
                    }
                u[p * plane + (int64_t)i * nx + j] = s;
            }
}

void ora_ddfb_Wt(const double* u, int ny, int nx, const double* wk, int P, int ks, double* v) {
    const int r = ks / 2;
    const int64_t plane = (int64_t)ny * nx;
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j) {
            double s = 0.0;
            for (int p = 0; p < P; ++p)
                for (int a = 0; a < ks; ++a)
                    for (int b = 0; b < ks; ++b) {
                        const int ii = i - a + r, jj = j - b + r;
                        if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
                        s += wk[(p * ks + a) * ks + b] * u[p * plane + (int64_t)ii * nx + jj];
                    }
            v[(int64_t)i * nx + j] = s;
        }
}

static double clip01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

void ora_ddfb_denoise(const double* v, int ny, int nx, const ora_ddfb* net, double* out) {
    const int64_t plane = (int64_t)ny * nx;
    const int K = net->K, P = net->P, ks = net->ks;
    const int64_t wsz = (int64_t)P * ks * ks;
    double* u = (double*)malloc(sizeof(double) * P * plane);
    double* wu = (double*)malloc(sizeof(double) * P * plane);
    double* s = (double*)malloc(sizeof(double) * plane);
    /* dual variable initialised at W_K v */
    ora_ddfb_W(v, ny, nx, net->w + (K - 1) * wsz, P, ks, u);
    for (int k = 0; k < K - 1; ++k) {
        const double* wk = net->w + k * wsz;
        ora_ddfb_Wt(u, ny, nx, wk, P, ks, s);
        for (int64_t n = 0; n < plane; ++n) s[n] = clip01(v[n] - s[n]);
        ora_ddfb_W(s, ny, nx, wk, P, ks, wu);
        for (int64_t n = 0; n < P * plane; ++n) {
            const double a = u[n] + net->gamma[k] * wu[n];
            u[n] = a < -net->ht ? -net->ht : (a > net->ht ? net->ht : a);
        }
    }
    ora_ddfb_Wt(u, ny, nx, net->w + (K - 1) * wsz, P, ks, s);
    for (int64_t n = 0; n < plane; ++n) out[n] = clip01(v[n] - net->gamma[K - 1] * s[n]);
    free(u);
    free(wu);
    free(s);
}
