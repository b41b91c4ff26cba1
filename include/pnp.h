/*
 * pnp.h -- C ABI of the B300 (sm_103a) PnP-ULA sampler for Gaussian deconvolution.
 *
 * The library runs the x-update of the paper's distributed sampler
 * (Algorithm 1 with f2 = 0, Sec. III-A2 / III-B(i)) on one GPU:
 *
 *   x+ = x - gamma H^T (H x - y) / sigma^2 + (alpha gamma / eps^2) (D_eps(x) - x)
 *          + (gamma / lambda) (proj_[0,1](x) - x) + sqrt(2 gamma) xi          (Eq. 8)
 *
 * with H a circular 2-D blur, D_eps a DnCNN-form denoiser (Sec. II-B, Example 1)
 * evaluated block-wise (Defs. 1-2), xi drawn from a counter-based Philox stream,
 * and MMSE / pixel-wise variance accumulated online after burn-in (Sec. III-C).
 *
 * Poisson observations (Sec. IV-B) use the asymptotically exact data
 * augmentation of Sec. III-A with two auxiliary variables, z1 (coupled to
 * eta H x with tolerance rho1) and z2 (coupled to x with tolerance rho2); each
 * iteration runs the x-update with the coupling gradients in place of the
 * Gaussian data term, then one proximal Langevin (PSGLA) step per auxiliary
 * variable: z1 through the proximal map of the Poisson negative log-likelihood,
 * z2 through the projection onto the non-negative orthant.
 *
 * Conventions for every entry point:
 *  - Return value is a pnp_status; PNP_OK on success. On failure nothing is
 *    left half-done on the host side and pnp_last_error() returns a
 *    thread-local message.
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are ordinary CPU memory. The caller owns every buffer it
 *    passes; objects created by the library own their own device memory and
 *    free it in the matching destroy call.
 *  - stream arguments are cudaStream_t passed as void* (NULL = legacy default
 *    stream). Operator entry points are asynchronous on that stream.
 *  - Images are row-major FP32 [ny][nx], one channel. Multi-chain and batch
 *    arrays are [n][ny][nx] with the image index slowest.
 *  - No callbacks, no exceptions cross the ABI. Calls on one object are not
 *    thread-safe; different objects may be used from different threads.
 */
#ifndef PNP_H
#define PNP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PNP_OK = 0,
    PNP_EINVAL = 1,    /* bad argument (sizes, pointers, step sizes, halo < K ...) */
    PNP_ENOMEM = 2,    /* device allocation failed                                */
    PNP_EBUSY = 3,     /* admission refused: request can never fit the budget    */
    PNP_ECUDA = 4,     /* CUDA runtime / driver error (message in pnp_last_error) */
    PNP_ETIMEOUT = 5,  /* a bounded device-side wait ran out                      */
    PNP_ESTATE = 6,    /* call not valid in the object's current state           */
    PNP_ENOTSUP = 7    /* feature not supported on this device                    */
} pnp_status;

typedef enum {
    PNP_FP32 = 0,      /* denoiser convolutions in FP32 on CUDA cores                     */
    PNP_BF16 = 1,      /* BF16 operands, FP32 accumulation, tcgen05 tensor cores          */
    PNP_FP8 = 2        /* E4M3 operands with per-output-channel scales, FP32 accumulation */
} pnp_precision;

typedef enum {
    PNP_GAUSSIAN = 0,  /* y = H x + sigma n, n ~ N(0, I): the x-update of Eq. 8                 */
    PNP_POISSON = 1    /* y ~ Poisson(eta H x): AXDA split with z1 ~ eta H x, z2 ~ x (Sec. IV-B) */
} pnp_noise_model;

typedef struct pnp_denoiser pnp_denoiser;
typedef struct pnp_problem pnp_problem;
typedef struct pnp_batch pnp_batch;
typedef struct pnp_server pnp_server;

/* Thread-local description of the last failure on this thread ("" if none). */
const char* pnp_last_error(void);
/* Library version string. */
const char* pnp_version(void);

/* ------------------------------------------------------------------------
 * Denoiser D_eps = Id - G_eps, G_eps = T_K o ... o T_1,
 * T_k(v) = ReLU(W_k v + b_k) for k < K, T_K(v) = W_K v + b_K
 * (Sec. II-B, Eqs. 5-6 and Example 1 "DnCNN").
 * Layers: 1 -> F, F -> F (K-2 times), F -> 1; 3x3 zero-padded ("half
 * padding") cross-correlations. weights: host FP32, per layer OIHW
 * [cout][cin][3][3], concatenated in layer order; biases: host FP32 [cout]
 * per layer, concatenated. Both are copied. lipschitz_eps is the L_eps bound
 * of Id - D_eps used for the step sizes (Sec. II-C). Supported: K >= 2,
 * F in {16, 32, 64} for FP32; F = 64 for BF16/FP8.
 * ------------------------------------------------------------------------ */
pnp_status pnp_create_denoiser(int K, int F, const float* weights, const float* biases,
                               double lipschitz_eps, pnp_denoiser** out);
void pnp_destroy_denoiser(pnp_denoiser* d);

/* Static activation scales of the FP8 (E4M3) variant: runs the FP32 network
 * on x (device [nimg][ny][nx]) and sets the scale of every layer's input to
 * twice its largest activation / 448. Weights are quantised per output
 * channel (amax / 448) at creation. pnp_denoise with PNP_FP8 calibrates on its
 * own input and pnp_create_problem on the observation y if this was not
 * called before. Synchronous; allocates temporary scratch. */
pnp_status pnp_denoiser_calibrate_fp8(pnp_denoiser* d, const float* x, int ny, int nx, int nimg,
                                      void* stream);

/* ------------------------------------------------------------------------
 * Operator entry points (device pointers, asynchronous on `stream`).
 * ------------------------------------------------------------------------ */

/* r[c] = h (*) x[c] - y for c < nimg: circular convolution with the kh x kw
 * kernel h (anchored at (kh/2, kw/2)), Gaussian-deconvolution likelihood
 * residual (Sec. III-A2, Eq. 12). x, r: device [nimg][ny][nx]; y: device
 * [ny][nx] or NULL (then r = h (*) x); h: device [kh][kw]. kh, kw odd,
 * <= 31 and <= the image size. */
pnp_status pnp_blur(const float* x, const float* y, const float* h, int kh, int kw,
                    int ny, int nx, int nimg, float* r, void* stream);

/* g[c] = scale * H^T r[c]: circular correlation with h (the adjoint of
 * pnp_blur's operator). Same layout rules as pnp_blur. */
pnp_status pnp_blur_adjoint(const float* r, const float* h, int kh, int kw, int ny, int nx,
                            int nimg, float scale, float* g, void* stream);

/* d[c] = D_eps(x[c]) for nimg images [nimg][ny][nx] (device). halo == 0:
 * layers run over the whole image, each tile reading its neighbours' pixels
 * directly (exact whole-image result for any block split). halo > 0: the
 * image is cut into blocks_y x blocks_x blocks (floor rule, Sec. II-B2 Eq. 7),
 * each block is extended by `halo` pixels, the network runs on every extended
 * block independently with out-of-image positions held at zero after every
 * layer, and block interiors are written back (receptive-field variant,
 * Sec. II-B2); equals the halo == 0 result iff halo >= K.
 * Scratch: the library allocates and caches device scratch per denoiser
 * (activations of two layers). */
pnp_status pnp_denoise(const pnp_denoiser* D, pnp_precision prec, const float* x, int ny,
                       int nx, int nimg, int blocks_y, int blocks_x, int halo, float* d,
                       void* stream);

/* Size of the fixed scratch area used by pnp_denoise_noalloc (64 MiB + 4 KiB). */
#define PNP_NOALLOC_SCRATCH_BYTES ((size_t)64 * 1024 * 1024 + 4096)

/* pnp_denoise without any device allocation. The paper has no counterpart:
 * this is a library-level variant for callers that must not allocate, such
 * as a process whose device memory is already reserved by another allocator
 * (a raw cudaMalloc would fail there) or a latency-bound loop that cannot
 * afford cudaMalloc/cudaFree synchronizing the device.
 * Same arguments and result as pnp_denoise with halo = 0 (whole-image
 * layers) for PNP_FP32 and PNP_BF16; PNP_FP8 returns PNP_ENOTSUP. Scratch is
 * a fixed area inside the library (a file-scope __device__ array of
 * PNP_NOALLOC_SCRATCH_BYTES), held on a GPU until the process exits. It needs
 *   FP32: 8 * F * nimg * ny * nx bytes,  BF16: 256 * nimg * ny * ceil8(nx) + 256 bytes
 * (BF16 fits a 512 x 512 image; FP32 with F = 64 fits about 362 x 362);
 * larger requests return PNP_EINVAL with the needed size and launch nothing.
 * The area is reserved, and its device address looked up
 * (cudaGetSymbolAddress), by pnp_create_denoiser on the device current at
 * creation: create the denoiser before another allocator takes the device's
 * memory. On any other device the first call does the lookup (and
 * reservation); make that first call before any stream capture.
 * All calls on a device share its one area and it keeps the previous call's
 * contents, so calls that can overlap on the GPU (for example on two streams
 * of the same device) race: serialize them on one stream. Calls no
 * cudaMalloc, cudaFree or other allocating routine. A tensor-core wait that
 * ran out is reported by pnp_denoise_status. */
pnp_status pnp_denoise_noalloc(const pnp_denoiser* D, pnp_precision prec, const float* x,
                               int ny, int nx, int nimg, float* d, void* stream);

/* Waits for `stream`, then reports whether a bounded device-side wait ran out
 * in a tensor-core layer of an earlier pnp_denoise or pnp_denoise_noalloc
 * call with D since the last report: PNP_ETIMEOUT (the flag is then cleared;
 * the outputs of the affected call are incomplete) or PNP_OK. The paper has
 * no counterpart: this is the library's error channel for its bounded waits
 * (each wait gives up after about two seconds instead of hanging the GPU). */
pnp_status pnp_denoise_status(const pnp_denoiser* D, void* stream);

/* Test hook (no counterpart in the paper): arms a one-shot fault for the next
 * F -> F tensor-core layer launched outside stream capture, on any thread:
 * CTA `cta` of that launch skips issuing its TMA load number `load_index`
 * (nothing is in flight for it), and every wait of that launch gives up
 * after budget_cycles SM clock cycles (>= 1000) instead of the default. The
 * CTA waiting for the missing row then aborts, waits for its own copies and
 * MMAs already in flight, releases its tensor memory and sets the caller's
 * timeout flag, which the next synchronising call reports as PNP_ETIMEOUT. */
pnp_status pnp_debug_inject_tc_timeout(int cta, int load_index, long long budget_cycles);
/* Test hook (no counterpart in the paper): arms a one-shot fault for the next
 * launch of the pipelined one-pass update (k_update_os: a single problem with
 * a separable blur of at most 15 taps under Gaussian noise) made outside
 * stream capture: CTA `cta` does not issue the shared-memory window of its
 * tile number `tile_index` (nothing is in flight for it), and the launch's
 * waits give up after budget_cycles (>= 1000). That CTA then waits for its own
 * copies in flight, sets the problem's timeout flag (PNP_ETIMEOUT at the next
 * synchronising call), skips its remaining tiles and still arrives on the
 * step counter. An out-of-range cta or tile_index leaves the launch
 * unaffected. */
pnp_status pnp_debug_inject_update_timeout(int cta, int tile_index, long long budget_cycles);

/* One fused PnP-ULA x-update (Eq. 8) for nchain chains sharing y and h:
 *   g = H^T r / sigma^2 (r = H x - y from pnp_blur, device [nchain][ny][nx]),
 *   x <- x - gamma g + (alpha gamma/eps^2)(d - x) + (gamma/lambda)(clamp(x,0,1) - x)
 *        + sqrt(2 gamma) xi,
 * xi[n] standard normal from Philox4x32-10 with counter (n/4, t, chain, 0) and
 * key (seed low, seed high), Box-Muller on word pairs. d: device [nchain][ny][nx]
 * or NULL (no prior term). lambda <= 0 switches the projection term off;
 * noise = 0 sets xi = 0. If n_kept > 0 the new x enters the FP32 Welford
 * accumulators (mean, m2; device [nchain][ny][nx]) as sample number n_kept. */
pnp_status pnp_langevin_update(float* x, const float* r, const float* d, const float* h,
                               int kh, int kw, int ny, int nx, int nchain, double sigma,
                               double alpha, double eps, double lambda, double gamma,
                               uint64_t seed, uint32_t t, int noise, float* mean, float* m2,
                               int64_t n_kept, void* stream);

/* Inpainting x-update (Eq. 8 with H = diag(mask), Sec. IV-A) for nchain
 * chains: g = x - y at observed pixels and 0 at missing ones, then the same
 * update, noise and Welford accumulation as pnp_langevin_update. y_obs:
 * device [ny][nx] shared by the chains, NaN at missing pixels (the mask is
 * read from it). x, d, mean, m2: device [nchain][ny][nx]. No stencil. */
pnp_status pnp_inpaint_update(float* x, const float* y_obs, const float* d, int ny, int nx,
                              int nchain, double sigma, double alpha, double eps, double lambda,
                              double gamma, uint64_t seed, uint32_t t, int noise, float* mean,
                              float* m2, int64_t n_kept, void* stream);

/* Final FP64 moments (Sec. III-C footnote): mmse = mean, var = m2 / (n - 1),
 * out2 = var (want_var != 0) or sqrt(var). mean, m2: device FP32 [n];
 * mmse, out2: device FP64 [n]. */
pnp_status pnp_finalize_moments(const float* mean, const float* m2, int64_t npix,
                                int64_t n_kept, int want_var, double* mmse, double* out2,
                                void* stream);

/* DDFB denoiser (Sec. II-B, Example 2): an unrolled dual forward-backward
 * algorithm with K layers, each with P analysis filters W_k (1 -> P channel
 * 3 x 3 cross-correlation, zero padding) and its adjoint W_k^*:
 *   u_0 = W_K v,
 *   u_k = HT(u_{k-1} + gamma_k W_k proj_[0,1](v - W_k^* u_{k-1})),  k = 1 .. K-1,
 *   D(v) = proj_[0,1](v - gamma_K W_K^* u_{K-1}),
 * HT = clip to [-ht, ht]. filters: host [K][P][3][3], gammas: host [K] (> 0);
 * both copied. 2 <= K <= 32, P in {16, 32, 64}, ht > 0. The result is a
 * pnp_denoiser for pnp_denoise / problems with PNP_FP32 and halo = 0 (its
 * FP32 kernels stream the P-channel dual variable; other precisions give
 * PNP_ENOTSUP). Its L_eps for the step sizes is 1 (Id - D is nonexpansive). */
pnp_status pnp_create_ddfb(int K, int P, const float* filters, const float* gammas, double ht,
                           pnp_denoiser** out);

/* Step sizes of the Gaussian-noise setting (Eq. 10 with H_2 = 0):
 * L = hnorm^2/sigma^2, lambda = 0.99 / (4L + 2 alpha L_eps / eps^2),
 * gamma = c / (3 (L + alpha L_eps / eps^2 + 1/lambda)), 0 < c < 1. */
pnp_status pnp_stepsizes(double hnorm, double sigma, double alpha, double eps, double lip_eps,
                         double c, double* lambda, double* gamma);

/* Step sizes of the Poisson setting (Eq. 12 with f1 = 0 and the AXDA
 * couplings as the smooth term: ||H_2||^2 = eta^2 hnorm^2 / rho1 + 1 / rho2):
 * lambda = 0.99 / (4 ||H_2||^2 + 2 alpha L_eps / eps^2),
 * gamma = c / (3 (alpha L_eps / eps^2 + ||H_2||^2 + 1/lambda)),
 * kappa_i = 0.99 rho_i (the PSGLA step of each auxiliary variable). */
pnp_status pnp_stepsizes_poisson(double hnorm, double eta, double rho1, double rho2, double alpha,
                                 double eps, double lip_eps, double c, double* lambda,
                                 double* gamma, double* kappa1, double* kappa2);

/* ------------------------------------------------------------------------
 * Problem: one posterior (Eq. 2 with the Gaussian-deconvolution likelihood)
 * and its chain state, resident on the device.
 * ------------------------------------------------------------------------ */
typedef struct {
    int ny, nx;                 /* image size, one channel                                  */
    const float* y;             /* host [ny*nx]; copied                                     */
    int kh, kw;                 /* blur size, odd                                           */
    const float* h;             /* host [kh*kw]; copied; circular boundary                  */
    double sigma;               /* noise std (> 0)                                          */
    double alpha, eps;          /* prior weight, denoiser level; eps <= 0 -> eps = sigma,
                                   alpha < 0 -> 1 (the paper's Gaussian setting)           */
    double lambda, gamma;       /* <= 0 -> derived by pnp_stepsizes with c = step_c        */
    double step_c;              /* <= 0 -> 0.99                                             */
    double hnorm;               /* ||H||_2; <= 0 -> sum |h| (exact for h >= 0)              */
    int blocks_y, blocks_x;     /* block split (>= 1)                                       */
    int halo;                   /* 0: direct whole-image layers; > 0: block + halo (>= K)  */
    int nchain;                 /* chains sharing y, h (>= 1)                               */
    uint64_t seed;              /* Philox key                                               */
    int burn_in;                /* samples x^(t) with t > burn_in enter the moments         */
    pnp_precision precision;    /* denoiser arithmetic                                      */
    const pnp_denoiser* D;      /* NULL: no prior term                                      */
    const float* x0;            /* host [nchain][ny*nx] or NULL (zeros)                     */
    void* stream;               /* stream for all work of this problem (NULL: own stream)  */
    /* Poisson model (noise_model = PNP_POISSON; sigma is then ignored, eps <= 0 -> 0.05):
     * y holds counts (>= 0); eta, rho1, rho2 > 0; kappa_i <= 0 -> 0.99 rho_i, else in
     * (0, rho_i). z1, z2 start at zero. Zero-initialised descriptors are Gaussian.     */
    pnp_noise_model noise_model;
    double eta, rho1, rho2;
    double kappa1, kappa2;
    /* Inpainting (Sec. IV-A): host [ny*nx], 1 = observed, 0 = missing; copied. H is
     * then diag(mask) (h, kh, kw ignored; hnorm <= 0 -> 1), y is read only where
     * mask = 1, noise_model must be PNP_GAUSSIAN, and x0 is the caller's
     * initialisation (the paper interpolates y). NULL: H is the blur h.            */
    const float* mask;
} pnp_problem_desc;

pnp_status pnp_create_problem(const pnp_problem_desc* desc, pnp_problem** out);
void pnp_destroy_problem(pnp_problem* p);
/* Derived parameters actually used (host). Any pointer may be NULL. */
pnp_status pnp_problem_params(const pnp_problem* p, double* lambda, double* gamma,
                              double* alpha, double* eps);
/* Enqueue n_iters iterations (asynchronous on the problem's stream). Uses a
 * captured CUDA graph of one iteration when use_graph != 0. */
pnp_status pnp_step(pnp_problem* p, int n_iters);
/* Captures and instantiates now the CUDA graphs that later pnp_step calls
 * replay (one and kGraphBatch = 8 iterations, for each state-buffer parity),
 * so that no capture happens inside a caller's timed region. Host work only;
 * needs one earlier pnp_step (its first iteration runs eagerly). PNP_OK and
 * nothing done when graph mode is off. */
pnp_status pnp_prepare_graphs(pnp_problem* p);
/* Run T iterations with the given burn-in (resets nothing) and wait. */
pnp_status pnp_run_chain(pnp_problem* p, int T, int burn_in);
/* Wait for the problem's stream. PNP_ETIMEOUT if a bounded device-side wait
 * (a tensor-core denoiser layer, or the pipelined one-pass update's window
 * copies) ran out since the last synchronising call
 * (pnp_sync, pnp_run_chain, pnp_get_state, pnp_get_moments report it once and
 * clear it; the chain state is then not trustworthy: reset it with
 * pnp_set_state). */
pnp_status pnp_sync(pnp_problem* p);
/* FP64 MMSE and std (want_var = 0) or variance for chain `chain`; host
 * buffers [ny*nx]; n_kept may be NULL. Synchronous. */
pnp_status pnp_get_moments(pnp_problem* p, int chain, double* mmse, double* std_or_var,
                           int64_t* n_kept, int want_var);
/* Chain state: x host [nchain][ny*nx], t = iterations done. Synchronous. */
pnp_status pnp_get_state(pnp_problem* p, float* x, int64_t* t);
pnp_status pnp_set_state(pnp_problem* p, const float* x, int64_t t);
/* Auxiliary variables of a Poisson problem, host [nchain][ny*nx] each (either
 * may be NULL). PNP_EINVAL for a Gaussian problem. Synchronous. */
pnp_status pnp_get_aux_state(pnp_problem* p, float* z1, float* z2);
pnp_status pnp_set_aux_state(pnp_problem* p, const float* z1, const float* z2);
/* Device pointer of the chain state x [nchain][ny][nx] after the iterations
 * enqueued so far (valid until destroy). With a separable blur under Gaussian
 * noise the state alternates between two buffers from one iteration to the
 * next (the fused update reads the current state with a halo while writing the
 * new one), so the pointer changes with every step; call again after stepping. */
float* pnp_problem_x_device(pnp_problem* p);
/* Replay captured CUDA graphs (one of 8 iterations, plus a one-iteration graph
 * for remainders; default on) or launch every kernel eagerly. */
pnp_status pnp_set_graph_mode(int enable);
/* Programmatic dependent launch between the kernels of an iteration (default
 * on): a kernel's prologue (barriers, TMEM, weights) overlaps its
 * predecessor's tail. Changes timings only, never results. */
pnp_status pnp_set_pdl(int enable);
/* Spectral likelihood gradient (default on) for problems created afterwards
 * whose blur is wider than 31 taps, under Gaussian noise, on an image whose
 * sides are powers of two in [64, 4096] (Sec. IV-A's motion blurs): since
 * H^T H is a circular convolution, (H^T H) x = F^-1(|F h|^2 F x) is evaluated
 * by hand-written FP32 FFTs (row FFTs, column FFTs with the product and their
 * inverse, inverse row FFTs fused with the update), with H^T y formed once.
 * Off: the direct wide stencil (r = H x - y, then H^T r). The two agree to
 * FP32 FFT rounding (about 1e-6 of the gradient's scale), not bitwise. */
pnp_status pnp_set_spectral(int enable);

/* ------------------------------------------------------------------------
 * Stencil tile shapes (library tuning; the paper has no counterpart). The
 * H / H^T stencils and the fused update (Eq. 8) run with one of
 * pnp_stencil_tile_count() tile shapes; pnp_create_problem times them all on
 * the new problem's buffers and keeps the fastest for each kernel (cached per
 * image size, kernel size and chain count). Every shape sums each output in
 * the same order, so the choice changes timings, never results.
 * pnp_set_stencil_tile(k) forces shape k for every later stencil launch
 * (operators and problems, all threads); k = -1 restores the per-problem
 * choice. PNP_EINVAL for k outside [-1, count). A blur kernel that is rank
 * one up to FP32 rounding (h = u v^T, |h - u v^T|_F <= 1e-7 |h|_F: Gaussian,
 * uniform) runs as two 1-D passes (kh + kw instead of kh kw FMAs per pixel).
 * pnp_problem_stencil_tiles reports a problem's tile choices and whether it
 * uses the separable form (any pointer may be NULL).
 * ------------------------------------------------------------------------ */
int pnp_stencil_tile_count(void);
pnp_status pnp_set_stencil_tile(int tile);
pnp_status pnp_problem_stencil_tiles(const pnp_problem* p, int* blur_tile, int* update_tile,
                                     int* separable);

/* ------------------------------------------------------------------------
 * Batch: independent problems of different sizes stepped together (all with
 * the same denoiser and precision, FP32 or BF16, halo = 0). One batch iteration = one
 * iteration of every job; the denoiser's tensor-core layers run as one launch
 * per layer over the rows of all jobs, and the iteration is replayed as one
 * CUDA graph. Each job's chain is identical to the same problem run alone
 * (Algorithm 1 applied to each posterior independently).
 * ------------------------------------------------------------------------ */
pnp_status pnp_batch_create(const pnp_problem_desc* descs, int njobs, void* stream,
                            pnp_batch** out);
void pnp_batch_destroy(pnp_batch* b);
/* Enqueue n_iters iterations of every job (asynchronous). */
pnp_status pnp_batch_step(pnp_batch* b, int n_iters);
/* Set every job's burn-in, run T iterations and wait. */
pnp_status pnp_batch_run(pnp_batch* b, int T, int burn_in);
/* Wait for the batch's stream; PNP_ETIMEOUT as for pnp_sync (any job's flag). */
pnp_status pnp_batch_sync(pnp_batch* b);
/* Borrowed handle of job `job` (for pnp_get_moments / pnp_get_state); owned by the batch. */
pnp_status pnp_batch_job(pnp_batch* b, int job, pnp_problem** p);
int pnp_batch_size(const pnp_batch* b);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of sampling jobs. A worker thread admits
 * queued jobs in arrival order while their device footprint (chain state,
 * observation, denoiser scratch) fits hbm_budget_bytes, steps all admitted
 * jobs together with the batch engine, and between rounds of a few
 * iterations retires finished jobs: FP64 MMSE and std maps are copied to host
 * memory and the job's device memory is freed. Jobs that arrive while others
 * run join at the next round. Each job's chain is independent of which other
 * jobs share its steps. All served jobs use the server's denoiser and
 * precision (FP32 or BF16); desc.halo must be 0; desc.stream is ignored. Thread-safe: submit,
 * poll, wait and cancel may be called from any host thread.
 * Job states: 0 queued, 1 running, 2 done, 3 failed, 4 cancelled.
 * ------------------------------------------------------------------------ */
pnp_status pnp_server_create(const pnp_denoiser* D, pnp_precision prec, size_t hbm_budget_bytes,
                             void* stream, pnp_server** out);
/* Copies the job's inputs. PNP_EBUSY if the job alone exceeds the budget. */
pnp_status pnp_server_submit(pnp_server* s, const pnp_problem_desc* desc, int T, int burn_in,
                             int64_t* job_id);
/* State of a job; when done, copies MMSE / std (host [ny*nx], either may be NULL).
 * A round in which a bounded device-side wait ran out fails its jobs (state 3,
 * error PNP_ETIMEOUT). */
pnp_status pnp_server_poll(pnp_server* s, int64_t job_id, double* mmse, double* std, int* state);
/* Wait up to timeout_s seconds for the job to end; PNP_ETIMEOUT if it did not. */
pnp_status pnp_server_wait(pnp_server* s, int64_t job_id, double timeout_s, int* state);
/* Host-side cancellation of a queued or running job; other jobs are unaffected. */
pnp_status pnp_server_cancel(pnp_server* s, int64_t job_id);
/* Seconds since server creation at submission, admission and completion (-1: not yet). */
pnp_status pnp_server_job_times(pnp_server* s, int64_t job_id, double* t_submit, double* t_admit,
                                double* t_done);
pnp_status pnp_server_stats(pnp_server* s, int64_t* pixel_iters, int* active, int* queued,
                            size_t* used_bytes);
/* Device time (seconds) of the work of all rounds so far, measured with CUDA
 * events around each round's launches: the sampling itself, without the
 * admission copies, the retirement read-backs or idle time between arrivals. */
pnp_status pnp_server_device_seconds(pnp_server* s, double* seconds);
/* Scheduling: in each round (between retire/admit points) a job runs
 * iters x min(max_boost, largest active job's pixels / its pixels) iterations
 * (never past its T), so small jobs finish early while large ones keep the
 * batch full. Defaults 8 and 16; max_boost = 1 steps every job equally. */
pnp_status pnp_server_set_round(pnp_server* s, int iters, int max_boost);
void pnp_server_destroy(pnp_server* s);

/* ------------------------------------------------------------------------
 * Instrumentation: CUDA events around every launch of the hot kernels
 * ("blur", "update", "conv_fp32", "conv_tc", "conv_edge" = first layer and the
 * FP32 last layer, "conv_last" = tensor-core last layer, "zupdate" = the
 * auxiliary-variable update of the Poisson model). Enabling resets
 * the counters and forces eager launches (no graph replay). Reading
 * synchronizes the device and returns the summed device time and launches.
 * ------------------------------------------------------------------------ */
pnp_status pnp_kernel_timer(int enable);
/* Number of kernel launches the library has enqueued eagerly since it was
 * loaded (any thread); kernels replayed from a captured CUDA graph are not
 * counted again. */
int64_t pnp_launch_count(void);
pnp_status pnp_kernel_timer_read(const char* name, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* PNP_H */
