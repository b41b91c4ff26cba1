// Internal declarations shared by the CUDA translation units of libpnp.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pnp.h"

namespace pnp {

// Large blur kernels (kh or kw above 31, up to 129: the paper's 65^2-129^2
// motion blurs) run on a wide-window stencil that visits only the nonzero
// taps, in groups of up to four taps on consecutive rows of one window column:
// the group's weights (zero where h is zero) and the window offset of its
// first tap (row * pitch + col, pitch = 128 + kw - 1).
struct alignas(16) WTap {
    float w[4];
    int off;
    int pad[3];
};
constexpr int STENCIL_MAXK = 31;     // template (small-kernel) stencils
constexpr int WIDE_MAXK = 129;
inline bool is_wide(int kh, int kw) { return kh > STENCIL_MAXK || kw > STENCIL_MAXK; }

// Thread-local error message, set by fail().
void set_error(const std::string& msg);
pnp_status fail(pnp_status st, const std::string& msg);
pnp_status cuda_fail(cudaError_t e, const char* what);

#define PNP_CUDA_TRY(expr)                                         \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::pnp::cuda_fail(_e, #expr); \
    } while (0)

#define PNP_TRY(expr)                           \
    do {                                        \
        pnp_status _s = (expr);                 \
        if (_s != PNP_OK) return _s;            \
    } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per device).
int num_sms();

// Optional per-kernel timing with CUDA events (enabled by pnp_kernel_timer;
// eager launches only). No-ops when disabled.
bool timer_enabled();
void timer_begin(int id, cudaStream_t s);
void timer_end(int id, cudaStream_t s);
enum TimerId { T_BLUR = 0, T_UPDATE = 1, T_CONV_FP32 = 2, T_CONV_TC = 3, T_CONV_EDGE = 4, T_CONV_LAST = 5,
               T_ZUPDATE = 6, T_COUNT = 7 };

// Programmatic dependent launch for the kernels of one iteration (stencils,
// tensor-core conv layers): a kernel launched this way may start while its
// predecessor in the stream drains; it runs its prologue (barriers, TMEM,
// constant weights), then waits in griddepcontrol.wait for the predecessor to
// complete before touching any buffer the predecessor reads or writes. Every
// such kernel signals griddepcontrol.launch_dependents only after its own TMEM
// allocation, so a dependent that holds TMEM can never block a predecessor.
bool pdl_enabled();
// Counts kernel launches the library enqueues eagerly (pnp_launch_count);
// launches replayed from a captured graph are not counted again.
void note_launch();
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
    note_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// --------------------------------------------------------------------------
// Valid rectangle of an activation image: positions outside [y0,y1) x [x0,x1)
// are held at zero after every layer (image border of a block-with-halo tile).
// --------------------------------------------------------------------------
struct Rect {
    int y0, y1, x0, x1;
};

// --------------------------------------------------------------------------
// Denoiser parameters on the device.
// --------------------------------------------------------------------------
struct DenoiserDev {
    int K, F;
    double lip;
    // FP32 SIMT layouts, per layer: weights [cin][9][cout] (co fastest), bias [cout]
    float* w32 = nullptr;     // concatenated
    float* b32 = nullptr;
    int64_t* w32_off = nullptr;   // host offsets per layer
    int64_t* b_off = nullptr;
    // BF16 tensor-core layout of the F->F layers: per layer [dx 3][cg 8][dy 3 x co 64][8 ci]
    __nv_bfloat16* wtc = nullptr;
    // last layer (F -> 1): [dx 3][cg 8][16 rows: kernel row dy in row dy][8 ci]
    __nv_bfloat16* wtc_last = nullptr;
    // first layer (1 -> F) on tensor cores: [kc 4][co 64][8], K = 32 holding
    // w_hi (taps 0-8), w_hi, w_lo, b_hi, b_lo (BF16 head/tail split of FP32)
    __nv_bfloat16* wtc_first = nullptr;
    // E4M3 variant: same blobs with 16-channel groups ([dx][4 cg][rows][16 ci]),
    // per-output-channel weight scales (host, [K][64]) and per-layer static
    // activation scales (host; a8_scale[k] = scale of layer k's input)
    uint8_t* wtc8 = nullptr;
    uint8_t* wtc8_last = nullptr;
    float* w8_scale = nullptr;
    float a8_scale[32] = {0};
    bool fp8_calibrated = false;
    float last_bias = 0.f;      // bias of the single output channel of the last layer
    // host copies (FP32, OIHW) for reference / re-packing
    float* hw = nullptr;
    float* hb = nullptr;
    // DDFB form (ddfb = true): K layers of F = P analysis filters (host,
    // [K][P][3][3]), steps gamma_k and the hard-tanh threshold
    bool ddfb = false;
    float* ddfb_w = nullptr;
    float ddfb_gamma[32] = {0};
    float ddfb_ht = 0.f;
};

// Step counter read by the update kernel during graph replay; the update's
// last block to finish advances t (arrive counts the blocks done).
struct StepState {
    uint32_t t;
    int32_t burn_in;
    uint32_t arrive;
};

}  // namespace pnp

struct pnp_denoiser {
    pnp::DenoiserDev dev;
    // device flag set to PNP_ETIMEOUT by a tensor-core layer of pnp_denoise or
    // pnp_denoise_noalloc whose bounded wait ran out (read by pnp_denoise_status)
    int* err = nullptr;
    // cached scratch (activation ping-pong), grown on demand
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int device = 0;
};

namespace pnp {

// Tap groups of h for the forward operator (convolution) or its adjoint
// (correlation): window columns in order, rows ascending within a column.
std::vector<WTap> wide_taps(const float* h, int kh, int kw, bool adjoint);

// ---------------------------------------------------------------- kernels
// Stencils take a tile-shape index (stencil_autotune's choice; -1 = default);
// every shape gives bitwise the same results.
// hsep (optional): separable taps [u | v | u flipped | v flipped] of a rank-one h.
// r = a (h * x) - y per image; y shared (y_img_stride 0) or one plane per image.
// Large kernels (is_wide) take the wide stencil with the forward taps wt (or,
// when wt is NULL, every nonzero entry of the device array h in the same order).
cudaError_t launch_blur(const float* x, const float* y, const float* h, int kh, int kw, int ny,
                        int nx, int nimg, float* r, cudaStream_t s, int tile = -1,
                        const float* hsep = nullptr, float a = 1.0f, int64_t y_img_stride = 0,
                        const WTap* wt = nullptr, int nwt = 0);
cudaError_t launch_blur_adjoint(const float* r, const float* h, int kh, int kw, int ny, int nx,
                                int nimg, float scale, float* g, cudaStream_t s, int tile = -1);
// Arguments of one r = (a (h * x) - y) scale stencil launch (or of its
// adjoint), one entry of a grouped launch.
struct BlurArgs {
    const float* x;
    const float* y;
    const float* h;        // 2-D taps, or the separable taps of a rank-one h
    int kh, ny, nx, nimg;
    float scale;
    int adjoint;
    float* out;
    float a;
    int64_t y_img_stride;
};
int stencil_tile_count();
bool set_forced_stencil_tile(int tile);   // -1 = use each launch's own choice

struct UpdateParams {
    float* x;
    const float* r;
    const float* d;
    const float* h;
    int kh, kw, ny, nx, nchain;
    float inv_s2;       // 1 / sigma^2
    float gamma;
    float c_prior;      // alpha gamma / eps^2 (0 if d == NULL)
    float c_proj;       // gamma / lambda (0 when off)
    float c_noise;      // sqrt(2 gamma) (0 when noise off)
    uint32_t key0, key1;
    uint32_t t;
    const uint32_t* t_dev;     // if non-null, t is read from device memory (graph replay)
    float* mean;
    float* m2;
    float inv_n;        // 1 / n_kept (0: no accumulation)
    const int32_t* burn_dev;   // if non-null: sample number n = t + 1 - *burn_dev,
                               // accumulated when n > 0 (graph replay)
    int d_residual;            // d holds G = x - D(x) instead of D(x)
    uint32_t* arrive;          // if non-null: the last block advances *t_dev (graph replay)
    int tile;                  // stencil tile shape (-1 = default)
    const float* hsep;         // separable taps of a rank-one h (nullptr: 2-D taps)
    const float* z2;           // Poisson: auxiliary z2 [chain][N]; adds -c_z2 (x - z2)
    float c_z2;                // gamma / rho2
    const WTap* wtaps;         // large kernels: adjoint taps (NULL: read h)
    int nwtaps;
    // One-pass gradient (qb != NULL): g = (H^T H) r - qb with r the current
    // state x (read through the stencil window, halo 2 r_h), the separable taps
    // of H^T H in hsep and its size in kh, kw (2 kh_h - 1, 2 kw_h - 1), qb =
    // H^T y [ny][nx]; x+ is written to x_out (not r: neighbouring tiles still
    // read the current state).
    const float* qb;
    float* x_out;
    // One-pass form: os != 0 lets the launch use the pipelined kernel
    // (k_update_os) when the form fits it; err receives 1 if one of that
    // kernel's bounded waits ran out.
    int os = 0;
    int* err = nullptr;
};

// Auxiliary-variable update of the Poisson sampler (k_zupdate).
struct ZParams {
    const float* x;            // new x [chain][N]
    float* z1;                 // [chain][N], updated in place
    float* z2;                 // [chain][N], updated in place
    const float* y;            // counts [N]
    const float* h;
    const float* hsep;
    int kh, kw, ny, nx, nchain;
    float eta;
    float a1, a2;              // kappa_i / rho_i
    float s1, s2;              // sqrt(2 kappa_i)
    float kappa1;
    int noise;
    float* r_out;              // if non-null: eta H x+ - z1+ [chain][N], the next iteration's r
    uint32_t key0, key1;
    uint32_t t;
    const uint32_t* t_dev;
    uint32_t* arrive;          // if non-null: the last block advances *t_dev
    int tile;
};
cudaError_t launch_zupdate(const ZParams& p, cudaStream_t s);
// Grouped launches for batches: the jobs of one call share the stencil width
// (kw, a template parameter of the kernels) and form (separable or 2-D taps);
// each job keeps its own sizes, buffers and step counter, and its outputs are
// the same sums as in its own launch. At most STENCIL_TABLE_MAXJ jobs travel
// by value per launch; more jobs take several launches.
constexpr int STENCIL_TABLE_MAXJ = 48;
cudaError_t launch_blur_group(const BlurArgs* jobs, int n, int kw, bool sep, cudaStream_t s);
cudaError_t launch_update_group(const UpdateParams* jobs, int n, cudaStream_t s);
cudaError_t launch_zupdate_group(const ZParams* jobs, int n, cudaStream_t s);
// Inpainting x-update: p.r is the observation with NaN at missing pixels
// (shared by the chains); no stencil, p.h unused.
cudaError_t launch_update_mask(const UpdateParams& p, cudaStream_t s);
cudaError_t launch_langevin_update(const UpdateParams& p, cudaStream_t s);
// Pipelined one-pass update (k_update_os.cu) with stencil tile shape `tile`:
// cudaErrorNotSupported when p is not of its form (the caller then launches
// the per-tile kernel).
cudaError_t launch_update_os(const UpdateParams& p, int tile, cudaStream_t s);
// Arms the one-shot test fault of the next uncaptured k_update_os launch.
void os_inject_timeout(int cta, int tile_index, long long budget_cycles);
// Spectral gradient of a wide blur (k_spectral.cu): g = F^-1(|H^|^2 F(x)) -
// H^T y for power-of-two images, the spectrum in 4-column panels.
struct SpectralPlan {
    int ny = 0, nx = 0, lgny = 0, lgnx = 0;
    float2* Z = nullptr;     // [nchain] half spectra of the rows (nx / 2 columns), panel layout
    float* P = nullptr;      // |H^|^2 / (2 ny nx) of the half spectrum, panel layout
    float* PN = nullptr;     // the same for the Nyquist column nx / 2, [ny]
    float2* twx = nullptr;   // exp(-2 pi i n / nx)
    float2* twy = nullptr;   // exp(-2 pi i n / ny)
};
// ny, nx powers of two in [64, 4096] and the kernel no larger than the image
bool spectral_eligible(int ny, int nx, int kh, int kw);
// Allocates the plan and computes P from the device kernel h [kh][kw]
// (synchronises s); cudaErrorNotSupported if not eligible.
cudaError_t spectral_setup(const float* h, int kh, int kw, int ny, int nx, int nchain,
                           cudaStream_t s, SpectralPlan** out);
void spectral_free(SpectralPlan* S);
// Z = F^-1-ready spectra P F(x) (row FFTs, then column FFTs, multiply,
// inverse column FFTs) of the nchain planes of x.
cudaError_t spectral_pre(const SpectralPlan& S, const float* x, int nchain, cudaStream_t s);
// Inverse row FFTs and the x-update with g = Re(.) - p.qb, x updated in place.
cudaError_t spectral_update(const SpectralPlan& S, const UpdateParams& p, cudaStream_t s);

// cuTensorMapEncodeTiled from the driver (nullptr if unavailable).
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
PFN_encodeTiled get_encode();
// Times the stencil tile shapes for r = H x - y and for the update `u` (which it
// runs, overwriting u.x / u.mean / u.m2) and returns the fastest of each.
cudaError_t stencil_autotune(const float* x, const float* y, const float* h, const float* hsep,
                             int kh, int kw, int ny, int nx, int nimg, float* r,
                             const UpdateParams& u, cudaStream_t s, int* blur_tile,
                             int* update_tile);
cudaError_t launch_finalize_moments(const float* mean, const float* m2, int64_t npix,
                                    int64_t n_kept, int want_var, double* mmse, double* out2,
                                    cudaStream_t s);

// FP32 SIMT denoiser over a batch of nimg images [nimg][ny][nx]; optional per-image
// valid rects (device, nimg entries) for block-with-halo tiles. scratch must hold
// 2 * nimg * F * ny * nx floats. d = x - G(x).
cudaError_t denoise_fp32(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, float* scratch, cudaStream_t s);
size_t denoise_fp32_scratch(const DenoiserDev& D, int ny, int nx, int nimg);
// DDFB denoiser, direct layout (rects must be NULL); scratch as denoise_fp32.
cudaError_t ddfb_forward(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, float* scratch, cudaStream_t s);

// One job of a tensor-core conv launch: the images of one size that share a
// tensor map (input activations) and an output plane; row_begin/rows place
// the job in the launch's concatenated row stream.
struct TcJob {   // 256 B, 128-B aligned (the tensor map requires it)
    CUtensorMap tin;
    __nv_bfloat16* out;       // F -> F layers: BF16 activations out
    const Rect* rects;
    const float* xin;         // last layer: x (FP32 [img][ny][nx]) ...
    float* dout;              // ... and d = x - G(x) out
    int64_t row_begin;
    int64_t rows;
    int ny, nx, nxp, strips, nimg, pad0, pad1, pad2;
};
int bf16_pad_width(int nx);
cudaError_t tc_make_job(TcJob* J, const void* in, void* out, int ny, int nx, int nimg,
                        const Rect* rects, int64_t row_begin, bool fp8 = false);
// jobs_dev == nullptr: run job0 alone (passed by value); else the device table.
// bias_host: the layer's biases in host memory (passed by value to the kernel).
// last: the F -> 1 layer fused with d = x - G(x) (wblob = last-layer blob).
// fp8: E4M3 operands; scale_host = per-output-channel dequantisation scales,
// inv_out = 1 / scale of the output activations.
cudaError_t tc_launch(const TcJob& job0, const TcJob* jobs_dev, int njobs, int64_t total_rows,
                      const void* wblob, const float* bias_host, int* err, bool last,
                      cudaStream_t s, bool fp8 = false, const float* scale_host = nullptr,
                      float inv_out = 1.f);
cudaError_t first_layer_bf16(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                             const Rect* rects, __nv_bfloat16* out, int* err, cudaStream_t s);
// First layer over several image stacks in one launch (a by-value table of up
// to FIRST_MAXJ jobs per launch): x, out, rects, ny, nx, nimg set by the
// caller; nxp, nsx and seg_begin are filled by the launcher.
struct FirstJob {
    const float* x;
    void* out;
    const Rect* rects;
    int ny, nx, nxp, nimg;
    uint32_t seg_begin, nsx;
};
constexpr int FIRST_MAXJ = 64;
struct FirstTable {
    FirstJob j[FIRST_MAXJ];
    int n;
    uint32_t nseg;
};
cudaError_t first_layer_bf16_jobs(const DenoiserDev& D, const FirstJob* jobs, int njobs, int* err,
                                  cudaStream_t s);
cudaError_t last_layer_bf16(const DenoiserDev& D, const __nv_bfloat16* act, const float* x,
                            int ny, int nx, int nimg, float* d, int* err, cudaStream_t s);

// BF16 tcgen05 denoiser (F = 64). scratch must hold denoise_bf16_scratch() bytes.
// residual = true: write G = x - D(x) instead of d = D(x) (the chain's update
// takes either; the tensor-core last layer then reads no x).
// err: device flag that a layer whose bounded wait ran out sets to PNP_ETIMEOUT
// (nullptr: an int right after the two activation planes in scratch).
cudaError_t denoise_bf16(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, void* scratch, cudaStream_t s,
                         bool residual = false, int* err = nullptr);
size_t denoise_bf16_scratch(const DenoiserDev& D, int ny, int nx, int nimg);
cudaError_t denoise_fp8(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                        const Rect* rects, float* d, void* scratch, cudaStream_t s,
                        bool residual = false, int* err = nullptr);
// Arms a one-shot fault for the next F -> F tensor-core launch that is not
// being captured: CTA `cta` skips its load number `load_index`, and every wait
// of that launch gives up after budget_cycles (pnp_debug_inject_tc_timeout).
void tc_inject_timeout(int cta, int load_index, long long budget_cycles);
// Reads the device timeout flag (after waiting for stream s) and clears it:
// PNP_ETIMEOUT with a message naming `who` if it was set, else PNP_OK.
pnp_status take_timeout(int* flag, cudaStream_t s, const char* who);
// Resolves the allocation-free entry point's fixed scratch area on the
// current device (which reserves it); idempotent.
pnp_status noalloc_reserve();
size_t denoise_fp8_scratch(const DenoiserDev& D, int ny, int nx, int nimg);
// FP32 denoiser that also records the largest activation of every layer's
// output (amax_dev[k], k < K-1; activations are >= 0 after ReLU).
cudaError_t denoise_fp32_amax(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                              float* d, float* scratch, unsigned* amax_dev, cudaStream_t s);
cudaError_t convert_e4m3(const float* src, uint8_t* dst, size_t n, cudaStream_t s);

// Block-with-halo gather / scatter (Sec. II-B2 receptive-field variant).
struct BlockDesc {
    int img;        // source image index
    int r0, r1;     // interior rows  [r0, r1)
    int c0, c1;     // interior cols  [c0, c1)
};
cudaError_t launch_gather_blocks(const float* x, int ny, int nx, const BlockDesc* blocks,
                                 int nblocks, int halo, int ty, int tx, float* tiles,
                                 Rect* rects, cudaStream_t s);
cudaError_t launch_scatter_blocks(const float* dtiles, int ny, int nx, const BlockDesc* blocks,
                                  int nblocks, int halo, int ty, int tx, float* d,
                                  cudaStream_t s);

}  // namespace pnp

// A problem's device state (one posterior, nchain chains). Defined here so
// the batch and serving engines can drive problems directly.
struct pnp_problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int ny = 0, nx = 0, nchain = 1, kh = 0, kw = 0;
    int64_t N = 0;
    float* y = nullptr;
    float* h = nullptr;
    // current chain state; with the one-pass gradient the state alternates
    // between xb[0] and xb[1] (x = xb[par] at the point of the stream where the
    // next enqueued iteration starts), otherwise xb[0] = xb[1] = x
    float* x = nullptr;
    float* xb[2] = {nullptr, nullptr};
    int par = 0;
    float* r = nullptr;
    float* d = nullptr;
    float* mean = nullptr;
    float* m2 = nullptr;
    double sigma = 0, alpha = 0, eps = 0, lambda = 0, gamma = 0, hnorm = 0;
    uint64_t seed = 0;
    int burn_in = 0;
    pnp_precision prec = PNP_FP32;
    const pnp_denoiser* D = nullptr;
    int by = 1, bx = 1, halo = 0;
    // block + halo mode
    pnp::BlockDesc* blocks = nullptr;
    int nblocks = 0, ty = 0, tx = 0;
    float* tiles = nullptr;
    float* dtiles = nullptr;
    pnp::Rect* rects = nullptr;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    pnp::StepState* st = nullptr;
    int64_t t = 0;
    int blur_tile = -1, update_tile = -1;   // autotuned stencil tile shapes
    // Poisson model (AXDA + PSGLA): z1 ~ eta H x, z2 ~ x, [chain][N] each
    bool poisson = false;
    double eta = 0, rho1 = 0, rho2 = 0, kappa1 = 0, kappa2 = 0;
    float* z1 = nullptr;
    float* z2 = nullptr;
    // inpainting (H = diag(mask)): y holds NaN at missing pixels, no blur
    bool inpaint = false;
    float* hsep = nullptr;                  // separable taps when h is rank one
    pnp::WTap* wt_fwd = nullptr;            // large kernels: forward / adjoint taps
    pnp::WTap* wt_adj = nullptr;
    int nwt = 0;
    // one-pass gradient g = (H^T H) x - H^T y of a separable blur (Gaussian
    // noise, 2 kh - 1 and 2 kw - 1 <= 31): qb = H^T y, qsep = the separable
    // taps of H^T H; the residual r is then not formed and xb[1] reuses its plane
    bool fused = false;
    float* qb = nullptr;
    float* qsep = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};         // one iteration, per start parity
    cudaGraphExec_t graph_batch[2] = {nullptr, nullptr};   // kGraphBatch iterations
    bool eager_done = false;                 // one eager iteration ran (lazy kernel setup)
    int* err = nullptr;                      // device timeout flag of the tensor-core layers
    // spectral gradient of a wide blur (Gaussian noise, power-of-two image):
    // no residual plane, qb = H^T y, x updated in place
    pnp::SpectralPlan* sp = nullptr;
};

namespace pnp {
constexpr int kGraphBatch = 8;   // iterations per replayed graph
// The two halves of one iteration around the denoiser: r = H x - y, and the
// fused update (+ step counter advance).
pnp_status problem_pre(pnp_problem* p, cudaStream_t s);
pnp_status problem_post(pnp_problem* p, cudaStream_t s);
// Arguments of the problem's update (and Poisson z-update) launches for the
// iteration that starts from its current state buffer.
pnp_status problem_update_params(const pnp_problem* p, UpdateParams& u);
ZParams problem_z_params(const pnp_problem* p);
// Advances the host-side state buffer after an iteration has been enqueued
// (problem_post does it; graph replays do it for the iterations they hold).
inline void problem_flip(pnp_problem* p) {
    p->par ^= 1;
    p->x = p->xb[p->par];
}
}  // namespace pnp

namespace pnp {
// Device job tables of a batch step: [F->F A->B][F->F B->A][last], one entry per job.
struct BatchPlan {
    TcJob* tables = nullptr;
    size_t cap = 0;
    int n = 0;
    int64_t total_rows = 0;
    bool bf16 = false;
    int* err = nullptr;
    static size_t table_bytes(int n);
};
pnp_status plan_build(BatchPlan& plan, const std::vector<pnp_problem*>& jobs, cudaStream_t s);
void plan_free(BatchPlan& plan);
// One iteration of every job (all share denoiser and precision).
pnp_status plan_enqueue_step(const BatchPlan& plan, const std::vector<pnp_problem*>& jobs,
                             cudaStream_t s);
}  // namespace pnp
