// BF16 denoiser: the F -> F 3x3 layers as an implicit GEMM on tcgen05 tensor
// cores, the 1 -> F and F -> 1 layers on CUDA cores (Sec. II-B, Eqs. 5-6,
// Example 1: D = Id - G, ReLU on all layers but the last).
//
// Activation layout ("channel-group planar"): act[img][y][cg][xp][8] BF16,
// cg = channel / 8, xp over the width padded to a multiple of 8 (padding
// columns hold zeros). One TMA box per input row - 8 channel groups x 144
// pixels (the 128-pixel output segment plus 8 on each side) - lands in shared
// memory exactly in the UMMA no-swizzle K-major layout: a core matrix is 8
// consecutive pixels x 8 channels = 128 contiguous bytes, consecutive pixel
// octets are 128 B apart (SBO) and consecutive channel groups 2304 B apart
// (LBO). A tap shift dx is then a 16-byte offset of the descriptor start
// address and a tap shift dy selects another row slot, so each input row is
// fetched from HBM/L2 once per 128-pixel column strip.
//
// The GEMM is organised around input rows: input row i at column shift dx
// (M = 128 pixels, K = 16 channels per MMA) is multiplied by the stacked
// weights [W(dy=0,dx); W(dy=1,dx); W(dy=2,dx)] (N = 3 x 64): 12 MMAs of
// 128 x 192 x 16 give P_i = (P_i^0, P_i^1, P_i^2), the row's contributions to
// output rows i+1, i and i-1. (A 128 x 64 x 16 MMA runs at only ~60 % of the
// tensor rate; N = 192 runs at the full rate.) P_i goes to one of two fixed,
// non-overlapping 192-column TMEM regions (alternating per input row: MMAs
// whose accumulator ranges partially overlap the previous row's run ~40 %
// slower). The epilogue sums output row r = P_{r-1}^0 + P_r^1 + P_{r+1}^2 in
// registers, two partial rows at a time. Warp roles: warp 0 = TMA producer,
// warp 1 = MMA issuer, warps 2-5 = epilogue (TMEM -> registers, sum, bias,
// ReLU, zero outside the valid rect, BF16, global store); the epilogue makes
// two TMEM round trips per input row with 64-column loads (a load and wait
// per 16 columns left the epilogue, not the tensor core, setting the pace).
// Input rows circulate through an 8-slot shared-memory ring. The last layer
// (one output channel) drains four input rows per wait, with a 12-slot ring
// and eight 32-column TMEM regions.
//
// One launch covers a table of jobs (images of possibly different sizes,
// each with its own tensor map): every CTA walks a contiguous range of the
// concatenated (job, image, strip, row) stream, so the work of all jobs is
// balanced across the SMs to within one row.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda_fp8.h>

#include "pdl.cuh"
#include "pnp_internal.h"
#include "tc_ptx.cuh"

namespace pnp {

// Two FP32 values -> packed BF16x2 (lo in the low half) with ReLU applied by
// the conversion itself (cvt.rn.relu: negative results become +0).
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Four FP32 values -> packed E4M3 (a in the lowest byte), saturating to the
// finite range, with ReLU applied by the conversion.
__device__ __forceinline__ uint32_t pack_e4m3x4_relu(float a, float b, float c, float d) {
    unsigned short lo, hi;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;\n" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;\n" : "=h"(hi) : "f"(d), "f"(c));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

namespace tc {
constexpr int F = 64;
constexpr int SEG = 128;                    // output pixels per row segment (UMMA M)
constexpr int HALO_PX = 8;                  // smem row starts 8 px left of the segment
constexpr int ROW_PX = SEG + 2 * HALO_PX;   // 144
constexpr int CG_BYTES = ROW_PX * 16;       // 2304: one channel-group plane of a row
constexpr int ROW_BYTES = 8 * CG_BYTES;     // 18432
constexpr int TMEM_COLS = 512;              // allocation (power of two >= 2 x 192)
constexpr int NB = 3 * F;                   // stacked rows of one column shift (dy, co)
constexpr int DX_W_BYTES = 8 * NB * 16;     // 24576: [cg][dy*64+co][8 ci] of one dx
constexpr int W_BYTES = 3 * DX_W_BYTES;     // 73728
constexpr uint32_t IDESC192 = ptx::idesc_bf16_f32(SEG, 192);
constexpr long long BUDGET = 4000000000LL;        // ~2 s of SM clock per wait
// descriptor words (no swizzle, K-major): low = start>>4 | (LBO>>4)<<16,
// high = SBO>>4 | version bit 46
constexpr uint32_t A_LBO_FIELD = (uint32_t)(CG_BYTES >> 4) << 16;
constexpr uint32_t B_LBO_FIELD = (uint32_t)((NB * 16) >> 4) << 16;
constexpr uint32_t DESC_HI = (128u >> 4) | (1u << 14);
}  // namespace tc

static_assert(sizeof(TcJob) == 256 && alignof(TcJob) == 128, "TcJob layout");

// F -> F layers (LAST = false): N = 3 x 64, kernel row dy in columns
// [64 dy, 64 dy + 64). Last layer (LAST = true): its single output channel for
// kernel rows dy = 0, 1, 2 in B rows 0, 1, 2 of one 16-row block (N = 16).
// BF16 (FP8 = false): 8 channel groups of 8 per pixel, K = 16 per MMA.
// E4M3 (FP8 = true): 4 channel groups of 16, K = 32 per MMA (kind::f8f6f4);
// the shared-memory geometry (16-byte core-matrix rows, 2304-byte planes) is
// the same, with half the planes.
template <bool LAST, bool FP8>
struct TcMode {
    static constexpr int NROW = LAST ? 1 : 64;
    static constexpr int NB = LAST ? 16 : 3 * NROW;
    static constexpr int NCG = FP8 ? 4 : 8;             // 16-byte channel-group planes
    static constexpr int KK = NCG / 2;                  // MMAs per column shift
    static constexpr int ROWB = NCG * tc::CG_BYTES;     // bytes of one input row in smem
    static constexpr int DX_W = NCG * NB * 16;
    static constexpr int WB = 3 * DX_W;
    static constexpr uint32_t IDESC = FP8 ? ptx::idesc_e4m3_f32(tc::SEG, NB)
                                          : ptx::idesc_bf16_f32(tc::SEG, NB);
    static constexpr uint32_t B_LBO = (uint32_t)((NB * 16) >> 4) << 16;
    // pipeline depth: input-row ring slots and TMEM accumulator regions. The
    // F -> F layers hold 72 KB of weights and 2 x 192 TMEM columns; the last
    // layer's 6 KB of weights and 16-column regions leave room for a deeper
    // ring and 8 regions, so its MMAs run further ahead of its epilogue.
    static constexpr int NS = LAST ? 12 : 8;
    static constexpr int NACC = LAST ? 8 : 2;
    static constexpr int RSTRIDE = LAST ? 32 : NB;   // TMEM columns between regions
    // epilogue warps, one per TMEM lane quadrant
    static constexpr int EPI_WARPS = 4;
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    static constexpr int OFF_W = NS * tc::ROW_BYTES;
    static constexpr int OFF_BAR = OFF_W + WB;
    static constexpr int NBAR = 2 * NS + 1 + 2 * NACC + 1;   // full, empty, weights, tfull, tempty, drain
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr int SMEM = OFF_MISC + 16 + 1024;        // + alignment slack
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(NACC * RSTRIDE <= tc::TMEM_COLS, "TMEM regions");
};

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

struct TcCommon {
    const void* wblob;            // [3 dx][cg][3 dy x 64 co][16 B of input channels]
    float bias[64];               // by value: constant-bank operands in the epilogue
    float scale[64];              // E4M3: dequantisation scale per output channel
    float inv_out;                // E4M3: 1 / scale of the output activations
    int* err;
    const TcJob* jobs;            // device table, or nullptr: the single job parameter
    int njobs;
    int64_t total_rows;
    long long budget;             // clock cycles a wait may last before the CTA gives up
    int skip_cta, skip_load;      // fault injection: CTA skip_cta never issues its load
                                  // number skip_load (skip_cta < 0: off)
};

// Position in the concatenated row stream of a launch.
struct RowPos {
    const TcJob* J;
    int img, strip, y, len;
};

__device__ __forceinline__ const TcJob* job_at(const TcJob& job0, const TcCommon& c, int j) {
    return c.jobs ? c.jobs + j : &job0;
}

// Advance job index j to the job holding global row g and decompose g.
__device__ __forceinline__ RowPos locate(const TcJob& job0, const TcCommon& c, int& j, int64_t g,
                                         int64_t g_end) {
    const TcJob* J = job_at(job0, c, j);
    while (g >= J->row_begin + J->rows && j + 1 < c.njobs) J = job_at(job0, c, ++j);
    const int64_t local = g - J->row_begin;
    const int64_t q = local / J->ny;
    RowPos p;
    p.J = J;
    p.y = (int)(local - q * J->ny);
    p.strip = (int)(q % J->strips);
    p.img = (int)(q / J->strips);
    p.len = (int)imin64(imin64(g_end, J->row_begin + J->rows) - g, (int64_t)J->ny - p.y);
    return p;
}

// D[tmem] (+)= A * B with both descriptors given by their low words (the
// high words are the same constant).
template <bool FP8>
__device__ __forceinline__ void mma_lo(uint32_t d_tmem, uint32_t a_lo, uint32_t b_lo,
                                       uint32_t idesc, uint32_t accumulate) {
    if constexpr (FP8) {
        asm volatile(
            "{\n.reg .b64 da, db;\n.reg .pred p;\n"
            "mov.b64 da, {%1, %2};\n"
            "mov.b64 db, {%3, %2};\n"
            "setp.ne.b32 p, %5, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], da, db, %4, p;\n}\n" ::"r"(d_tmem),
            "r"(a_lo), "r"(tc::DESC_HI), "r"(b_lo), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n.reg .b64 da, db;\n.reg .pred p;\n"
            "mov.b64 da, {%1, %2};\n"
            "mov.b64 db, {%3, %2};\n"
            "setp.ne.b32 p, %5, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n}\n" ::"r"(d_tmem),
            "r"(a_lo), "r"(tc::DESC_HI), "r"(b_lo), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Epilogue helpers. TMEM column block `col` (64 columns) of this warp's lanes.
__device__ __forceinline__ void tm_add64(uint32_t taddr, float* acc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t t[16];
        ptx::tmem_ld_32x32b_x16(taddr + q * 16, t);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[q * 16 + e] += __uint_as_float(t[e]);
    }
}
__device__ __forceinline__ void tm_load64(uint32_t taddr, float* acc) {
    uint32_t t[64];
    ptx::tmem_ld_32x32b_x64(taddr, t);
    ptx::tmem_ld_wait();
#pragma unroll
    for (int e = 0; e < 64; ++e) acc[e] = __uint_as_float(t[e]);
}

template <bool LAST, bool FP8>
__global__ void __launch_bounds__(TcMode<LAST, FP8>::THREADS, 1)
    k_conv_tc(const __grid_constant__ TcJob job0, const __grid_constant__ TcCommon c) {
    using namespace tc;
    using Mode = TcMode<LAST, FP8>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int NS = Mode::NS, NACC = Mode::NACC;
    uint8_t* ring = smem;
    uint8_t* wsm = smem + Mode::OFF_W;
    uint64_t* bars = (uint64_t*)(smem + Mode::OFF_BAR);
    uint64_t* full = bars;
    uint64_t* empty = bars + NS;
    uint64_t* wbar = bars + 2 * NS;
    uint64_t* tfull = bars + 2 * NS + 1;
    uint64_t* tempty = tfull + NACC;
    uint64_t* drain = tempty + NACC;
    uint32_t* tmem_slot = (uint32_t*)(smem + Mode::OFF_MISC);
    volatile int* abort_flag = (volatile int*)(smem + Mode::OFF_MISC + 4);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            ptx::mbar_init(&full[i], 1);
            ptx::mbar_init(&empty[i], 1);
        }
        ptx::mbar_init(wbar, 1);
        for (int i = 0; i < NACC; ++i) {
            ptx::mbar_init(&tfull[i], 1);
            ptx::mbar_init(&tempty[i], Mode::EPI_WARPS);
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        // the layer's weights are constant: fetched before the predecessor finishes
        ptx::mbar_arrive_expect_tx(wbar, Mode::WB);
        for (int t = 0; t < 3; ++t)
            ptx::bulk_load(wsm + t * Mode::DX_W, (const uint8_t*)c.wblob + t * Mode::DX_W,
                           Mode::DX_W, wbar);
    }
    if (warp == 0 && lane == 0 && !c.jobs) ptx::prefetch_tensormap(&job0.tin);
    if (warp == 2) {
        ptx::tmem_alloc(tmem_slot, TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_launch_dependents();   // after this CTA's TMEM allocation
    pdl_wait();                // the predecessor's output is this layer's input

    // this CTA's share of the concatenated row stream
    const int64_t g_begin = c.total_rows * blockIdx.x / gridDim.x;
    const int64_t g_end = c.total_rows * (blockIdx.x + 1) / gridDim.x;
    const long long budget = c.budget;
    // loads issued by the producer and the one it skipped (fault injection),
    // read again when unwinding after an abort
    uint32_t loads = 0, skipped = 0xffffffffu;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            uint32_t L = 0;
            bool ok = true;
            int j = 0;
            const uint32_t skip_at =
                (int)blockIdx.x == c.skip_cta ? (uint32_t)c.skip_load : 0xffffffffu;
            for (int64_t g = g_begin; g < g_end && ok;) {
                const RowPos p = locate(job0, c, j, g, g_end);
                for (int r = p.y - 1; r <= p.y + p.len && ok; ++r, ++L) {
                    const uint32_t slot = L % NS, u = L / NS;
                    if (!ptx::mbar_wait(&empty[slot], (u & 1) ^ 1, abort_flag, budget)) { ok = false; break; }
                    if (L == skip_at) {   // nothing is issued or expected for this row
                        skipped = L;
                        continue;
                    }
                    ptx::mbar_arrive_expect_tx(&full[slot], Mode::ROWB);
                    ptx::tma_load_5d(ring + slot * ROW_BYTES, &p.J->tin, &full[slot], 0,
                                     p.strip * (SEG / 8) - HALO_PX / 8, 0, r, p.img);
                }
                g += p.len;
            }
            loads = L;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: 12 MMAs (N = 192) per input row
            bool ok = ptx::mbar_wait(wbar, 0, abort_flag, budget);
            const bool w_landed = ok;
            const uint32_t ring_lo = (ptx::smem_u32(ring) >> 4) | A_LBO_FIELD;
            const uint32_t w_lo = (ptx::smem_u32(wsm) >> 4) | Mode::B_LBO;
            uint32_t L = 0;
            bool issued = false;
            int j = 0;
            for (int64_t g = g_begin; g < g_end && ok;) {
                const RowPos p = locate(job0, c, j, g, g_end);
                for (int ri = -1; ri <= p.len && ok; ++ri, ++L) {
                    const uint32_t reg = L % NACC, u = L / NACC;
                    ok = ptx::mbar_wait(&full[L % NS], (L / NS) & 1, abort_flag, budget);
                    if (ok) ok = ptx::mbar_wait(&tempty[reg], (u & 1) ^ 1, abort_flag, budget);
                    if (!ok) break;
                    ptx::tc_fence_after();
                    const uint32_t a_row = ring_lo + (L % NS) * (ROW_BYTES >> 4);
                    const uint32_t d = tmem_base + reg * Mode::RSTRIDE;
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                        for (int kk = 0; kk < Mode::KK; ++kk)
                            mma_lo<FP8>(d, a_row + kk * 2 * (CG_BYTES >> 4) + (HALO_PX - 1 + dx),
                                   w_lo + dx * (Mode::DX_W >> 4) + kk * 2 * (Mode::NB * 16 >> 4),
                                   Mode::IDESC, (dx | kk) != 0);
                    issued = true;
                    ptx::mma_commit(&empty[L % NS]);   // input row consumed
                    ptx::mma_commit(&tfull[reg]);      // P_i ready
                }
                g += p.len;
            }
            // every MMA of this thread completes before TMEM is released, and the
            // weight copy lands before the CTA exits, also after an abort
            if (issued) {
                ptx::mma_commit(drain);
                ptx::mbar_wait_drain(drain, 0, budget);
            }
            if (!w_landed) ptx::mbar_wait_drain(wbar, 0, budget);
        }
    } else if constexpr (LAST) {
        // ---------------- epilogue of the last layer: warps 2..5 own TMEM lane
        // quadrants 2,3,0,1. Output row r = P_{r-1}[col 0] + P_r[col 1] +
        // P_{r+1}[col 2] (+ bias): G, or d = x - G when x is given. Input rows
        // are drained four at a time: four TMEM loads, one wait.
        const int quad = warp & 3;
        const int jx = quad * 32 + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
        uint32_t L = 0;
        bool ok = true;
        int j = 0;
        float X0 = 0.f, X1 = 0.f;
        for (int64_t g = g_begin; g < g_end && ok;) {
            const RowPos p = locate(job0, c, j, g, g_end);
            const TcJob* J = p.J;
            const int x = p.strip * SEG + jx;
            const bool in_img = x < J->nx;
            const int64_t plane = (int64_t)J->ny * J->nx;
            const float* xin = J->xin ? J->xin + p.img * plane : nullptr;
            float* dout = J->dout + p.img * plane;
            auto step = [&](float& Xprev, float& Xcur, int ri, const uint32_t* pr, float xv) {
                if (ri >= 1) {
                    Xprev += __uint_as_float(pr[2]);
                    const float G = FP8 ? fmaf(Xprev, c.scale[0], c.bias[0]) : Xprev + c.bias[0];
                    // d = x - G, or the residual G itself when no x is given
                    if (in_img) dout[(int64_t)(p.y + ri - 1) * J->nx + x] = xin ? xv - G : G;
                }
                if (ri >= 0 && ri < p.len) Xcur += __uint_as_float(pr[1]);
                if (ri + 1 < p.len) Xprev = __uint_as_float(pr[0]);
            };
            // chunks of 4 input rows starting at ri0 = -1, 3, 7, ...: the row
            // parity of chunk member k is that of k
            for (int ri0 = -1; ri0 <= p.len && ok; ri0 += 4) {
                const int nb = min(4, p.len + 1 - ri0);
                float xv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int ri = ri0 + k;
                    xv[k] = (k < nb && xin && ri >= 1 && in_img)
                                ? __ldg(xin + (int64_t)(p.y + ri - 1) * J->nx + x) : 0.f;
                }
                bool w = true;
                for (int k = 0; k < nb && w; ++k) {
                    const uint32_t Lk = L + k;
                    w = ptx::mbar_wait(&tfull[Lk % NACC], (Lk / NACC) & 1, abort_flag, budget);
                }
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                ptx::tc_fence_after();
                uint32_t pr[4][4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < nb) ptx::tmem_ld_32x32b_x4(lane_base + ((L + k) % NACC) * Mode::RSTRIDE, pr[k]);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < 4; ++k) ptx::tie_regs4(pr[k]);
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    for (int k = 0; k < nb; ++k) ptx::mbar_arrive(&tempty[(L + k) % NACC]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k >= nb) break;
                    // output row q lives in X[q & 1]: prev = X[(ri-1) & 1], cur = X[ri & 1]
                    if (k & 1) step(X1, X0, ri0 + k, pr[k], xv[k]);
                    else step(X0, X1, ri0 + k, pr[k], xv[k]);
                }
                L += nb;
            }
            g += p.len;
        }
    } else {
        // ---------------- epilogue of an F -> F layer: warps 2..5 own TMEM lane
        // quadrants 2,3,0,1. Per input row two TMEM round trips: P^2 (completes
        // output row ri - 1, stored), then P^1 and P^0 together (P^0 straight
        // into the registers the stored row freed).
        const int quad = warp & 3;
        const int jx = quad * 32 + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
        uint32_t L = 0;
        bool ok = true;
        int j = 0;
        // partial sums of the output rows of even / odd index, FP32 bit patterns
        // (TMEM loads write them directly)
        uint32_t X0[64], X1[64];
        for (int64_t g = g_begin; g < g_end && ok;) {
            const RowPos p = locate(job0, c, j, g, g_end);
            const TcJob* J = p.J;
            const Rect rc = J->rects ? J->rects[p.img] : Rect{0, J->ny, 0, J->nx};
            const int x = p.strip * SEG + jx;
            const int nxp = J->nxp;
            const bool col_ok = x < nxp;
            const bool x_valid = x < J->nx && x >= rc.x0 && x < rc.x1;
            auto store_row = [&](const uint32_t* accb, int yy) {
                auto acc = [&](int k) { return __uint_as_float(accb[k]); };
                if (!col_ok) return;
                const bool valid = x_valid && yy >= rc.y0 && yy < rc.y1;
                if constexpr (FP8) {
                    // E4M3 activations: [img][y][4 cg][xp][16]
                    uint8_t* o = reinterpret_cast<uint8_t*>(J->out) +
                                 (((int64_t)p.img * J->ny + yy) * 4 * nxp + x) * 16;
                    if (!valid) {
                        // zero outside the valid rect
#pragma unroll
                        for (int cg = 0; cg < 4; ++cg)
                            *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 16) = make_uint4(0u, 0u, 0u, 0u);
                        return;
                    }
#pragma unroll
                    for (int cg = 0; cg < 4; ++cg) {
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float v[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const int ch = cg * 16 + 4 * e + h;
                                // relu(t) s = relu(t s) for the scale s > 0: the
                                // conversion applies the ReLU
                                v[h] = fmaf(acc(ch), c.scale[ch], c.bias[ch]) * c.inv_out;
                            }
                            pk[e] = pack_e4m3x4_relu(v[0], v[1], v[2], v[3]);
                        }
                        *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                } else {
                    // BF16 activations: [img][y][8 cg][xp][8]
                    __nv_bfloat16* o = J->out + ((((int64_t)p.img * J->ny + yy) * 8) * nxp + x) * 8;
                    if (!valid) {
                        // zero outside the valid rect
#pragma unroll
                        for (int cg = 0; cg < 8; ++cg)
                            *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 8) = make_uint4(0u, 0u, 0u, 0u);
                        return;
                    }
#pragma unroll
                    for (int cg = 0; cg < 8; ++cg) {
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c0 = cg * 8 + 2 * e;
                            pk[e] = pack_bf16_relu(acc(c0) + c.bias[c0], acc(c0 + 1) + c.bias[c0 + 1]);
                        }
                        *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                }
            };
            // input row ri adds P^2 to output row ri-1 (then complete), P^1 to
            // output row ri, and starts output row ri+1 with P^0
            auto step = [&](uint32_t* Xprev, uint32_t* Xcur, int ri, uint32_t taddr) {
                uint32_t t[64];
                if (ri >= 1) {
                    ptx::tmem_ld_32x32b_x64(taddr + 2 * F, t);
                    ptx::tmem_ld_wait();
                    ptx::tie_regs32(t);
                    ptx::tie_regs32(t + 32);
#pragma unroll
                    for (int e = 0; e < 64; ++e)
                        Xprev[e] = __float_as_uint(__uint_as_float(Xprev[e]) + __uint_as_float(t[e]));
                    store_row(Xprev, p.y + ri - 1);
                }
                // both loads unconditional (conditional asm outputs into the
                // register arrays would force them to memory): P^1 is added only
                // when row ri exists, and Xprev holds no live data any more -
                // it was stored above, or belongs to a row before the image
                const bool s1 = ri >= 0 && ri < p.len;
                ptx::tmem_ld_32x32b_x64(taddr + F, t);
                ptx::tmem_ld_32x32b_x64(taddr, Xprev);
                ptx::tmem_ld_wait();
                ptx::tie_regs32(t);
                ptx::tie_regs32(t + 32);
                ptx::tie_regs32(Xprev);
                ptx::tie_regs32(Xprev + 32);
                if (s1) {
#pragma unroll
                    for (int e = 0; e < 64; ++e)
                        Xcur[e] = __float_as_uint(__uint_as_float(Xcur[e]) + __uint_as_float(t[e]));
                }
            };
            for (int ri = -1; ri <= p.len; ++ri, ++L) {
                const uint32_t reg = L % NACC, u = L / NACC;
                if (!__all_sync(0xffffffffu, ptx::mbar_wait(&tfull[reg], u & 1, abort_flag, budget))) { ok = false; break; }
                ptx::tc_fence_after();
                const uint32_t taddr = lane_base + reg * Mode::RSTRIDE;
                // output row q lives in X[q & 1]: prev = X[(ri-1) & 1], cur = X[ri & 1]
                if ((ri + 1) & 1) step(X1, X0, ri, taddr);
                else step(X0, X1, ri, taddr);
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[reg]);
            }
            g += p.len;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    // after an abort the producer waits for its loads still in flight (the
    // last NS issued; older ones were consumed before their slot was reused)
    if (warp == 0 && lane == 0 && *abort_flag) {
        for (uint32_t k = loads > (uint32_t)NS ? loads - NS : 0; k < loads; ++k)
            if (k != skipped) ptx::mbar_wait_drain(&full[k % NS], (k / NS) & 1, budget);
    }
    if (warp == 2) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, TMEM_COLS);
    }
    if (threadIdx.x == 0 && *abort_flag && c.err) atomicExch(c.err, (int)PNP_ETIMEOUT);
}

// ---------------------------------------------------------------------------
// First layer 1 -> 64 on the tensor cores. Persistent CTAs of 128 threads walk
// the image's 128-pixel row segments; for each, every thread gathers its
// pixel's 3 x 3 taps of the FP32 image (zero outside it) into one row of A
// (M = 128 pixels, K = 32), one thread issues two 128 x 64 x 16 MMAs into one
// of two 64-column TMEM buffers, and the four warps read their 32 lanes back,
// apply ReLU and the valid-rect mask and store 64 channels per pixel (BF16
// planes, or E4M3 scaled by inv_out). The loop is software-pipelined: the
// taps of segment k + 1 are loaded while the epilogue of segment k - 1 runs
// and the MMAs of segment k are in flight.
//
// BF16 operands would round the FP32 image and weights to 8 bits; instead each
// is split into a BF16 head and a BF16 tail (v = hi + lo, |lo| <= 2^-9 |v|)
// and K carries x_hi w_hi + x_lo w_hi + x_hi w_lo + b_hi + b_lo (the dropped
// x_lo w_lo is below 2^-17 of each product), accumulated in FP32:
//   A row (pixel)  : [x_hi(9) | x_lo(9) | x_hi(9) | 1 | 1 | 0 0 0]
//   B row (channel): [w_hi(9) | w_hi(9) | w_lo(9) | b_hi | b_lo | 0 0 0]
// Operands in the no-swizzle K-major layout: A [kc 4][pixel 128][8] (LBO
// 2048 B, SBO 128 B), B [kc 4][channel 64][8] (LBO 1024 B, SBO 128 B).
// ---------------------------------------------------------------------------
namespace ftc {
constexpr int A_BYTES = 4 * 128 * 16;          // 8192 per buffer
constexpr int B_BYTES = 4 * 64 * 16;           // 4096
constexpr int OFF_A = 0;                       // two A buffers
constexpr int OFF_B = OFF_A + 2 * A_BYTES;
constexpr int OFF_BAR = OFF_B + B_BYTES;       // two mbarriers
constexpr int OFF_MISC = OFF_BAR + 16;
constexpr int CTAS_PER_SM = 4;
constexpr int TMEM_COLS = 128;                 // 2 x 64; 4 CTAs x 128 = 512 per SM
// requested dynamic shared memory: also caps residency at 4 CTAs per SM, so the
// CTAs of an SM never ask for more than its 512 TMEM columns
constexpr int SMEM = 52 * 1024;
constexpr uint32_t IDESC = ptx::idesc_bf16_f32(128, 64);
constexpr long long BUDGET = 2000000000LL;
}  // namespace ftc

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <bool FP8>
__global__ void __launch_bounds__(128) k_first_tc(const __grid_constant__ FirstTable T,
                                                  const uint4* __restrict__ wb, float inv_out,
                                                  int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* Bs = smem + ftc::OFF_B;
    uint64_t* bar = (uint64_t*)(smem + ftc::OFF_BAR);
    uint32_t* tmem_slot = (uint32_t*)(smem + ftc::OFF_MISC);
    volatile int* abort_flag = (volatile int*)(smem + ftc::OFF_MISC + 4);
    const int warp = threadIdx.x / 32;
    const int p = threadIdx.x;
    const uint32_t nseg = T.nseg;   // all jobs' segments, < 2^31 (checked by the host)

    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar[0], 1);
        ptx::mbar_init(&bar[1], 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    // the .sync.aligned TMEM calls are issued by warp 1, whose lanes never diverge before them
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, ftc::TMEM_COLS);
        ptx::tmem_relinquish();
    }
    // B: 4 KB of weights, 32 B per thread (constant: read before the predecessor finishes)
    reinterpret_cast<uint4*>(Bs)[2 * p] = __ldg(wb + 2 * p);
    reinterpret_cast<uint4*>(Bs)[2 * p + 1] = __ldg(wb + 2 * p + 1);
    ptx::tc_fence_before();
    __syncthreads();   // TMEM allocated before dependents may launch
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_launch_dependents();
    pdl_wait();

    // segment -> (job, image, row, 128-pixel column block). A CTA's segments
    // increase, so its job index only moves forward.
    struct Seg {
        int job, img, yy, bx;
    };
    int jcur = 0;
    auto decompose = [&](uint32_t seg) {
        while (jcur + 1 < T.n && seg >= T.j[jcur + 1].seg_begin) ++jcur;
        const FirstJob& J = T.j[jcur];
        const uint32_t local = seg - J.seg_begin;
        const uint32_t r = local / J.nsx;
        Seg q;
        q.job = jcur;
        q.bx = (int)(local - r * J.nsx);
        q.img = (int)(r / (uint32_t)J.ny);
        q.yy = (int)(r - (uint32_t)q.img * (uint32_t)J.ny);
        return q;
    };
    // segment s_new = seg(q) + gridDim.x: within one job, gridDim.x segments are
    // step_rows rows and step_bx column blocks, so q moves by those (one more
    // row on a column carry, then image wrap) instead of two divisions; a
    // segment in a later job is decomposed afresh
    uint32_t step_rows = 0, step_bx = 0;
    int step_job = -1;
    auto advance = [&](const Seg& q, uint32_t s_new) {
        if (jcur + 1 < T.n && s_new >= T.j[jcur + 1].seg_begin) return decompose(s_new);
        const FirstJob& J = T.j[jcur];
        if (step_job != jcur) {
            step_rows = gridDim.x / J.nsx;
            step_bx = gridDim.x - step_rows * J.nsx;
            step_job = jcur;
        }
        Seg n = q;
        uint32_t bx = (uint32_t)q.bx + step_bx, dr = step_rows;
        if (bx >= J.nsx) {
            bx -= J.nsx;
            ++dr;
        }
        n.bx = (int)bx;
        uint32_t yy = (uint32_t)q.yy + dr;
        while (yy >= (uint32_t)J.ny) {
            yy -= (uint32_t)J.ny;
            ++n.img;
        }
        n.yy = (int)yy;
        return n;
    };
    // taps of one pixel of segment q (zero outside the image). Lanes hold
    // consecutive pixels, so only the centre column is loaded per row (raw[0..2])
    // and the left and right taps come from the adjacent lanes when the taps are
    // expanded (expand_taps, after the loads have landed); lane 0 loads its left
    // and lane 31 its right neighbour (raw[3..5]), which lie outside the warp.
    auto load_taps = [&](const Seg& q, float raw[6]) {
        const FirstJob& J = T.j[q.job];
        const int yy = q.yy, img = q.img, ny = J.ny, nx = J.nx;
        const int xx = q.bx * 128 + p;
        const int lane = p & 31;
        const int xe = lane == 0 ? xx - 1 : xx + 1;   // the edge lanes' outside neighbour
        const bool edge = lane == 0 || lane == 31;
        const float* x = J.x + (int64_t)img * ny * nx;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int sy = yy + dy - 1;
            const bool row_ok = sy >= 0 && sy < ny;
            const float* xr = x + (int64_t)sy * nx;
            raw[dy] = (row_ok && xx < nx) ? __ldg(xr + xx) : 0.f;
            raw[3 + dy] = (edge && row_ok && xe >= 0 && xe < nx) ? __ldg(xr + xe) : 0.f;
        }
    };
    // the 9 taps from the raw loads; every thread of the CTA calls it together
    // (the shuffles need all lanes)
    auto expand_taps = [&](const float raw[6], float v[9]) {
        const int lane = p & 31;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const float c = raw[dy];
            float l = __shfl_up_sync(0xffffffffu, c, 1);
            float r = __shfl_down_sync(0xffffffffu, c, 1);
            if (lane == 0) l = raw[3 + dy];
            if (lane == 31) r = raw[3 + dy];
            v[3 * dy] = l;
            v[3 * dy + 1] = c;
            v[3 * dy + 2] = r;
        }
    };
    auto write_a = [&](int buf, const float v[9]) {
        float hi[9], lo[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            hi[t] = __bfloat162float(__float2bfloat16_rn(v[t]));
            lo[t] = v[t] - hi[t];
        }
        uint4 ch[4];
        ch[0] = make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                           pack_bf16(hi[6], hi[7]));
        ch[1] = make_uint4(pack_bf16(hi[8], lo[0]), pack_bf16(lo[1], lo[2]), pack_bf16(lo[3], lo[4]),
                           pack_bf16(lo[5], lo[6]));
        ch[2] = make_uint4(pack_bf16(lo[7], lo[8]), pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]),
                           pack_bf16(hi[4], hi[5]));
        ch[3] = make_uint4(pack_bf16(hi[6], hi[7]), pack_bf16(hi[8], 1.f), pack_bf16(1.f, 0.f), 0u);
        uint8_t* As = smem + ftc::OFF_A + buf * ftc::A_BYTES;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
            *reinterpret_cast<uint4*>(As + kc * 2048 + (p / 8) * 128 + (p % 8) * 16) = ch[kc];
    };
    // TMEM buffer `buf` -> ReLU, mask, 64 channels of this thread's pixel of segment q
    auto epilogue = [&](const Seg& q, int buf) {
        uint32_t acc[64];
        ptx::tmem_ld_32x32b_x64(tmem_base + ((uint32_t)(warp * 32) << 16) + buf * 64, acc);
        ptx::tmem_ld_wait();
        const FirstJob& J = T.j[q.job];
        const int yy = q.yy, img = q.img, ny = J.ny, nx = J.nx, nxp = J.nxp;
        const int xx = q.bx * 128 + p;
        if (xx >= nxp) return;   // past the padded width: nothing to store
        const Rect rc = J.rects ? J.rects[img] : Rect{0, ny, 0, nx};
        const bool valid = xx < nx && yy >= rc.y0 && yy < rc.y1 && xx >= rc.x0 && xx < rc.x1;
        if constexpr (FP8) {
            uint8_t* o = reinterpret_cast<uint8_t*>(J.out) + (((int64_t)img * ny + yy) * 4 * nxp + xx) * 16;
            if (!valid) {
                // zero outside the valid rect
#pragma unroll
                for (int cg = 0; cg < 4; ++cg)
                    *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 16) = make_uint4(0u, 0u, 0u, 0u);
                return;
            }
#pragma unroll
            for (int cg = 0; cg < 4; ++cg) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t* a = acc + cg * 16 + 4 * e;
                    // relu(t) s = relu(t s) for s = inv_out > 0: the conversion applies the ReLU
                    pk[e] = pack_e4m3x4_relu(__uint_as_float(a[0]) * inv_out, __uint_as_float(a[1]) * inv_out,
                                             __uint_as_float(a[2]) * inv_out, __uint_as_float(a[3]) * inv_out);
                }
                *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        } else {
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(J.out) + ((((int64_t)img * ny + yy) * 8) * nxp + xx) * 8;
            if (!valid) {
                // zero outside the valid rect
#pragma unroll
                for (int cg = 0; cg < 8; ++cg)
                    *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 8) = make_uint4(0u, 0u, 0u, 0u);
                return;
            }
#pragma unroll
            for (int cg = 0; cg < 8; ++cg) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    pk[e] = pack_bf16_relu(__uint_as_float(acc[cg * 8 + 2 * e]),
                                           __uint_as_float(acc[cg * 8 + 2 * e + 1]));
                *reinterpret_cast<uint4*>(o + (int64_t)cg * nxp * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
    };

    bool ok = true;
    uint32_t seg = blockIdx.x;
    float raw[6];
    Seg cur = decompose(seg), prev = cur;
    if (seg < nseg) load_taps(cur, raw);
    uint32_t k = 0;
    for (; seg < nseg && ok; seg += gridDim.x, ++k) {
        const int buf = k & 1;
        // A[buf] and TMEM[buf] were last used by segment k - 2, whose MMAs the
        // epilogue of iteration k - 1 waited for
        {
            float v[9];
            expand_taps(raw, v);
            write_a(buf, v);
        }
        ptx::fence_proxy_async_shared();   // generic-proxy smem writes -> tensor core
        ptx::tc_fence_before();
        __syncthreads();
        ptx::tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t a0 = ptx::smem_u32(smem + ftc::OFF_A + buf * ftc::A_BYTES);
            const uint32_t b0 = ptx::smem_u32(Bs);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
                ptx::mma_bf16(tmem_base + buf * 64,
                              ptx::smem_desc_noswizzle(a0 + kk * 2 * 2048, 2048, 128),
                              ptx::smem_desc_noswizzle(b0 + kk * 2 * 1024, 1024, 128), ftc::IDESC,
                              kk);
            ptx::mma_commit(&bar[buf]);
        }
        __syncwarp();
        // taps of the next segment in flight during the previous segment's epilogue
        const Seg next = advance(cur, seg + gridDim.x);
        if (seg + gridDim.x < nseg) load_taps(next, raw);
        if (k > 0) {
            const int pb = buf ^ 1;
            // block-uniform: every thread leaves the loop in the same iteration
            ok = __syncthreads_and(ptx::mbar_wait(&bar[pb], ((k - 1) >> 1) & 1, abort_flag, ftc::BUDGET));
            ptx::tc_fence_after();
            if (ok) epilogue(prev, pb);
            ptx::tc_fence_before();
        }
        prev = cur;
        cur = next;
    }
    if (ok && k > 0) {
        const int pb = (k - 1) & 1;
        ok = __syncthreads_and(ptx::mbar_wait(&bar[pb], ((k - 1) >> 1) & 1, abort_flag, ftc::BUDGET));
        ptx::tc_fence_after();
        if (ok) epilogue(prev, pb);
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, ftc::TMEM_COLS);
    }
    if (threadIdx.x == 0 && *abort_flag && err) atomicExch(err, (int)PNP_ETIMEOUT);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

int bf16_pad_width(int nx) { return (nx + 7) & ~7; }

size_t denoise_bf16_scratch(const DenoiserDev& D, int ny, int nx, int nimg) {
    (void)D;
    return 2 * (size_t)nimg * ny * bf16_pad_width(nx) * 64 * sizeof(__nv_bfloat16) + 256;
}

cudaError_t tc_make_job(TcJob* J, const void* in, void* out, int ny, int nx, int nimg,
                        const Rect* rects, int64_t row_begin, bool fp8) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    memset(J, 0, sizeof(*J));
    const int nxp = bf16_pad_width(nx);
    // dim0 = 8 pixels x one 16-byte channel group (128 B), dim1 = pixel octets,
    // dim2 = channel groups (8 of BF16 x 8, or 4 of E4M3 x 16), dim3 = rows, dim4 = images
    const int ncg = fp8 ? 4 : 8;
    const cuuint64_t dims[5] = {(cuuint64_t)(fp8 ? 128 : 64), (cuuint64_t)nxp / 8, (cuuint64_t)ncg,
                                (cuuint64_t)ny, (cuuint64_t)nimg};
    const cuuint64_t strides[4] = {128, (cuuint64_t)nxp * 16, (cuuint64_t)nxp * 16 * ncg,
                                   (cuuint64_t)nxp * 16 * ncg * ny};
    const cuuint32_t box[5] = {(cuuint32_t)(fp8 ? 128 : 64), tc::ROW_PX / 8, (cuuint32_t)ncg, 1, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(&J->tin, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     5, (void*)in, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    J->out = (__nv_bfloat16*)out;
    J->rects = rects;
    J->ny = ny;
    J->nx = nx;
    J->nxp = nxp;
    J->nimg = nimg;
    J->strips = ceil_div(nx, tc::SEG);
    J->row_begin = row_begin;
    J->rows = (int64_t)nimg * J->strips * ny;
    return cudaSuccess;
}

// One-shot fault injection for the F -> F layers (pnp_debug_inject_tc_timeout):
// armed by the host, consumed by the next such launch that is not being
// captured into a graph.
static std::mutex g_inject_mu;
static bool g_inject_armed = false;
static int g_inject_cta = -1, g_inject_load = 0;
static long long g_inject_budget = 0;

void tc_inject_timeout(int cta, int load_index, long long budget_cycles) {
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_armed = true;
    g_inject_cta = cta;
    g_inject_load = load_index;
    g_inject_budget = budget_cycles;
}

cudaError_t tc_launch(const TcJob& job0, const TcJob* jobs_dev, int njobs, int64_t total_rows,
                      const void* wblob, const float* bias_host, int* err, bool last,
                      cudaStream_t s, bool fp8, const float* scale_host, float inv_out) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaSuccess;
        using KFn = void (*)(TcJob, TcCommon);
        const std::pair<KFn, int> fns[] = {
            {k_conv_tc<false, false>, TcMode<false, false>::SMEM},
            {k_conv_tc<true, false>, TcMode<true, false>::SMEM},
            {k_conv_tc<false, true>, TcMode<false, true>::SMEM},
            {k_conv_tc<true, true>, TcMode<true, true>::SMEM}};
        for (const auto& f : fns)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(f.first, cudaFuncAttributeMaxDynamicSharedMemorySize, f.second);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (total_rows <= 0) return cudaSuccess;
    TcCommon c;
    c.wblob = wblob;
    memset(c.bias, 0, sizeof(c.bias));
    memcpy(c.bias, bias_host, (last ? 1 : 64) * sizeof(float));
    memset(c.scale, 0, sizeof(c.scale));
    if (scale_host) memcpy(c.scale, scale_host, (last ? 1 : 64) * sizeof(float));
    c.inv_out = inv_out;
    c.err = err;
    c.jobs = jobs_dev;
    c.njobs = jobs_dev ? njobs : 1;
    c.total_rows = total_rows;
    c.budget = tc::BUDGET;
    c.skip_cta = -1;
    c.skip_load = 0;
    if (!last) {
        std::lock_guard<std::mutex> lk(g_inject_mu);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (g_inject_armed && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
            cs == cudaStreamCaptureStatusNone) {
            g_inject_armed = false;
            c.skip_cta = g_inject_cta;
            c.skip_load = g_inject_load;
            c.budget = g_inject_budget;
        }
    }
    const int grid = (int)std::min<int64_t>(num_sms(), total_rows);
    timer_begin(last ? T_CONV_LAST : T_CONV_TC, s);
    cudaError_t e;
    if (fp8) {
        if (last) e = launch_pdl(k_conv_tc<true, true>, dim3(grid), dim3(TcMode<true, true>::THREADS), TcMode<true, true>::SMEM, s, job0, c);
        else e = launch_pdl(k_conv_tc<false, true>, dim3(grid), dim3(TcMode<false, true>::THREADS), TcMode<false, true>::SMEM, s, job0, c);
    } else {
        if (last) e = launch_pdl(k_conv_tc<true, false>, dim3(grid), dim3(TcMode<true, false>::THREADS), TcMode<true, false>::SMEM, s, job0, c);
        else e = launch_pdl(k_conv_tc<false, false>, dim3(grid), dim3(TcMode<false, false>::THREADS), TcMode<false, false>::SMEM, s, job0, c);
    }
    timer_end(last ? T_CONV_LAST : T_CONV_TC, s);
    return e;
}

cudaError_t conv_tc_layer(const __nv_bfloat16* in, const __nv_bfloat16* wblob, const float* bias_host,
                          int ny, int nx, int nimg, const Rect* rects, __nv_bfloat16* out,
                          int* err, cudaStream_t s) {
    TcJob J;
    cudaError_t e = tc_make_job(&J, in, out, ny, nx, nimg, rects, 0);
    if (e != cudaSuccess) return e;
    return tc_launch(J, nullptr, 1, J.rows, wblob, bias_host, err, false, s, false, nullptr, 1.f);
}

// One launch over up to FIRST_MAXJ image stacks (jobs); more jobs take
// several launches. Jobs with no pixels are skipped.
template <bool FP8>
static cudaError_t launch_first_tc(const DenoiserDev& D, const FirstJob* jobs, int njobs,
                                   float inv_out, int* err, cudaStream_t s) {
    static bool attr_done[2] = {false, false};
    if (!attr_done[FP8]) {
        cudaError_t e = cudaFuncSetAttribute(k_first_tc<FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ftc::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_first_tc<FP8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_done[FP8] = true;
    }
    for (int j0 = 0; j0 < njobs; j0 += FIRST_MAXJ) {
        FirstTable T;
        memset(&T, 0, sizeof(T));
        int64_t nseg = 0;
        for (int k = j0; k < std::min(njobs, j0 + FIRST_MAXJ); ++k) {
            FirstJob J = jobs[k];
            J.nxp = bf16_pad_width(J.nx);
            J.nsx = (uint32_t)ceil_div(J.nxp, 128);
            J.seg_begin = (uint32_t)nseg;
            nseg += (int64_t)J.nimg * J.ny * J.nsx;
            if (nseg + (int64_t)num_sms() * ftc::CTAS_PER_SM >= ((int64_t)1 << 31))
                return cudaErrorInvalidValue;
            T.j[T.n++] = J;
        }
        if (nseg == 0) continue;
        T.nseg = (uint32_t)nseg;
        const int grid = (int)std::min<int64_t>(nseg, (int64_t)num_sms() * ftc::CTAS_PER_SM);
        timer_begin(T_CONV_EDGE, s);
        cudaError_t e = launch_pdl(k_first_tc<FP8>, dim3(grid), dim3(128), ftc::SMEM, s, T,
                                   reinterpret_cast<const uint4*>(D.wtc_first), inv_out, err);
        timer_end(T_CONV_EDGE, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <bool FP8>
static cudaError_t launch_first_tc(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                                   const Rect* rects, void* out, float inv_out, int* err,
                                   cudaStream_t s) {
    FirstJob J;
    memset(&J, 0, sizeof(J));
    J.x = x;
    J.out = out;
    J.rects = rects;
    J.ny = ny;
    J.nx = nx;
    J.nimg = nimg;
    return launch_first_tc<FP8>(D, &J, 1, inv_out, err, s);
}

cudaError_t first_layer_bf16(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                             const Rect* rects, __nv_bfloat16* out, int* err, cudaStream_t s) {
    return launch_first_tc<false>(D, x, ny, nx, nimg, rects, out, 1.f, err, s);
}

cudaError_t first_layer_bf16_jobs(const DenoiserDev& D, const FirstJob* jobs, int njobs, int* err,
                                  cudaStream_t s) {
    return launch_first_tc<false>(D, jobs, njobs, 1.f, err, s);
}

cudaError_t last_layer_bf16(const DenoiserDev& D, const __nv_bfloat16* act, const float* x,
                            int ny, int nx, int nimg, float* d, int* err, cudaStream_t s) {
    TcJob J;
    cudaError_t e = tc_make_job(&J, act, nullptr, ny, nx, nimg, nullptr, 0);
    if (e != cudaSuccess) return e;
    J.xin = x;   // nullptr: write the residual G instead of d = x - G
    J.dout = d;
    return tc_launch(J, nullptr, 1, J.rows, D.wtc_last, &D.last_bias, err, true, s, false,
                     nullptr, 1.f);
}

cudaError_t denoise_bf16(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                         const Rect* rects, float* d, void* scratch, cudaStream_t s, bool residual,
                         int* err) {
    if (D.F != 64 || !D.wtc || !D.wtc_last || !D.wtc_first || D.K < 2) return cudaErrorInvalidValue;
    const int nxp = bf16_pad_width(nx);
    const size_t act = (size_t)nimg * ny * nxp * 64;
    __nv_bfloat16* A = (__nv_bfloat16*)scratch;
    __nv_bfloat16* B = A + act;
    if (!err) err = (int*)(B + act);
    cudaError_t e = first_layer_bf16(D, x, ny, nx, nimg, rects, A, err, s);
    if (e != cudaSuccess) return e;
    for (int k = 1; k < D.K - 1; ++k) {
        // host copy of the layer's biases (layers before k all have 64 outputs)
        e = conv_tc_layer(A, D.wtc + (size_t)(k - 1) * (tc::W_BYTES / 2), D.hb + 64 * k, ny,
                          nx, nimg, rects, B, err, s);
        if (e != cudaSuccess) return e;
        __nv_bfloat16* t = A; A = B; B = t;
    }
    return last_layer_bf16(D, A, residual ? nullptr : x, ny, nx, nimg, d, err, s);
}

__global__ void k_to_e4m3(const float* __restrict__ src, uint8_t* __restrict__ dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (uint8_t)__nv_cvt_float_to_fp8(src[i], __NV_SATFINITE, __NV_E4M3);
}

cudaError_t convert_e4m3(const float* src, uint8_t* dst, size_t n, cudaStream_t s) {
    note_launch();
    k_to_e4m3<<<ceil_div((int64_t)n, 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

size_t denoise_fp8_scratch(const DenoiserDev& D, int ny, int nx, int nimg) {
    (void)D;
    return 2 * (size_t)nimg * ny * bf16_pad_width(nx) * 64 + 256;
}

// E4M3 denoiser: activations quantised with the per-layer static scales
// D.a8_scale (input of layer k), weights with per-output-channel scales.
cudaError_t denoise_fp8(const DenoiserDev& D, const float* x, int ny, int nx, int nimg,
                        const Rect* rects, float* d, void* scratch, cudaStream_t s, bool residual,
                        int* err) {
    if (D.F != 64 || !D.wtc8 || !D.wtc8_last || !D.wtc_first || !D.fp8_calibrated)
        return cudaErrorInvalidValue;
    const int nxp = bf16_pad_width(nx);
    const size_t act = (size_t)nimg * ny * nxp * 64;
    uint8_t* A = (uint8_t*)scratch;
    uint8_t* B = A + act;
    if (!err) err = (int*)(B + act);
    cudaError_t e = launch_first_tc<true>(D, x, ny, nx, nimg, rects, A, 1.f / D.a8_scale[1], err, s);
    if (e != cudaSuccess) return e;
    const size_t blob = 3 * 4 * 192 * 16;   // bytes of one F -> F layer
    for (int k = 1; k < D.K - 1; ++k) {
        TcJob J;
        e = tc_make_job(&J, A, B, ny, nx, nimg, rects, 0, true);
        if (e != cudaSuccess) return e;
        float sc[64];
        for (int c = 0; c < 64; ++c) sc[c] = D.a8_scale[k] * D.w8_scale[k * 64 + c];
        e = tc_launch(J, nullptr, 1, J.rows, D.wtc8 + (size_t)(k - 1) * blob, D.hb + 64 * k, err,
                      false, s, true, sc, 1.f / D.a8_scale[k + 1]);
        if (e != cudaSuccess) return e;
        uint8_t* t = A; A = B; B = t;
    }
    TcJob J;
    e = tc_make_job(&J, A, nullptr, ny, nx, nimg, nullptr, 0, true);
    if (e != cudaSuccess) return e;
    J.xin = residual ? nullptr : x;
    J.dout = d;
    const float sl = D.a8_scale[D.K - 1] * D.w8_scale[(D.K - 1) * 64];
    return tc_launch(J, nullptr, 1, J.rows, D.wtc8_last, &D.last_bias, err, true, s, true, &sl, 1.f);
}

}  // namespace pnp
