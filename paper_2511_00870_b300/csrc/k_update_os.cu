// Pipelined one-pass Langevin x-update (Eq. 8, Algorithm 1's x-update) for a
// separable blur under Gaussian noise: g = ((H^T H) x - H^T y) / sigma^2 by one
// separable stencil of the square taps of H^T H over the current state x, then
// the update, the Philox noise and the Welford step, exactly as the per-tile
// kernel k_update does it (the same inlined functions, so every pixel gets
// bitwise the same x+, mean and m2).
//
// What differs is the schedule. A persistent grid (as many CTAs as fit on the
// SMs) walks the tiles of all chains; each CTA keeps two shared-memory
// windows and fills the next tile's window while it computes the current one.
// Interior windows come in as one TMA box (cp.async.bulk.tensor, one thread
// issues it); windows that need the circular wrap are copied per element with
// cp.async. Both complete on the buffer's mbarrier (count = the CTA's threads:
// the TMA thread's expect_tx arrival and plain arrivals, or one
// cp.async.mbarrier.arrive.noinc per thread). The operands of a tile's
// epilogue (H^T y, d, mean, m2) are prefetched into L2 when its window is
// issued. Every mbarrier wait is bounded; a CTA whose wait runs out sets the
// error flag, waits (bounded) for its own copies in flight and exits.
#include "pdl.cuh"
#include "stencil_dev.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

namespace pnp {
namespace {

// About one second of SM cycles: a wait that long means a copy was lost.
constexpr long long kOsBudget = 2000000000LL;

template <int KW, int R, int BY>
struct OsGeom {
    using G = Geom<KW>;
    static constexpr int NT = 16 * BY;                  // threads
    static constexpr int ROWS = R * BY;                 // output rows per tile
    static constexpr int RY = KW / 2;                   // square taps: kh = KW
    static constexpr int WY = ROWS + KW - 1;            // window rows
    static constexpr int WINF = (WY * G::WP + 31) & ~31;   // floats per window (128-byte multiple)
    static constexpr int VF = ROWS * G::WP;             // separable strip
    static constexpr int TAPF = 2 * G::KWP;             // vs, then us
    static constexpr uint32_t BOX_BYTES = (uint32_t)(WY * G::WP * 4);
    // floats before the two mbarriers (a multiple of 4: 16-byte aligned)
    static constexpr int FLOATS = 2 * WINF + VF + TAPF;
    static constexpr size_t SMEM = 128 + sizeof(float) * FLOATS + 2 * sizeof(uint64_t) + 16;
    static_assert(WY <= 256 && G::WP <= 256, "TMA box dimensions");
    static_assert(ROWS % SEP_VR == 0 && ROWS % 2 == 0, "tile rows");
    static_assert(FLOATS % 4 == 0, "mbarrier alignment");
};

struct OsTile {
    int bx, by, chain;
};

__device__ __forceinline__ OsTile os_tile(int tile, int ntx, int nty) {
    OsTile T;
    const int rest = tile / ntx;
    T.bx = tile - rest * ntx;
    T.chain = rest / nty;
    T.by = rest - T.chain * nty;
    return T;
}

// Issues the window of `tile` into `win` (completion on `bar`) and prefetches
// its epilogue operands into L2. Every thread of the CTA calls it once.
template <int KW, int R, int BY>
__device__ __forceinline__ void os_issue(const UpdateParams& p, const CUtensorMap* map, int tile,
                                         int ntx, int nty, float* win, uint64_t* bar, int tid) {
    using G = Geom<KW>;
    using O = OsGeom<KW, R, BY>;
    const OsTile T = os_tile(tile, ntx, nty);
    const int ny = p.ny, nx = p.nx;
    const int i0 = T.by * O::ROWS, j0 = T.bx * ST_TX;
    const int64_t plane = (int64_t)ny * nx;
    const bool interior = i0 - O::RY >= 0 && i0 + O::ROWS - 1 + O::RY < ny && j0 - G::AL >= 0 &&
                          j0 - G::AL + G::WXA <= nx;
    if (interior) {
        // one box of WP x WY floats (columns past WXA are not used; past the
        // image they read as zeros)
        if (tid == 0) {
            ptx::fence_proxy_async_shared();
            ptx::mbar_arrive_expect_tx(bar, O::BOX_BYTES);
            ptx::tma_load_3d(win, map, bar, j0 - G::AL, i0 - O::RY, T.chain);
        } else {
            ptx::mbar_arrive(bar);
        }
    } else {
        const float* img = p.r + (int64_t)T.chain * plane;
        for (int e = tid; e < O::WY * G::WXA; e += O::NT) {
            const int u = e / G::WXA, v = e - u * G::WXA;
            const int gi = wrap(i0 - O::RY + u, ny), gj = wrap(j0 - G::AL + v, nx);
            cp_async4(win + u * G::WP + v, img + (int64_t)gi * nx + gj);
        }
        ptx::cp_async_mbar_arrive_noinc(bar);
    }
    const int tx = tid & 15, ty = tid >> 4;
    const int j = j0 + 4 * tx;
    if (j < nx && (tx & 7) == 0) {
        // one 128-byte line per 8 threads of a row
#pragma unroll
        for (int o = 0; o < R; ++o) {
            const int i = i0 + ty * R + o;
            if (i >= ny) break;
            const int64_t n = (int64_t)i * nx + j, nc = (int64_t)T.chain * plane + n;
            prefetch_l2(p.qb + n);
            if (p.d) prefetch_l2(p.d + nc);
            if (p.mean) {
                prefetch_l2(p.mean + nc);
                prefetch_l2(p.m2 + nc);
            }
        }
    }
}

// Epilogue of one tile: the horizontal pass over the strip V, then for each of
// the thread's R rows x+ = update1(...) with g = (H^T H) x - H^T y and the
// Welford step, in the same order as k_update's aligned path.
template <int KW, int R, int BY>
__device__ __forceinline__ void os_epilogue(const UpdateParams& p, const OsTile& T,
                                            const float* win, const float* V, const float* vs,
                                            uint32_t t, float inv_n) {
    using G = Geom<KW>;
    using O = OsGeom<KW, R, BY>;
    const int ny = p.ny, nx = p.nx;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = T.by * O::ROWS, j = T.bx * ST_TX + 4 * tx;
    if (j >= nx || i0 + ty * R >= ny) return;
    float g[R][4];
    sep_horz<KW, R>(V, vs, ty, tx, g);
    const int64_t plane = (int64_t)ny * nx, cofs = (int64_t)T.chain * plane;
    const float* xwin = win + (ty * R + O::RY) * G::WP + 4 * tx + G::AL;
    float* xo = p.x_out + cofs;
    const float* dc = p.d ? p.d + cofs : nullptr;
    float* mc = p.mean ? p.mean + cofs : nullptr;
    float* qc = p.m2 ? p.m2 + cofs : nullptr;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int o = 0; o < R; ++o) {
        const int i = i0 + ty * R + o;
        if (i >= ny) break;
        const int64_t n0 = (int64_t)i * nx + j;
        const float4 bv = __ldg(reinterpret_cast<const float4*>(p.qb + n0));
        const float4 dv = dc ? __ldg(reinterpret_cast<const float4*>(dc + n0)) : zero4;
        float4 mo = zero4, qo = zero4;
        if (inv_n > 0.f) {
            mo = *reinterpret_cast<const float4*>(mc + n0);
            qo = *reinterpret_cast<const float4*>(qc + n0);
        }
        const float4 xv = *reinterpret_cast<const float4*>(xwin + o * G::WP);
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (p.c_noise != 0.f)
            normals_group((uint32_t)(n0 >> 2), t, (uint32_t)T.chain, p.key0, p.key1, z);
        g[o][0] -= bv.x;
        g[o][1] -= bv.y;
        g[o][2] -= bv.z;
        g[o][3] -= bv.w;
        float4 v;
        v.x = update1(p, xv.x, g[o][0], dv.x, z[0], 0.f);
        v.y = update1(p, xv.y, g[o][1], dv.y, z[1], 0.f);
        v.z = update1(p, xv.z, g[o][2], dv.z, z[2], 0.f);
        v.w = update1(p, xv.w, g[o][3], dv.w, z[3], 0.f);
        *reinterpret_cast<float4*>(xo + n0) = v;
        if (inv_n > 0.f) {
            welford1(v.x, inv_n, mo.x, qo.x);
            welford1(v.y, inv_n, mo.y, qo.y);
            welford1(v.z, inv_n, mo.z, qo.z);
            welford1(v.w, inv_n, mo.w, qo.w);
            *reinterpret_cast<float4*>(mc + n0) = mo;
            *reinterpret_cast<float4*>(qc + n0) = qo;
        }
    }
}

// Wait budget and the one-shot test fault (pnp_debug_inject_update_timeout):
// CTA skip_cta does not issue the window of its tile number skip_k (no copy,
// no arrival), so its wait on that window runs out.
struct OsCtl {
    long long budget;
    int skip_cta, skip_k;
};

template <int KW, int R, int BY>
__global__ void __launch_bounds__(16 * BY) k_update_os(const UpdateParams p,
                                                       const __grid_constant__ CUtensorMap map,
                                                       int ntx, int nty, int ntiles, OsCtl ctl) {
    using G = Geom<KW>;
    using O = OsGeom<KW, R, BY>;
    extern __shared__ unsigned char os_raw[];
    float* sm = reinterpret_cast<float*>(
        os_raw + ((128u - (ptx::smem_u32(os_raw) & 127u)) & 127u));
    float* win[2] = {sm, sm + O::WINF};
    float* V = sm + 2 * O::WINF;
    float* vs = V + O::VF;
    float* us = vs + G::KWP;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + O::FLOATS);
    __shared__ int abort_s;
    const int tid = threadIdx.y * 16 + threadIdx.x;
    if (tid == 0) {
        ptx::mbar_init(&bar[0], O::NT);
        ptx::mbar_init(&bar[1], O::NT);
        ptx::fence_mbar_init();
        ptx::prefetch_tensormap(&map);
        abort_s = 0;
    }
    load_taps_sep<KW>(p.hsep, KW, false, vs, us);    // H^T H taps: fixed for the problem
    __syncthreads();
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t t = p.t_dev ? *p.t_dev : p.t;
    float inv_n = p.inv_n;
    if (p.burn_dev) {
        const int64_t n = (int64_t)t + 1 - *p.burn_dev;
        inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
    }
    const bool inject = (int)blockIdx.x == ctl.skip_cta;
    int tile = blockIdx.x;
    if (tile < ntiles && !(inject && ctl.skip_k == 0))
        os_issue<KW, R, BY>(p, &map, tile, ntx, nty, win[0], &bar[0], tid);
    for (int k = 0; tile < ntiles; ++k) {
        const int b = k & 1;
        const int next = tile + gridDim.x;
        if (next < ntiles && !(inject && ctl.skip_k == k + 1))
            os_issue<KW, R, BY>(p, &map, next, ntx, nty, win[b ^ 1], &bar[b ^ 1], tid);
        const uint32_t par = (uint32_t)(k >> 1) & 1u;
        const bool ok = ptx::mbar_wait(&bar[b], par, &abort_s, ctl.budget);
        if (!__syncthreads_and(ok)) {
            // unwind: wait (bounded) for this CTA's own copies still in flight
            // (a window that was never issued simply runs out the budget
            // again), report, and skip the remaining tiles; the CTA still
            // arrives on the step counter below, so the count stays whole
            ptx::mbar_wait_drain(&bar[b], par, ctl.budget);
            if (next < ntiles)
                ptx::mbar_wait_drain(&bar[b ^ 1], (uint32_t)((k + 1) >> 1) & 1u, ctl.budget);
            if (tid == 0 && p.err) atomicExch(p.err, 1);
            break;
        }
        sep_vert<KW, SEP_VR>(win[b], us, KW, O::ROWS, V);
        __syncthreads();
        os_epilogue<KW, R, BY>(p, os_tile(tile, ntx, nty), win[b], V, vs, t, inv_n);
        __syncthreads();   // window b and V are free again
        tile = next;
    }
    if (p.arrive) {
        // the last CTA to finish advances the step counter (all have read t)
        __syncthreads();
        if (tid == 0 && atomicAdd(p.arrive, 1u) == gridDim.x - 1) {
            *p.arrive = 0u;
            *const_cast<uint32_t*>(p.t_dev) = t + 1u;
        }
    }
}

// ------------------------------------------------------------------ host side

using OsFn = void (*)(const UpdateParams, const CUtensorMap, int, int, int, OsCtl);

std::mutex g_os_inject_mu;
bool g_os_inject_armed = false;
OsCtl g_os_inject{kOsBudget, -1, 0};

template <int KW>
OsFn os_fn_kw(int tile) {
    switch (tile) {
        case 0: return k_update_os<KW, 1, 16>;
        case 1: return k_update_os<KW, 2, 8>;
        case 2: return k_update_os<KW, 2, 16>;
        case 3: return k_update_os<KW, 4, 8>;
        case 4: return k_update_os<KW, 1, 8>;
        case 5: return k_update_os<KW, 4, 16>;
    }
    return nullptr;
}

template <int KW>
size_t os_smem_kw(int tile) {
    switch (tile) {
        case 0: return OsGeom<KW, 1, 16>::SMEM;
        case 1: return OsGeom<KW, 2, 8>::SMEM;
        case 2: return OsGeom<KW, 2, 16>::SMEM;
        case 3: return OsGeom<KW, 4, 8>::SMEM;
        case 4: return OsGeom<KW, 1, 8>::SMEM;
        case 5: return OsGeom<KW, 4, 16>::SMEM;
    }
    return 0;
}

// The taps of H^T H for an odd blur size L have 2 L - 1 = 1 (mod 4) entries.
bool os_lookup(int kw, int tile, OsFn* fn, size_t* smem) {
    switch (kw) {
#define PNP_OS_CASE(K)               \
    case K:                          \
        *fn = os_fn_kw<K>(tile);     \
        *smem = os_smem_kw<K>(tile); \
        return *fn != nullptr;
        PNP_OS_CASE(1)
        PNP_OS_CASE(5)
        PNP_OS_CASE(9)
        PNP_OS_CASE(13)
        PNP_OS_CASE(17)
        PNP_OS_CASE(21)
        PNP_OS_CASE(25)
        PNP_OS_CASE(29)
#undef PNP_OS_CASE
    }
    return false;
}

// tile shapes (R, BY), in the order of the stencil autotuner's candidates
constexpr int kOsR[6] = {1, 2, 2, 4, 1, 4};
constexpr int kOsBY[6] = {16, 8, 16, 8, 8, 16};

// CTAs per SM of each (kernel, smem), and the SM count, looked up once
int os_ctas_per_sm(OsFn fn, int nt, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void*, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(reinterpret_cast<const void*>(fn), smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, nt, smem) != cudaSuccess)
        n = 0;
    cache[key] = n;
    return n;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    }
    return n;
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

}  // namespace

cudaError_t launch_update_os(const UpdateParams& p, int tile, cudaStream_t s) {
    if (!p.os || !p.qb || !p.hsep || !p.x_out || p.h || p.z2 || p.kh != p.kw ||
        tile < 0 || tile >= 6 || (p.nx & 3) != 0 || p.nx < 4 || p.ny < 1 || p.nchain < 1 ||
        !aligned16(p.r) || !aligned16(p.x_out) || !aligned16(p.qb) || !aligned16(p.d) ||
        !aligned16(p.mean) || !aligned16(p.m2) || (p.inv_n > 0.f && !p.mean) ||
        (p.burn_dev && !p.mean))
        return cudaErrorNotSupported;
    OsFn fn = nullptr;
    size_t smem = 0;
    if (!os_lookup(p.kw, tile, &fn, &smem)) return cudaErrorNotSupported;
    // the window wraps circularly within one period of the image
    if (p.kh / 2 > p.ny || p.kw / 2 + 3 > p.nx) return cudaErrorNotSupported;
    PFN_encodeTiled enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const int R = kOsR[tile], BY = kOsBY[tile], NT = 16 * BY, rows = R * BY;
    const int rx = p.kw / 2, al = (rx + 3) & ~3, shift = al - rx;
    const int nw4 = (p.kw + 6) / 4 + (shift > 0 ? 1 : 0);
    const int wxa = ST_TX + 2 * al, wp = wxa > ST_TX + 4 * nw4 ? wxa : ST_TX + 4 * nw4;
    const int wy = rows + p.kh - 1;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nchain};
    const cuuint64_t strides[2] = {(cuuint64_t)p.nx * 4, (cuuint64_t)p.nx * p.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)wp, (cuuint32_t)wy, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(p.r), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    const int per_sm = os_ctas_per_sm(fn, NT, smem);
    if (per_sm < 1) return cudaErrorNotSupported;
    const int ntx = ceil_div(p.nx, ST_TX), nty = ceil_div(p.ny, rows);
    const int64_t ntiles64 = (int64_t)ntx * nty * p.nchain;
    if (ntiles64 > (1 << 30)) return cudaErrorNotSupported;
    const int ntiles = (int)ntiles64;
    const int grid = (int)std::min<int64_t>(ntiles64, (int64_t)per_sm * sm_count());
    OsCtl ctl{kOsBudget, -1, 0};
    {
        // the armed test fault goes to the next launch that is not being captured
        std::lock_guard<std::mutex> lk(g_os_inject_mu);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (g_os_inject_armed && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
            cs == cudaStreamCaptureStatusNone) {
            g_os_inject_armed = false;
            ctl = g_os_inject;
        }
    }
    return launch_pdl(fn, dim3(grid), dim3(16, BY), smem, s, p, map, ntx, nty, ntiles, ctl);
}

void os_inject_timeout(int cta, int tile_index, long long budget_cycles) {
    std::lock_guard<std::mutex> lk(g_os_inject_mu);
    g_os_inject_armed = true;
    g_os_inject = OsCtl{budget_cycles, cta, tile_index};
}

}  // namespace pnp
