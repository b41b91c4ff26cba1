// pnp_denoise_noalloc: the denoiser without any device allocation.
//
// pnp_denoise grows a per-denoiser scratch buffer with cudaMalloc the first
// time it sees a larger image. Some callers cannot allow that: a process in
// which another allocator (for example a framework's caching allocator) has
// already reserved nearly all of HBM, so a raw cudaMalloc would fail; or a
// latency-bound loop that must never stall, where cudaMalloc/cudaFree can
// synchronize the device. This entry point runs the same kernels on a fixed
// scratch area that lives in the library itself: a file-scope __device__
// array, held on a GPU from the moment its module is loaded there until the
// process exits. With CUDA's lazy module loading that moment is the first
// lookup of the array's address; pnp_create_denoiser does that lookup on the
// current device (noalloc_reserve), so the area is reserved while device
// memory is still free rather than at the first allocation-free call.
#include "pnp_internal.h"

namespace pnp {

constexpr size_t NOALLOC_SCRATCH_BYTES = PNP_NOALLOC_SCRATCH_BYTES;

// The shared scratch. Host code must not use this symbol as a pointer: on the
// host it names a stand-in object, not device memory. Its device address is
// obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, resolved once per device.
static void* g_noalloc_ptr[64] = {nullptr};

static pnp_status noalloc_scratch(void** out) {
    int dev = 0;
    PNP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PNP_ENOTSUP, "pnp_denoise_noalloc: device index >= 64");
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PNP_OK;
}

pnp_status noalloc_reserve() {
    void* p = nullptr;
    return noalloc_scratch(&p);
}

}  // namespace pnp

using namespace pnp;

extern "C" pnp_status pnp_denoise_noalloc(const pnp_denoiser* den, pnp_precision prec,
                                          const float* x, int ny, int nx, int nimg, float* d,
                                          void* stream) {
    if (!den || !x || !d) return fail(PNP_EINVAL, "pnp_denoise_noalloc: NULL argument");
    if (ny < 1 || nx < 1 || nimg < 1) return fail(PNP_EINVAL, "pnp_denoise_noalloc: empty image");
    const DenoiserDev& D = den->dev;
    if (D.ddfb && prec != PNP_FP32)
        return fail(PNP_ENOTSUP, "pnp_denoise_noalloc: the DDFB denoiser runs in FP32");
    size_t need = 0;
    if (prec == PNP_FP32) {
        need = denoise_fp32_scratch(D, ny, nx, nimg);
    } else if (prec == PNP_BF16) {
        if (D.F != 64) return fail(PNP_EINVAL, "pnp_denoise_noalloc: BF16 path needs F = 64");
        need = denoise_bf16_scratch(D, ny, nx, nimg);
    } else {
        return fail(PNP_ENOTSUP, "pnp_denoise_noalloc: precision not supported");
    }
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(PNP_EINVAL, "pnp_denoise_noalloc: the image needs " + std::to_string(need) +
                                    " bytes of scratch, more than the fixed " +
                                    std::to_string(NOALLOC_SCRATCH_BYTES) +
                                    " bytes; use pnp_denoise or a smaller image/batch");
    void* scratch = nullptr;
    PNP_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PNP_FP32) {
        // every activation plane is fully written before it is read
        PNP_CUDA_TRY(denoise_fp32(D, x, ny, nx, nimg, nullptr, d, (float*)scratch, s));
    } else {
        // the activation planes (padding columns included) are fully rewritten
        // by every layer; a tensor-core wait that runs out is reported in the
        // denoiser's own flag (pnp_denoise_status)
        PNP_CUDA_TRY(denoise_bf16(D, x, ny, nx, nimg, nullptr, d, scratch, s, false, den->err));
    }
    return PNP_OK;
}
