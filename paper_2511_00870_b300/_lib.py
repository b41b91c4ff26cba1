"""ctypes declarations of libpnp's C ABI (include/pnp.h). Marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpnp.so")

PNP_OK, PNP_EINVAL, PNP_ENOMEM, PNP_EBUSY, PNP_ECUDA, PNP_ETIMEOUT, PNP_ESTATE, PNP_ENOTSUP = range(8)
STATUS_NAMES = ["PNP_OK", "PNP_EINVAL", "PNP_ENOMEM", "PNP_EBUSY", "PNP_ECUDA", "PNP_ETIMEOUT",
                "PNP_ESTATE", "PNP_ENOTSUP"]
PNP_FP32, PNP_BF16, PNP_FP8 = 0, 1, 2
PNP_GAUSSIAN, PNP_POISSON = 0, 1


class PnpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class ProblemDesc(C.Structure):
    _fields_ = [
        ("ny", C.c_int), ("nx", C.c_int),
        ("y", C.POINTER(C.c_float)),
        ("kh", C.c_int), ("kw", C.c_int),
        ("h", C.POINTER(C.c_float)),
        ("sigma", C.c_double), ("alpha", C.c_double), ("eps", C.c_double),
        ("lam", C.c_double), ("gamma", C.c_double), ("step_c", C.c_double), ("hnorm", C.c_double),
        ("blocks_y", C.c_int), ("blocks_x", C.c_int), ("halo", C.c_int), ("nchain", C.c_int),
        ("seed", C.c_uint64), ("burn_in", C.c_int), ("precision", C.c_int),
        ("D", C.c_void_p),
        ("x0", C.POINTER(C.c_float)),
        ("stream", C.c_void_p),
        ("noise_model", C.c_int),
        ("eta", C.c_double), ("rho1", C.c_double), ("rho2", C.c_double),
        ("kappa1", C.c_double), ("kappa2", C.c_double),
        ("mask", C.POINTER(C.c_float)),
    ]


_lib = None

fp = C.POINTER(C.c_float)
dp = C.POINTER(C.c_double)
vp = C.c_void_p
i32, i64, u32, u64, f32, f64 = C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_float, C.c_double

SIGNATURES = {
    "pnp_last_error": ([], C.c_char_p),
    "pnp_version": ([], C.c_char_p),
    "pnp_create_denoiser": ([i32, i32, fp, fp, f64, C.POINTER(vp)], i32),
    "pnp_destroy_denoiser": ([vp], None),
    "pnp_create_ddfb": ([i32, i32, fp, fp, f64, C.POINTER(vp)], i32),
    "pnp_denoiser_calibrate_fp8": ([vp, vp, i32, i32, i32, vp], i32),
    "pnp_blur": ([vp, vp, vp, i32, i32, i32, i32, i32, vp, vp], i32),
    "pnp_blur_adjoint": ([vp, vp, i32, i32, i32, i32, i32, f32, vp, vp], i32),
    "pnp_denoise": ([vp, i32, vp, i32, i32, i32, i32, i32, i32, vp, vp], i32),
    "pnp_denoise_noalloc": ([vp, i32, vp, i32, i32, i32, vp, vp], i32),
    "pnp_denoise_status": ([vp, vp], i32),
    "pnp_debug_inject_tc_timeout": ([i32, i32, C.c_longlong], i32),
    "pnp_debug_inject_update_timeout": ([i32, i32, C.c_longlong], i32),
    "pnp_langevin_update": ([vp, vp, vp, vp, i32, i32, i32, i32, i32, f64, f64, f64, f64, f64,
                             u64, u32, i32, vp, vp, i64, vp], i32),
    "pnp_inpaint_update": ([vp, vp, vp, i32, i32, i32, f64, f64, f64, f64, f64, u64, u32, i32,
                            vp, vp, i64, vp], i32),
    "pnp_finalize_moments": ([vp, vp, i64, i64, i32, vp, vp, vp], i32),
    "pnp_stepsizes": ([f64, f64, f64, f64, f64, f64, dp, dp], i32),
    "pnp_stepsizes_poisson": ([f64, f64, f64, f64, f64, f64, f64, f64, dp, dp, dp, dp], i32),
    "pnp_create_problem": ([C.POINTER(ProblemDesc), C.POINTER(vp)], i32),
    "pnp_destroy_problem": ([vp], None),
    "pnp_problem_params": ([vp, dp, dp, dp, dp], i32),
    "pnp_step": ([vp, i32], i32),
    "pnp_run_chain": ([vp, i32, i32], i32),
    "pnp_sync": ([vp], i32),
    "pnp_prepare_graphs": ([vp], i32),
    "pnp_get_moments": ([vp, i32, dp, dp, C.POINTER(i64), i32], i32),
    "pnp_get_state": ([vp, fp, C.POINTER(i64)], i32),
    "pnp_set_state": ([vp, fp, i64], i32),
    "pnp_get_aux_state": ([vp, fp, fp], i32),
    "pnp_set_aux_state": ([vp, fp, fp], i32),
    "pnp_problem_x_device": ([vp], vp),
    "pnp_set_graph_mode": ([i32], i32),
    "pnp_set_pdl": ([i32], i32),
    "pnp_set_spectral": ([i32], i32),
    "pnp_stencil_tile_count": ([], i32),
    "pnp_set_stencil_tile": ([i32], i32),
    "pnp_problem_stencil_tiles": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], i32),
    "pnp_batch_create": ([C.POINTER(ProblemDesc), i32, vp, C.POINTER(vp)], i32),
    "pnp_batch_destroy": ([vp], None),
    "pnp_batch_step": ([vp, i32], i32),
    "pnp_batch_run": ([vp, i32, i32], i32),
    "pnp_batch_sync": ([vp], i32),
    "pnp_batch_job": ([vp, i32, C.POINTER(vp)], i32),
    "pnp_batch_size": ([vp], i32),
    "pnp_server_create": ([vp, i32, C.c_size_t, vp, C.POINTER(vp)], i32),
    "pnp_server_submit": ([vp, C.POINTER(ProblemDesc), i32, i32, C.POINTER(i64)], i32),
    "pnp_server_poll": ([vp, i64, dp, dp, C.POINTER(i32)], i32),
    "pnp_server_wait": ([vp, i64, f64, C.POINTER(i32)], i32),
    "pnp_server_cancel": ([vp, i64], i32),
    "pnp_server_job_times": ([vp, i64, dp, dp, dp], i32),
    "pnp_server_stats": ([vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_size_t)], i32),
    "pnp_server_set_round": ([vp, i32, i32], i32),
    "pnp_server_destroy": ([vp], None),
    "pnp_kernel_timer": ([i32], i32),
    "pnp_launch_count": ([], i64),
    "pnp_server_device_seconds": ([vp, dp], i32),
    "pnp_kernel_timer_read": ([C.c_char_p, dp, C.POINTER(i64)], i32),
}


def load(path: str = LIB_PATH):
    """Load libpnp.so. Raises if the CUDA library has not been built: there is
    no CPU fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libpnp.so not found at {path}; build it with "
                              "`python -m paper_2511_00870_b300.build`")
        lib = C.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def check(status: int):
    if status != PNP_OK:
        raise PnpError(status, load().pnp_last_error().decode())
    return status
