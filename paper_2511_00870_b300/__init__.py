"""B300 (sm_103a) PnP-ULA sampler for Gaussian deconvolution.

Python binding of the C ABI in ``include/pnp.h``: the functions here only
marshal arguments (numpy arrays on the host, torch CUDA tensors on the device,
torch's current stream) into ``libpnp.so``; every step of the sampler runs in
that library's CUDA kernels. There is no CPU fallback: importing the
low-level functions loads the library and fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import (PNP_BF16, PNP_FP8, PNP_FP32, PNP_GAUSSIAN, PNP_POISSON, PnpError,  # noqa: F401
                   ProblemDesc, check, load)

__all__ = ["Denoiser", "Problem", "Batch", "Server", "PnpError", "load", "version"]

PRECISIONS = {"fp32": PNP_FP32, "bf16": PNP_BF16, "fp8": PNP_FP8}


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream(stream=None):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t):
    if t is None:
        return C.c_void_p(0)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _f32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def version() -> str:
    return load().pnp_version().decode()


# ------------------------------------------------------------------ operators

def pnp_blur(x, y, h, r, stream=None):
    """r = h (*) x - y (circular); x, r: [n, ny, nx] CUDA float32; y: [ny, nx] or None."""
    n, ny, nx = x.shape
    check(load().pnp_blur(_ptr(x), _ptr(y), _ptr(h), h.shape[0], h.shape[1], ny, nx, n, _ptr(r),
                          _stream(stream)))
    return r


def pnp_blur_adjoint(r, h, g, scale=1.0, stream=None):
    n, ny, nx = r.shape
    check(load().pnp_blur_adjoint(_ptr(r), _ptr(h), h.shape[0], h.shape[1], ny, nx, n,
                                  float(scale), _ptr(g), _stream(stream)))
    return g


def pnp_langevin_update(x, r, d, h, sigma, alpha, eps, lam, gamma, seed, t, noise=True,
                        mean=None, m2=None, n_kept=0, stream=None):
    n, ny, nx = x.shape
    check(load().pnp_langevin_update(_ptr(x), _ptr(r), _ptr(d), _ptr(h), h.shape[0], h.shape[1],
                                     ny, nx, n, sigma, alpha, eps, lam, gamma, int(seed), int(t),
                                     int(bool(noise)), _ptr(mean), _ptr(m2), int(n_kept),
                                     _stream(stream)))
    return x


def pnp_inpaint_update(x, y_obs, d, sigma, alpha, eps, lam, gamma, seed, t, noise=True,
                       mean=None, m2=None, n_kept=0, stream=None):
    """Inpainting x-update; y_obs holds NaN at missing pixels."""
    n, ny, nx = x.shape
    check(load().pnp_inpaint_update(_ptr(x), _ptr(y_obs), _ptr(d), ny, nx, n, sigma, alpha, eps,
                                    lam, gamma, int(seed), int(t), int(bool(noise)), _ptr(mean),
                                    _ptr(m2), int(n_kept), _stream(stream)))
    return x


def pnp_finalize_moments(mean, m2, n_kept, mmse, out2, want_var=False, stream=None):
    check(load().pnp_finalize_moments(_ptr(mean), _ptr(m2), mean.numel(), int(n_kept),
                                      int(bool(want_var)), _ptr(mmse), _ptr(out2),
                                      _stream(stream)))
    return mmse, out2


def pnp_stepsizes(hnorm, sigma, alpha, eps, lip_eps, c=0.99):
    lam, gam = C.c_double(), C.c_double()
    check(load().pnp_stepsizes(hnorm, sigma, alpha, eps, lip_eps, c, C.byref(lam), C.byref(gam)))
    return lam.value, gam.value


def pnp_stepsizes_poisson(hnorm, eta, rho1, rho2, alpha, eps, lip_eps, c=0.99):
    """(lambda, gamma, kappa1, kappa2) of the Poisson setting."""
    out = [C.c_double() for _ in range(4)]
    check(load().pnp_stepsizes_poisson(float(hnorm), float(eta), float(rho1), float(rho2),
                                       float(alpha), float(eps), float(lip_eps), float(c),
                                       *[C.byref(o) for o in out]))
    return tuple(o.value for o in out)


def pnp_debug_inject_tc_timeout(cta: int, load_index: int, budget_cycles: int):
    """Test hook: one-shot skipped load and short wait budget for the next
    eager F -> F tensor-core layer (see include/pnp.h)."""
    check(load().pnp_debug_inject_tc_timeout(int(cta), int(load_index), int(budget_cycles)))


def pnp_debug_inject_update_timeout(cta: int, tile_index: int, budget_cycles: int):
    """Test hook: the next pipelined one-pass update launched outside stream
    capture has CTA `cta` skip issuing the window of its tile `tile_index`, with
    every wait bounded by budget_cycles; the problem then reports PNP_ETIMEOUT."""
    check(load().pnp_debug_inject_update_timeout(int(cta), int(tile_index), int(budget_cycles)))


def pnp_set_graph_mode(enable: bool):
    check(load().pnp_set_graph_mode(int(bool(enable))))


def pnp_set_pdl(enable: bool):
    """Programmatic dependent launch between the kernels of an iteration (default on)."""
    check(load().pnp_set_pdl(int(bool(enable))))


def pnp_set_spectral(enable: bool):
    """Spectral (FFT) likelihood gradient for wide blurs on power-of-two images
    (default on); applies to problems created afterwards."""
    check(load().pnp_set_spectral(int(bool(enable))))


def pnp_stencil_tile_count() -> int:
    return int(load().pnp_stencil_tile_count())


def pnp_set_stencil_tile(tile: int):
    """Force stencil tile shape `tile` for every later launch (-1: per-problem choice)."""
    check(load().pnp_set_stencil_tile(int(tile)))


def pnp_launch_count() -> int:
    """Kernel launches the library has enqueued eagerly so far (graph replays excluded)."""
    return int(load().pnp_launch_count())


def pnp_kernel_timer(enable: bool):
    check(load().pnp_kernel_timer(int(bool(enable))))


def pnp_kernel_timer_read(name: str):
    """-> (total device ms, launches) of the named kernel since the timer was enabled."""
    ms, n = C.c_double(), C.c_int64()
    check(load().pnp_kernel_timer_read(name.encode(), C.byref(ms), C.byref(n)))
    return ms.value, n.value


# ------------------------------------------------------------------ denoiser

class Denoiser:
    """DnCNN-form denoiser D = Id - G owned by the library (pnp_create_denoiser)."""

    def __init__(self, weights, biases, lipschitz: float):
        """weights: list of K arrays [cout, cin, 3, 3]; biases: list of K arrays [cout]."""
        self.K = len(weights)
        self.F = int(weights[0].shape[0])
        w = np.ascontiguousarray(np.concatenate([np.asarray(a, np.float32).ravel() for a in weights]))
        b = np.ascontiguousarray(np.concatenate([np.asarray(a, np.float32).ravel() for a in biases]))
        h = C.c_void_p()
        check(load().pnp_create_denoiser(self.K, self.F, _f32p(w), _f32p(b), float(lipschitz),
                                         C.byref(h)))
        self.handle = h
        self.lipschitz = float(lipschitz)

    @classmethod
    def from_weights(cls, dw):
        return cls(dw.weights, dw.biases, dw.lipschitz)

    @classmethod
    def ddfb(cls, filters, gammas, ht):
        """DDFB denoiser (pnp_create_ddfb): filters [K][P][3][3], gammas [K], ht > 0."""
        f = np.ascontiguousarray(filters, dtype=np.float32)
        g = np.ascontiguousarray(gammas, dtype=np.float32)
        obj = cls.__new__(cls)
        obj.K, obj.F = int(f.shape[0]), int(f.shape[1])
        h = C.c_void_p()
        check(load().pnp_create_ddfb(obj.K, obj.F, _f32p(f), _f32p(g), float(ht), C.byref(h)))
        obj.handle = h
        obj.lipschitz = 1.0
        return obj

    def denoise(self, x, out=None, precision="fp32", blocks=(1, 1), halo=0, stream=None):
        """pnp_denoise on x [n, ny, nx] (CUDA float32)."""
        import torch
        n, ny, nx = x.shape
        out = torch.empty_like(x) if out is None else out
        check(load().pnp_denoise(self.handle, _prec(precision), _ptr(x), ny, nx, n, blocks[0],
                                 blocks[1], halo, _ptr(out), _stream(stream)))
        return out

    def calibrate_fp8(self, x, stream=None):
        """pnp_denoiser_calibrate_fp8 on x [n, ny, nx] (CUDA float32)."""
        n, ny, nx = x.shape
        check(load().pnp_denoiser_calibrate_fp8(self.handle, _ptr(x), ny, nx, n, _stream(stream)))

    def denoise_noalloc(self, x, out, precision="fp32", stream=None):
        """pnp_denoise_noalloc: same result as denoise() with halo = 0, computed in
        the library's fixed scratch area instead of allocating; `out` is caller-owned.
        x and out must be float32 tensors of one shape on the current CUDA device
        (the fixed area is looked up for that device)."""
        import torch
        dev = torch.cuda.current_device()
        for name, t in (("x", x), ("out", out)):
            if t.dtype != torch.float32:
                raise ValueError(f"denoise_noalloc: {name} must be float32, not {t.dtype}")
            if not t.is_cuda or t.device.index != dev:
                raise ValueError(f"denoise_noalloc: {name} must be on the current CUDA device "
                                 f"cuda:{dev}, not {t.device}")
        if tuple(out.shape) != tuple(x.shape):
            raise ValueError("denoise_noalloc: out must have the shape of x")
        n, ny, nx = x.shape
        check(load().pnp_denoise_noalloc(self.handle, _prec(precision), _ptr(x), ny, nx, n,
                                         _ptr(out), _stream(stream)))
        return out

    def status(self, stream=None):
        """pnp_denoise_status: waits for the stream, raises PnpError (PNP_ETIMEOUT)
        if a bounded device-side wait of an earlier denoise call ran out."""
        check(load().pnp_denoise_status(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().pnp_destroy_denoiser(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ problem

def make_desc(y, h, sigma, denoiser=None, *, alpha=-1.0, eps=0.0, lam=0.0, gamma=0.0,
              step_c=0.0, hnorm=0.0, blocks=(1, 1), halo=0, nchain=1, seed=0, burn_in=0,
              precision="fp32", x0=None, stream=None, noise_model="gaussian", eta=0.0,
              rho1=0.0, rho2=0.0, kappa1=0.0, kappa2=0.0, mask=None):
    """Fill a pnp_problem_desc; returns (desc, keep-alive host arrays). With
    noise_model="poisson" y holds counts and sigma is ignored (pass 0)."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    h = np.ascontiguousarray(h if h is not None else np.ones((1, 1)), dtype=np.float32)
    d = ProblemDesc()
    d.ny, d.nx = y.shape
    d.y = _f32p(y)
    d.kh, d.kw = h.shape
    d.h = _f32p(h)
    d.sigma, d.alpha, d.eps = float(sigma), float(alpha), float(eps)
    d.lam, d.gamma, d.step_c, d.hnorm = float(lam), float(gamma), float(step_c), float(hnorm)
    d.blocks_y, d.blocks_x = int(blocks[0]), int(blocks[1])
    d.halo, d.nchain, d.seed, d.burn_in = int(halo), int(nchain), int(seed), int(burn_in)
    d.precision = _prec(precision)
    d.D = denoiser.handle if denoiser is not None else None
    keep = [y, h]
    if x0 is not None:
        x0a = np.ascontiguousarray(np.broadcast_to(x0, (nchain,) + y.shape), dtype=np.float32)
        d.x0 = _f32p(x0a)
        keep.append(x0a)
    d.stream = C.c_void_p(int(stream)) if stream is not None else None
    if noise_model not in ("gaussian", "poisson"):
        raise ValueError(f"unknown noise model {noise_model!r}")
    d.noise_model = PNP_POISSON if noise_model == "poisson" else PNP_GAUSSIAN
    d.eta, d.rho1, d.rho2 = float(eta), float(rho1), float(rho2)
    d.kappa1, d.kappa2 = float(kappa1), float(kappa2)
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.float32)
        if m.shape != y.shape:
            raise ValueError("mask must have the shape of y")
        d.mask = _f32p(m)
        keep.append(m)
    return d, keep


class Problem:
    """One posterior and its chains resident on the GPU (pnp_create_problem)."""

    def __init__(self, y, h, sigma, denoiser: Denoiser | None = None, **kw):
        d, keep = make_desc(y, h, sigma, denoiser, **kw)
        self.shape = (d.ny, d.nx)
        self.nchain = d.nchain
        hdl = C.c_void_p()
        check(load().pnp_create_problem(C.byref(d), C.byref(hdl)))
        self.handle = hdl
        self._owned = True
        self._denoiser = denoiser   # keep alive

    @classmethod
    def _borrow(cls, handle, shape, nchain, owner):
        obj = cls.__new__(cls)
        obj.handle = handle
        obj.shape = shape
        obj.nchain = nchain
        obj._owned = False
        obj._owner = owner
        return obj

    def params(self):
        lam, gam, al, ep = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        check(load().pnp_problem_params(self.handle, C.byref(lam), C.byref(gam), C.byref(al),
                                        C.byref(ep)))
        return dict(lam=lam.value, gamma=gam.value, alpha=al.value, eps=ep.value)

    def stencil_tiles(self):
        """(blur tile, update tile, separable) picked for this problem."""
        b, u, s = C.c_int(), C.c_int(), C.c_int()
        check(load().pnp_problem_stencil_tiles(self.handle, C.byref(b), C.byref(u), C.byref(s)))
        return b.value, u.value, bool(s.value)

    def step(self, n=1):
        check(load().pnp_step(self.handle, int(n)))

    def sync(self):
        check(load().pnp_sync(self.handle))

    def prepare_graphs(self):
        """pnp_prepare_graphs: capture the replayed graphs now (after one step)."""
        check(load().pnp_prepare_graphs(self.handle))

    def run_chain(self, T, burn_in):
        check(load().pnp_run_chain(self.handle, int(T), int(burn_in)))

    def moments(self, chain=0, want_var=False):
        ny, nx = self.shape
        mm = np.empty((ny, nx), np.float64)
        o2 = np.empty((ny, nx), np.float64)
        n = C.c_int64()
        check(load().pnp_get_moments(self.handle, chain, mm.ctypes.data_as(C.POINTER(C.c_double)),
                                     o2.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n),
                                     int(bool(want_var))))
        return mm, o2, n.value

    def state(self):
        x = np.empty((self.nchain,) + self.shape, np.float32)
        t = C.c_int64()
        check(load().pnp_get_state(self.handle, _f32p(x), C.byref(t)))
        return x, t.value

    def set_state(self, x, t):
        x = np.ascontiguousarray(np.broadcast_to(x, (self.nchain,) + self.shape), dtype=np.float32)
        check(load().pnp_set_state(self.handle, _f32p(x), int(t)))

    def aux_state(self):
        """(z1, z2) of a Poisson problem, each [nchain][ny][nx] FP32."""
        z1 = np.empty((self.nchain,) + self.shape, np.float32)
        z2 = np.empty_like(z1)
        check(load().pnp_get_aux_state(self.handle, _f32p(z1), _f32p(z2)))
        return z1, z2

    def set_aux_state(self, z1, z2):
        sh = (self.nchain,) + self.shape
        z1 = np.ascontiguousarray(np.broadcast_to(z1, sh), dtype=np.float32)
        z2 = np.ascontiguousarray(np.broadcast_to(z2, sh), dtype=np.float32)
        check(load().pnp_set_aux_state(self.handle, _f32p(z1), _f32p(z2)))

    def x_device_ptr(self):
        return load().pnp_problem_x_device(self.handle)

    def close(self):
        if getattr(self, "handle", None) and getattr(self, "_owned", True):
            load().pnp_destroy_problem(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batch

class Batch:
    """Independent problems stepped together (pnp_batch_create); each job is a
    dict of make_desc keyword arguments plus y, h, sigma."""

    def __init__(self, jobs, denoiser: Denoiser, precision="bf16", stream=None):
        descs = (ProblemDesc * len(jobs))()
        self._keep = []
        self.shapes = []
        for k, jb in enumerate(jobs):
            jb = dict(jb)
            d, keep = make_desc(jb.pop("y"), jb.pop("h"), jb.pop("sigma"), denoiser,
                                precision=precision, **jb)
            descs[k] = d
            self._keep.append(keep)
            self.shapes.append(((d.ny, d.nx), d.nchain))
        hdl = C.c_void_p()
        check(load().pnp_batch_create(descs, len(jobs), C.c_void_p(int(stream)) if stream else None,
                                      C.byref(hdl)))
        self.handle = hdl
        self._denoiser = denoiser

    def __len__(self):
        return len(self.shapes)

    def step(self, n=1):
        check(load().pnp_batch_step(self.handle, int(n)))

    def run(self, T, burn_in):
        check(load().pnp_batch_run(self.handle, int(T), int(burn_in)))

    def sync(self):
        check(load().pnp_batch_sync(self.handle))

    def job(self, j) -> Problem:
        h = C.c_void_p()
        check(load().pnp_batch_job(self.handle, int(j), C.byref(h)))
        shape, nchain = self.shapes[j]
        return Problem._borrow(h, shape, nchain, self)

    def close(self):
        if getattr(self, "handle", None):
            load().pnp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class Server:
    """Continuous-batching sampler service (pnp_server_create)."""

    def __init__(self, denoiser: Denoiser, precision="bf16", hbm_budget_bytes=64 << 30,
                 stream=None, round_iters=8, max_boost=16):
        hdl = C.c_void_p()
        check(load().pnp_server_create(denoiser.handle if denoiser else None, _prec(precision),
                                       int(hbm_budget_bytes),
                                       C.c_void_p(int(stream)) if stream else None, C.byref(hdl)))
        self.handle = hdl
        self._denoiser = denoiser
        self._shapes = {}
        check(load().pnp_server_set_round(self.handle, int(round_iters), int(max_boost)))

    def submit(self, y, h, sigma, T, burn_in, **kw):
        d, keep = make_desc(y, h, sigma, None, burn_in=burn_in, **kw)
        jid = C.c_int64()
        check(load().pnp_server_submit(self.handle, C.byref(d), int(T), int(burn_in), C.byref(jid)))
        self._shapes[jid.value] = (d.ny, d.nx)
        return jid.value

    def poll(self, job_id, fetch=True):
        """-> (state name, mmse or None, std or None)."""
        ny, nx = self._shapes[job_id]
        st = C.c_int()
        mm = np.empty((ny, nx)) if fetch else None
        sd = np.empty((ny, nx)) if fetch else None
        check(load().pnp_server_poll(self.handle, int(job_id),
                                     mm.ctypes.data_as(C.POINTER(C.c_double)) if fetch else None,
                                     sd.ctypes.data_as(C.POINTER(C.c_double)) if fetch else None,
                                     C.byref(st)))
        name = JOB_STATES[st.value]
        return (name, mm, sd) if name == "done" else (name, None, None)

    def wait(self, job_id, timeout=600.0):
        st = C.c_int()
        check(load().pnp_server_wait(self.handle, int(job_id), float(timeout), C.byref(st)))
        return JOB_STATES[st.value]

    def cancel(self, job_id):
        check(load().pnp_server_cancel(self.handle, int(job_id)))

    def times(self, job_id):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        check(load().pnp_server_job_times(self.handle, int(job_id), C.byref(a), C.byref(b), C.byref(c)))
        return dict(submit=a.value, admit=b.value, done=c.value)

    def stats(self):
        px, act, q, used = C.c_int64(), C.c_int(), C.c_int(), C.c_size_t()
        check(load().pnp_server_stats(self.handle, C.byref(px), C.byref(act), C.byref(q), C.byref(used)))
        return dict(pixel_iters=px.value, active=act.value, queued=q.value, used_bytes=used.value)

    def device_seconds(self):
        """Device time of all rounds so far (pnp_server_device_seconds)."""
        v = C.c_double()
        check(load().pnp_server_device_seconds(self.handle, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "handle", None):
            load().pnp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
