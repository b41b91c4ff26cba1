"""FP64 CPU oracle for the PnP-ULA Gaussian-deconvolution sampler.

TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers; the product path (the CUDA library and
its binding) never imports this package, and the two share no code. The
arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it with
gcc on first use and marshals numpy arrays through ctypes.

Parity status of each routine is listed in ``oracle.h``; every routine is
pinned by tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP over output pixels)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Net(C.Structure):
    _fields_ = [("K", C.c_int), ("cin", C.POINTER(C.c_int)), ("cout", C.POINTER(C.c_int)),
                ("ks", C.c_int), ("w", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


class _Problem(C.Structure):
    _fields_ = [("ny", C.c_int), ("nx", C.c_int), ("y", C.POINTER(C.c_double)),
                ("h", C.POINTER(C.c_double)), ("kh", C.c_int), ("kw", C.c_int),
                ("sigma", C.c_double), ("alpha", C.c_double), ("eps", C.c_double),
                ("lam", C.c_double), ("gamma", C.c_double), ("seed", C.c_uint64),
                ("net", C.POINTER(_Net)), ("noise", C.c_int), ("ddfb", C.c_void_p),
                ("mask", C.POINTER(C.c_double))]


class _Ddfb(C.Structure):
    _fields_ = [("K", C.c_int), ("P", C.c_int), ("ks", C.c_int), ("w", C.POINTER(C.c_double)),
                ("gamma", C.POINTER(C.c_double)), ("ht", C.c_double)]


class _Poisson(C.Structure):
    _fields_ = [("ny", C.c_int), ("nx", C.c_int), ("y", C.POINTER(C.c_double)),
                ("h", C.POINTER(C.c_double)), ("kh", C.c_int), ("kw", C.c_int),
                ("eta", C.c_double), ("rho1", C.c_double), ("rho2", C.c_double),
                ("kappa1", C.c_double), ("kappa2", C.c_double),
                ("alpha", C.c_double), ("eps", C.c_double),
                ("lam", C.c_double), ("gamma", C.c_double), ("seed", C.c_uint64),
                ("net", C.POINTER(_Net)), ("noise", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, u32, i64 = C.POINTER(C.c_double), C.c_int, C.c_uint32, C.c_int64
        _lib.ora_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32)]
        _lib.ora_normals.argtypes = [C.c_uint64, u32, u32, i64, d]
        _lib.ora_blur.argtypes = [d, i, i, d, i, i, d]
        _lib.ora_blur_adj.argtypes = [d, i, i, d, i, i, d]
        _lib.ora_conv_layer.argtypes = [d, i, i, i, d, d, i, i, i, d]
        _lib.ora_denoise.argtypes = [d, i, i, C.POINTER(_Net), d]
        _lib.ora_denoise_blockwise.argtypes = [d, i, i, C.POINTER(_Net), i, i, i, d]
        _lib.ora_denoise_blockwise.restype = C.c_int
        _lib.ora_stepsizes.argtypes = [C.c_double] * 6 + [d, d]
        _lib.ora_langevin_step.argtypes = [C.POINTER(_Problem), d, u32, u32, d]
        _lib.ora_langevin_step_window.argtypes = [C.POINTER(_Problem), d, u32, u32, i, i, i, i, d]
        _lib.ora_langevin_step_window.restype = C.c_int
        _lib.ora_run_chain.argtypes = [C.POINTER(_Problem), d, i, i, i, u32, d, d,
                                       C.POINTER(C.c_int64), d]
        _lib.ora_moments_two_pass.argtypes = [d, i64, i64, d, d]
        _lib.ora_normals_stream.argtypes = [C.c_uint64, u32, u32, u32, i64, d]
        _lib.ora_kl_prox.argtypes = [C.c_double] * 3
        _lib.ora_kl_prox.restype = C.c_double
        _lib.ora_poisson_stepsizes.argtypes = [C.c_double] * 8 + [d] * 4
        _lib.ora_poisson_step.argtypes = [C.POINTER(_Poisson), d, d, d, u32, u32, d, d, d]
        _lib.ora_ddfb_W.argtypes = [d, i, i, d, i, i, d]
        _lib.ora_ddfb_Wt.argtypes = [d, i, i, d, i, i, d]
        _lib.ora_ddfb_denoise.argtypes = [d, i, i, C.POINTER(_Ddfb), d]
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- RNG

def philox4x32_10(ctr, key):
    """ctr: uint32 [n, 4]; key: uint32 [2] -> uint32 [n, 4]."""
    ctr = np.ascontiguousarray(np.atleast_2d(ctr), dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(ctr)
    L = lib()
    for k in range(ctr.shape[0]):
        L.ora_philox4x32_10(ctr[k].ctypes.data_as(C.POINTER(C.c_uint32)),
                            key.ctypes.data_as(C.POINTER(C.c_uint32)),
                            out[k].ctypes.data_as(C.POINTER(C.c_uint32)))
    return out


def normals(seed: int, t: int, chain: int, n: int):
    xi = np.zeros(n)
    lib().ora_normals(C.c_uint64(seed), t, chain, n, _dp(xi))
    return xi


# ---------------------------------------------------------------- blur

def blur(x, h):
    x, h = _f64(x), _f64(h)
    out = np.empty_like(x)
    lib().ora_blur(_dp(x), x.shape[0], x.shape[1], _dp(h), h.shape[0], h.shape[1], _dp(out))
    return out


def blur_adj(r, h):
    r, h = _f64(r), _f64(h)
    out = np.empty_like(r)
    lib().ora_blur_adj(_dp(r), r.shape[0], r.shape[1], _dp(h), h.shape[0], h.shape[1], _dp(out))
    return out


# ---------------------------------------------------------------- denoiser

def conv_layer(inp, w, b=None, relu=False):
    """inp [cin, ny, nx]; w [cout, cin, ks, ks]; b [cout] -> [cout, ny, nx]."""
    inp, w = _f64(inp), _f64(w)
    cout, cin, ks, _ = w.shape
    out = np.empty((cout,) + inp.shape[1:])
    bp = _dp(_f64(b)) if b is not None else None
    bb = _f64(b) if b is not None else None
    lib().ora_conv_layer(_dp(inp), cin, inp.shape[1], inp.shape[2], _dp(w),
                         _dp(bb) if bb is not None else C.POINTER(C.c_double)(), cout, ks,
                         int(relu), _dp(out))
    del bp
    return out


class Net:
    """ctypes view of a DnCNN-form network given per-layer OIHW weights."""

    def __init__(self, weights, biases):
        self.K = len(weights)
        self.cin = (C.c_int * self.K)(*[int(w.shape[1]) for w in weights])
        self.cout = (C.c_int * self.K)(*[int(w.shape[0]) for w in weights])
        self.ks = int(weights[0].shape[2])
        self.w = np.concatenate([_f64(w).ravel() for w in weights])
        self.b = np.concatenate([_f64(b).ravel() for b in biases])
        self.s = _Net(self.K, self.cin, self.cout, self.ks, _dp(self.w), _dp(self.b))

    @classmethod
    def from_weights(cls, dw):
        return cls(dw.weights, dw.biases)


def denoise(v, net: Net):
    v = _f64(v)
    out = np.empty_like(v)
    lib().ora_denoise(_dp(v), v.shape[0], v.shape[1], C.byref(net.s), _dp(out))
    return out


def denoise_blockwise(v, net: Net, by: int, bx: int, halo: int):
    v = _f64(v)
    out = np.empty_like(v)
    rc = lib().ora_denoise_blockwise(_dp(v), v.shape[0], v.shape[1], C.byref(net.s),
                                     by, bx, halo, _dp(out))
    if rc != 0:
        raise ValueError("bad block arguments")
    return out


# ---------------------------------------------------------------- sampler

def stepsizes(hnorm, sigma, alpha, eps, lip_eps, c=0.99):
    lam, gam = C.c_double(), C.c_double()
    lib().ora_stepsizes(hnorm, sigma, alpha, eps, lip_eps, c, C.byref(lam), C.byref(gam))
    return lam.value, gam.value


class Problem:
    """Holds the FP64 arrays alive for the C struct."""

    def __init__(self, y, h, sigma, alpha, eps, lam, gamma, seed, net: Net | None = None,
                 noise=True, mask=None, ddfb=None):
        """mask (0/1 array of y's shape): inpainting, H = diag(mask), h unused.
        ddfb (a Ddfb): the DDFB denoiser in place of the DnCNN-form net."""
        self.y = _f64(y)
        self.h = _f64(h if h is not None else np.ones((1, 1)))
        self.mask = _f64(mask) if mask is not None else None
        self.net = net
        self.s = _Problem(self.y.shape[0], self.y.shape[1], _dp(self.y), _dp(self.h),
                          self.h.shape[0], self.h.shape[1], float(sigma), float(alpha),
                          float(eps), float(lam), float(gamma), C.c_uint64(seed),
                          C.pointer(net.s) if net is not None else C.POINTER(_Net)(),
                          int(bool(noise)),
                          C.cast(C.pointer(ddfb.s), C.c_void_p) if ddfb is not None else None,
                          _dp(self.mask) if self.mask is not None else C.POINTER(C.c_double)())
        self.ddfb = ddfb

    @property
    def shape(self):
        return self.y.shape


def langevin_step(p: Problem, x, t: int, chain: int = 0):
    x = _f64(x)
    out = np.empty_like(x)
    lib().ora_langevin_step(C.byref(p.s), _dp(x), t, chain, _dp(out))
    return out


def langevin_step_window(p: Problem, x, t: int, i0: int, j0: int, wy: int, wx: int,
                         chain: int = 0):
    """x^(t+1) of langevin_step at the pixels [i0, i0+wy) x [j0, j0+wx) only."""
    x = _f64(x)
    out = np.empty((wy, wx))
    rc = lib().ora_langevin_step_window(C.byref(p.s), _dp(x), t, chain, i0, j0, wy, wx, _dp(out))
    if rc != 0:
        raise ValueError("window outside the image, or a DDFB denoiser")
    return out


def run_chain(p: Problem, x0, T: int, burn_in: int, chain: int = 0, t0: int = 0,
              store_samples: bool = False):
    """Returns dict(x, mean, m2, n, samples)."""
    x = _f64(x0).copy()
    mean = np.zeros_like(x)
    m2 = np.zeros_like(x)
    n = C.c_int64(0)
    kept = max(0, t0 + T - max(burn_in, t0))
    samples = np.zeros((kept,) + x.shape) if store_samples else None
    lib().ora_run_chain(C.byref(p.s), _dp(x), t0, T, burn_in, chain, _dp(mean), _dp(m2),
                        C.byref(n), _dp(samples) if samples is not None
                        else C.POINTER(C.c_double)())
    return dict(x=x, mean=mean, m2=m2, n=n.value, samples=samples)


# ---------------------------------------------------------------- Poisson (AXDA + PSGLA)

def normals_stream(seed: int, t: int, chain: int, stream: int, n: int):
    xi = np.zeros(n)
    lib().ora_normals_stream(C.c_uint64(seed), t, chain, stream, n, _dp(xi))
    return xi


def kl_prox(v, y, kappa):
    return lib().ora_kl_prox(float(v), float(y), float(kappa))


def poisson_stepsizes(hnorm, eta, rho1, rho2, alpha, eps, lip_eps, c=0.99):
    """-> (lambda, gamma, kappa1, kappa2)."""
    o = [C.c_double() for _ in range(4)]
    lib().ora_poisson_stepsizes(hnorm, eta, rho1, rho2, alpha, eps, lip_eps, c,
                                *[C.byref(v) for v in o])
    return tuple(v.value for v in o)


class PoissonProblem:
    """Poisson-noise deconvolution sampled with AXDA + PnP-ULA / PSGLA."""

    def __init__(self, y, h, eta, rho1, rho2, kappa1, kappa2, alpha, eps, lam, gamma, seed,
                 net: Net | None = None, noise=True):
        self.y = _f64(y)
        self.h = _f64(h)
        self.net = net
        self.s = _Poisson(self.y.shape[0], self.y.shape[1], _dp(self.y), _dp(self.h),
                          self.h.shape[0], self.h.shape[1], float(eta), float(rho1), float(rho2),
                          float(kappa1), float(kappa2), float(alpha), float(eps), float(lam),
                          float(gamma), C.c_uint64(seed),
                          C.pointer(net.s) if net is not None else C.POINTER(_Net)(),
                          int(bool(noise)))

    @property
    def shape(self):
        return self.y.shape


def poisson_step(p: PoissonProblem, x, z1, z2, t: int, chain: int = 0):
    """-> (x+, z1+, z2+)."""
    x, z1, z2 = _f64(x), _f64(z1), _f64(z2)
    xn, z1n, z2n = np.empty_like(x), np.empty_like(x), np.empty_like(x)
    lib().ora_poisson_step(C.byref(p.s), _dp(x), _dp(z1), _dp(z2), t, chain, _dp(xn), _dp(z1n),
                           _dp(z2n))
    return xn, z1n, z2n


def moments_two_pass(samples):
    s = _f64(samples)
    n = s.shape[0]
    npix = int(np.prod(s.shape[1:]))
    mean = np.empty(s.shape[1:])
    var = np.empty(s.shape[1:])
    lib().ora_moments_two_pass(_dp(s), n, npix, _dp(mean), _dp(var))
    return mean, var


def final_moments(mean, m2, n):
    """MMSE = mean; var = M2 / (n - 1); std = sqrt(var)."""
    var = m2 / max(n - 1, 1)
    return mean, var, np.sqrt(var)


def psnr(xhat, xbar):
    """PSNR with peak 1 on the unclipped estimate."""
    mse = float(np.mean((np.asarray(xhat, np.float64) - xbar) ** 2))
    return 10.0 * np.log10(1.0 / mse)


class Ddfb:
    """DDFB denoiser: w [K][P][ks][ks] analysis filters, gamma [K] steps, ht the
    hard-tanh threshold."""

    def __init__(self, w, gamma, ht):
        self.w = _f64(w)
        self.gamma = _f64(gamma)
        self.K, self.P, self.ks = self.w.shape[0], self.w.shape[1], self.w.shape[2]
        self.s = _Ddfb(self.K, self.P, self.ks, _dp(self.w), _dp(self.gamma), float(ht))


def ddfb_W(v, wk):
    """W_k v for one layer's filters wk [P][ks][ks] -> [P][ny][nx]."""
    v, wk = _f64(v), _f64(wk)
    u = np.empty((wk.shape[0],) + v.shape)
    lib().ora_ddfb_W(_dp(v), v.shape[0], v.shape[1], _dp(wk), wk.shape[0], wk.shape[1], _dp(u))
    return u


def ddfb_Wt(u, wk):
    u, wk = _f64(u), _f64(wk)
    v = np.empty(u.shape[1:])
    lib().ora_ddfb_Wt(_dp(u), u.shape[1], u.shape[2], _dp(wk), wk.shape[0], wk.shape[1], _dp(v))
    return v


def ddfb_denoise(v, net: Ddfb):
    v = _f64(v)
    out = np.empty_like(v)
    lib().ora_ddfb_denoise(_dp(v), v.shape[0], v.shape[1], C.byref(net.s), _dp(out))
    return out
