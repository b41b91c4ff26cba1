"""Seeded synthetic workloads for the PnP-ULA Gaussian-deconvolution sampler.

This module only *makes inputs*: ground-truth images, blur kernels, noisy
observations, denoiser weights and the per-workload parameters. It holds none
of the sampler's arithmetic (no Langevin step, no denoiser evaluation, no
step-size rule) and it is shared by the FP64 oracle and the CUDA path, which
otherwise share no code.

Stand-ins for the paper's data (Sec. III-A): the pixabay crops, ImageNet /
DIV2K patches and the trained DnCNN/DDFB weights are not available, so

* ground truth = random ellipses on a 0.5 base plus a smooth Gaussian random
  field, clipped to C = [0, 1]^N (the paper normalises its crops into C);
* blur = normalised Gaussian, uniform or motion kernels (Sec. III-A2 uses a
  normalised motion blur);
* observation y = h (*) xbar + sigma * w with circular boundary, sigma set from
  the blurred-signal SNR (BSNR);
* denoiser = DnCNN form (Sec. II-B, Example "DnCNN") with He-normal weights,
  each layer rescaled by its spectral norm so that the product of the layer
  norms, an upper bound of the Lipschitz constant L_eps of Id - D_eps, is 0.9.

The blurred image used to synthesise y is computed here with numpy's FFT; this
is the data-generating forward model, implemented independently of both the
oracle (direct circular sums) and the CUDA stencil.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------


def ground_truth(ny: int, nx: int, seed: int, n_ellipses: tuple = (8, 32)) -> np.ndarray:
    """Natural-like image in [0,1]: ellipses + smooth Gaussian random field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    img = np.full((ny, nx), 0.5, dtype=np.float64)
    n = int(rng.integers(n_ellipses[0], n_ellipses[1] + 1))
    size = min(ny, nx)
    for _ in range(n):
        cy, cx = rng.uniform(0, ny), rng.uniform(0, nx)
        a, b = rng.uniform(0.02, 0.25, size=2) * size
        th = rng.uniform(0, math.pi)
        amp = rng.uniform(-0.5, 0.5)
        r = max(a, b)
        y0, y1 = max(0, int(cy - r) - 1), min(ny, int(cy + r) + 2)
        x0, x1 = max(0, int(cx - r) - 1), min(nx, int(cx + r) + 2)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        dy, dx = yy - cy, xx - cx
        u = dx * math.cos(th) + dy * math.sin(th)
        v = -dx * math.sin(th) + dy * math.cos(th)
        inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        img[y0:y1, x0:x1] += amp * inside
    # smooth Gaussian random field: white noise low-passed by a Gaussian of std N/16
    w = rng.standard_normal((ny, nx))
    s = size / 16.0
    fy = np.fft.fftfreq(ny)[:, None]
    fx = np.fft.rfftfreq(nx)[None, :]
    filt = np.exp(-2.0 * (math.pi * s) ** 2 * (fy ** 2 + fx ** 2))
    f = np.fft.irfft2(np.fft.rfft2(w) * filt, s=(ny, nx))
    sd = f.std()
    if sd > 0:
        img += 0.1 * f / sd
    return np.clip(img, 0.0, 1.0)


# --------------------------------------------------------------------------
# blur kernels (odd L x L, anchored at the centre)
# --------------------------------------------------------------------------


def gaussian_kernel(L: int, s: float) -> np.ndarray:
    r = L // 2
    u = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2.0 * s * s))
    return k / k.sum()


def uniform_kernel(L: int) -> np.ndarray:
    return np.full((L, L), 1.0 / (L * L))


def motion_kernel(L: int, angle: float) -> np.ndarray:
    """Segment of length L through the centre, bilinear splat of 4L points."""
    k = np.zeros((L, L))
    r = L // 2
    ts = np.linspace(-(L - 1) / 2.0, (L - 1) / 2.0, 4 * L)
    for t in ts:
        py, px = r + t * math.sin(angle), r + t * math.cos(angle)
        iy, ix = int(math.floor(py)), int(math.floor(px))
        fy, fx = py - iy, px - ix
        for yy, xx, wgt in ((iy, ix, (1 - fy) * (1 - fx)), (iy + 1, ix, fy * (1 - fx)),
                            (iy, ix + 1, (1 - fy) * fx), (iy + 1, ix + 1, fy * fx)):
            if 0 <= yy < L and 0 <= xx < L:
                k[yy, xx] += wgt
    return k / k.sum()


# --------------------------------------------------------------------------
# observation
# --------------------------------------------------------------------------


def fft_circular_blur(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Data-generating forward model: circular convolution via the DFT."""
    ny, nx = x.shape
    kh, kw = h.shape
    hp = np.zeros((ny, nx))
    for a in range(kh):
        for b in range(kw):
            hp[(a - kh // 2) % ny, (b - kw // 2) % nx] += h[a, b]
    return np.real(np.fft.ifft2(np.fft.fft2(x) * np.fft.fft2(hp)))


def sigma_for_bsnr(hx: np.ndarray, bsnr_db: float) -> float:
    """BSNR = 10 log10(var(Hx) / sigma^2), var mean-removed."""
    return float(math.sqrt(np.var(hx) / (10.0 ** (bsnr_db / 10.0))))


def observation(xbar: np.ndarray, h: np.ndarray, bsnr_db: float, seed: int):
    hx = fft_circular_blur(xbar, h)
    sigma = sigma_for_bsnr(hx, bsnr_db)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    y = hx + sigma * rng.standard_normal(xbar.shape)
    return y, sigma


# --------------------------------------------------------------------------
# denoiser weights (DnCNN form: 1 -> F -> ... -> F -> 1, 3x3, ReLU but last)
# --------------------------------------------------------------------------


def conv_layer_spectral_norm(w: np.ndarray, grid: int = 64) -> float:
    """Largest singular value of a multi-channel 2-D convolution.

    The transfer matrix at frequency (u, v) is sum_{a,b} w[:, :, a, b] e^{-2 pi i (u a + v b)/n}
    (Sedghi, Gupta & Long, ICLR 2019); the operator norm is its largest
    singular value maximised over frequencies, sampled on a grid x grid lattice.
    """
    cout, cin, kh, kw = w.shape
    f = np.arange(grid) / grid
    ea = np.exp(-2j * math.pi * np.outer(f, np.arange(kh)))   # [grid, kh]
    eb = np.exp(-2j * math.pi * np.outer(f, np.arange(kw)))   # [grid, kw]
    P = np.einsum("oiab,ua,vb->uvoi", w.astype(np.complex128), ea, eb)
    s = np.linalg.svd(P.reshape(grid * grid, cout, cin), compute_uv=False)
    return float(s.max())


@dataclass
class DenoiserWeights:
    K: int
    F: int
    weights: list = field(default_factory=list)   # K arrays [cout, cin, 3, 3] float64
    biases: list = field(default_factory=list)    # K arrays [cout] float64
    lipschitz: float = 0.9

    def channels(self):
        cin = [1] + [self.F] * (self.K - 1)
        cout = [self.F] * (self.K - 1) + [1]
        return cin, cout

    def flat(self, dtype=np.float32):
        w = np.concatenate([a.ravel() for a in self.weights]).astype(dtype)
        b = np.concatenate([a.ravel() for a in self.biases]).astype(dtype)
        return w, b


def denoiser_weights(K: int, F: int, seed: int, lipschitz: float = 0.9,
                     bias_std: float = 0.01) -> DenoiserWeights:
    rng = np.random.Generator(np.random.PCG64(seed))
    d = DenoiserWeights(K=K, F=F, lipschitz=lipschitz)
    cin, cout = d.channels()
    per_layer = lipschitz ** (1.0 / K)
    for k in range(K):
        w = rng.standard_normal((cout[k], cin[k], 3, 3)) * math.sqrt(2.0 / (cin[k] * 9))
        s = conv_layer_spectral_norm(w)
        w = w * (per_layer / s)
        # round through float32 so the oracle and the GPU use the same numbers
        w = w.astype(np.float32).astype(np.float64)
        b = (rng.standard_normal(cout[k]) * bias_std).astype(np.float32).astype(np.float64)
        d.weights.append(w)
        d.biases.append(b)
    return d


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------


@dataclass
class Problem:
    """One Gaussian-deconvolution sampling problem (inputs only)."""
    xbar: np.ndarray           # ground truth [ny, nx] float64
    y: np.ndarray              # observation  [ny, nx] float64 (stored as float32-exact values)
    h: np.ndarray              # blur kernel  [kh, kw] float64 (float32-exact)
    sigma: float
    seed: int                  # chain seed (Philox key)
    blocks: tuple = (1, 1)
    halo: int = 0
    T: int = 0
    burn_in: int = 0
    name: str = ""

    @property
    def shape(self):
        return self.y.shape


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def make_problem(ny, nx, h, bsnr_db, gt_seed, name="", blocks=(1, 1), halo=0, T=0, burn_in=0):
    xbar = ground_truth(ny, nx, gt_seed)
    h = _f32(h)
    h = h / h.sum()
    h = _f32(h)
    y, sigma = observation(xbar, h, bsnr_db, gt_seed)
    return Problem(xbar=xbar, y=_f32(y), h=h, sigma=float(np.float32(sigma)), seed=gt_seed,
                   blocks=blocks, halo=halo, T=T, burn_in=burn_in, name=name)


@dataclass
class PoissonProblem:
    """One Poisson-noise deconvolution problem (inputs only): y ~ Poisson(eta H xbar)."""
    xbar: np.ndarray           # ground truth [ny, nx] float64
    y: np.ndarray              # photon counts [ny, nx] float64 (integers)
    h: np.ndarray              # blur kernel  [kh, kw] float64 (float32-exact)
    eta: float
    seed: int                  # chain seed (Philox key)

    @property
    def shape(self):
        return self.y.shape


def make_poisson_problem(ny, nx, h, eta, gt_seed):
    """Counts y ~ Poisson(eta H xbar) (seeded numpy PCG64) for the synthetic
    ground truth; the paper uses eta = 250 with the Gaussian-case blur."""
    xbar = ground_truth(ny, nx, gt_seed)
    h = _f32(h)
    h = _f32(h / h.sum())
    hx = np.maximum(fft_circular_blur(xbar, h), 0.0)
    rng = np.random.Generator(np.random.PCG64(gt_seed + 104729))
    y = rng.poisson(eta * hx).astype(np.float64)
    return PoissonProblem(xbar=xbar, y=y, h=h, eta=float(eta), seed=gt_seed)


@dataclass
class InpaintingProblem:
    """One Gaussian-noise inpainting problem (inputs only): y = M (xbar + sigma w)."""
    xbar: np.ndarray           # ground truth [ny, nx] float64
    mask: np.ndarray           # 1 observed / 0 missing [ny, nx] float64
    y: np.ndarray              # observation, 0 where missing [ny, nx] float64 (float32-exact)
    sigma: float
    x0: np.ndarray             # chain initialisation: spline interpolant of y (float32-exact)
    seed: int                  # chain seed (Philox key)

    @property
    def shape(self):
        return self.y.shape


def spline_init(y, mask):
    """Initial state for inpainting: the piecewise-cubic (Clough-Tocher) scattered-
    data interpolant of the observed pixels (scipy.interpolate.griddata), nearest
    observed value outside their convex hull. It is the chain's starting point,
    an input to the sampler, not part of its transition."""
    from scipy.interpolate import griddata
    ny, nx = y.shape
    pts = np.argwhere(mask > 0)
    vals = y[mask > 0]
    gi, gj = np.mgrid[0:ny, 0:nx]
    x0 = griddata(pts, vals, (gi, gj), method="cubic")
    bad = ~np.isfinite(x0)
    if bad.any():
        x0[bad] = griddata(pts, vals, (gi[bad], gj[bad]), method="nearest")
    return x0


def make_inpainting_problem(ny, nx, frac, snr_db, gt_seed):
    """A random mask keeping a fraction `frac` of the pixels (the paper keeps
    M = 0.3 N), noise level from the input SNR over the observed pixels:
    SNR = 10 log10(var(xbar[observed]) / sigma^2) (15 dB in the paper)."""
    xbar = ground_truth(ny, nx, gt_seed)
    rng = np.random.Generator(np.random.PCG64(gt_seed + 7919))
    mask = (rng.random((ny, nx)) < frac).astype(np.float64)
    sigma = float(np.float32(math.sqrt(xbar[mask > 0].var() / 10 ** (snr_db / 10))))
    y = _f32(mask * (xbar + sigma * rng.standard_normal((ny, nx))))
    x0 = _f32(spline_init(y, mask))
    return InpaintingProblem(xbar=xbar, mask=mask, y=y, sigma=sigma, x0=x0, seed=gt_seed)


def gt_seed(config: int, job: int = 0) -> int:
    return 1000 + config * 100 + job


# The five workloads. Sizes, blurs, BSNRs and denoiser shapes follow the
# sampler's published setting scaled to grayscale synthetic images.
WORKLOADS = {
    1: dict(name="deconv128_gauss7_K4F16", ny=128, nx=128, blur=("gaussian", 7, 1.5), bsnr=30.0,
            K=4, F=16, blocks=(2, 2), halo=4, T=64, burn_in=16),
    2: dict(name="deconv1024_unif9_K8F64", ny=1024, nx=1024, blur=("uniform", 9, None), bsnr=20.0,
            K=8, F=64, blocks=(4, 4), halo=8, T=2000, burn_in=500),
    3: dict(name="deconv8192_gauss13_K8F64", ny=8192, nx=8192, blur=("gaussian", 13, 3.0), bsnr=30.0,
            K=8, F=64, blocks=(16, 16), halo=8, T=1000, burn_in=200),
    # the paper's Gaussian-deconvolution scale: normalised motion blur whose
    # size grows with the image (65^2 at 2048^2, 129^2 at 4096^2), 25 dB
    6: dict(name="deconv2048_motion65_K8F64", ny=2048, nx=2048, blur=("motion", 65, 0.9),
            bsnr=25.0, K=8, F=64, blocks=(8, 8), halo=8, T=1000, burn_in=200),
    7: dict(name="deconv4096_motion129_K8F64", ny=4096, nx=4096, blur=("motion", 129, 0.9),
            bsnr=25.0, K=8, F=64, blocks=(16, 16), halo=8, T=1000, burn_in=200),
}


def blur_from_spec(spec, seed=0):
    kind, L, p = spec
    if kind == "gaussian":
        return gaussian_kernel(L, p)
    if kind == "uniform":
        return uniform_kernel(L)
    if kind == "motion":
        return motion_kernel(L, p if p is not None else
                             np.random.Generator(np.random.PCG64(seed)).uniform(0, math.pi))
    raise ValueError(kind)


def workload_problem(config: int, job: int = 0, shrink: int = 1) -> Problem:
    """Problem of workload `config` (1..3, 6, 7); `shrink` divides the image size."""
    w = WORKLOADS[config]
    h = blur_from_spec(w["blur"])
    return make_problem(w["ny"] // shrink, w["nx"] // shrink, h, w["bsnr"], gt_seed(config, job),
                        name=w["name"], blocks=w["blocks"], halo=w["halo"], T=w["T"],
                        burn_in=w["burn_in"])


def workload_denoiser(config: int) -> DenoiserWeights:
    w = WORKLOADS.get(config, WORKLOADS[2])
    return denoiser_weights(w["K"], w["F"], seed=77 + w["K"] * 1000 + w["F"])


@dataclass
class DdfbWeights:
    filters: np.ndarray      # [K][P][3][3] float64 (float32-exact)
    gammas: np.ndarray       # [K]
    ht: float


def ddfb_weights(K: int, P: int, seed: int, ht: float = 0.05) -> DdfbWeights:
    """Seeded DDFB parameters: zero-mean 3 x 3 analysis filters (high-pass, as
    a learned sparsifying frame) with the layer operator norm ||W_k|| = 1
    computed from the DFT of the filters, and steps gamma_k = 1.8 inside
    (0, 2 / ||W_k||^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.standard_normal((K, P, 3, 3))
    f -= f.mean(axis=(2, 3), keepdims=True)
    for k in range(K):
        # ||W_k||^2 = max over frequencies of sum_p |DFT(w_p)|^2 (1 -> P channels)
        pad = np.zeros((P, 64, 64))
        pad[:, :3, :3] = f[k]
        nrm = math.sqrt(float((np.abs(np.fft.fft2(pad)) ** 2).sum(axis=0).max()))
        f[k] /= nrm
    return DdfbWeights(filters=_f32(f), gammas=np.full(K, 1.8), ht=float(ht))


def random_blur(rng: np.random.Generator):
    """Blur mix of the batched/serving workloads: uniform 5-15 px, Gaussian
    sigma 1-4, or a 1-D motion kernel of length 9-21 (odd sizes)."""
    kind = int(rng.integers(0, 3))
    if kind == 0:
        L = int(rng.choice([5, 7, 9, 11, 13, 15]))
        return uniform_kernel(L), ("uniform", L, None)
    if kind == 1:
        s = float(rng.uniform(1.0, 4.0))
        L = min(21, 2 * int(math.ceil(2.5 * s)) + 1)
        return gaussian_kernel(L, s), ("gaussian", L, s)
    L = int(rng.choice([9, 11, 13, 15, 17, 19, 21]))
    ang = float(rng.uniform(0, math.pi))
    return motion_kernel(L, ang), ("motion", L, ang)


def batched_problems(n: int = 48, seed: int = 4000, lo: int = 256, hi: int = 2048,
                     size_quantum: int = 1):
    """Independent problems with sizes log-uniform in [lo, hi] (batched workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(n):
        s = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        s = max(lo, (s // size_quantum) * size_quantum)
        h, spec = random_blur(rng)
        bsnr = float(rng.uniform(15.0, 40.0))
        p = make_problem(s, s, h, bsnr, gt_seed(4, j), name=f"job{j}_{s}_{spec[0]}{spec[1]}")
        out.append(p)
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 5000):
    """Arrival times (s) of a Poisson stream (serving workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def serving_jobs(n: int = 64, seed: int = 5000, sizes=(512, 1024, 2048, 4096)):
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    jobs = []
    for j in range(n):
        s = int(rng.choice(sizes))
        h, spec = random_blur(rng)
        bsnr = float(rng.uniform(15.0, 40.0))
        jobs.append(dict(size=s, h=h, spec=spec, bsnr=bsnr, gt_seed=gt_seed(5, j)))
    return jobs
