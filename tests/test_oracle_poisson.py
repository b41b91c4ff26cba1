"""Pins of the oracle's Poisson-noise sampler (Poisson deconvolution of
Sec. IV-A with the AXDA split and the PnP-ULA / PSGLA transitions of Eqs.
13-14), independent of the oracle's own arithmetic:

* the closed-form prox of kappa KL(y || .) against scalar numerical
  minimisation (scipy), including y = 0 and arguments below kappa;
* the extra Philox streams (counter word 3) for zeta_1, zeta_2: stream 0 is
  the x-update's stream, the others are standard normal and uncorrelated;
* the step sizes of the paper's Poisson setting satisfy Eq. 12;
* with noise, denoiser and projection off, the iteration is a gradient step
  in x and a proximal-gradient step in z on
      Phi(x, z) = KL(y || z1) + iota_{R+}(z2) + |z1 - eta H x|^2 / (2 rho1)
                  + |z2 - x|^2 / (2 rho2),
  so its fixed point is Phi's minimiser, computed here by L-BFGS-B with an
  FFT forward model (a dropped term, a wrong sign or a transposed H moves it).
"""
import numpy as np
import pytest

import synth

scipy_opt = pytest.importorskip("scipy.optimize")


def test_kl_prox_minimises_the_scalar_objective(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        v = rng.uniform(-20, 300)
        y = float(rng.integers(0, 300)) if rng.random() > 0.1 else 0.0
        kappa = rng.uniform(1e-3, 20)
        u = orc.kl_prox(v, y, kappa)
        if y == 0.0:
            ref = max(v - kappa, 0.0)
        else:
            obj = lambda w: kappa * (w - y * np.log(w)) + 0.5 * (w - v) ** 2
            res = scipy_opt.minimize_scalar(obj, bounds=(1e-12, max(v, 0) + kappa + y + 10),
                                            method="bounded", options={"xatol": 1e-12})
            ref = res.x
        assert u >= 0.0
        assert abs(u - ref) <= 1e-6 * max(1.0, abs(ref)), (v, y, kappa, u, ref)


def test_noise_streams(orc):
    n = 40000
    s0 = orc.normals_stream(77, 5, 2, 0, n)
    np.testing.assert_array_equal(s0, orc.normals(77, 5, 2, n))
    s1 = orc.normals_stream(77, 5, 2, 1, n)
    s2 = orc.normals_stream(77, 5, 2, 2, n)
    for s in (s1, s2):
        assert abs(s.mean()) < 4 / np.sqrt(n)
        assert abs(s.var() - 1) < 4 * np.sqrt(2 / n)
    for a, b in ((s0, s1), (s0, s2), (s1, s2)):
        assert abs(np.corrcoef(a, b)[0, 1]) < 4 / np.sqrt(n)


def test_poisson_stepsizes_satisfy_the_conditions(orc):
    for hnorm, eta, rho1, rho2, L in [(1.0, 250.0, 10.0, 1e-3, 0.9), (1.0, 5.0, 1.0, 0.5, 0.9),
                                      (0.8, 30.0, 2.0, 0.1, 0.5)]:
        alpha, eps = 1.0, 0.05
        lam, gam, k1, k2 = orc.poisson_stepsizes(hnorm, eta, rho1, rho2, alpha, eps, L)
        h2 = (eta * hnorm) ** 2 / rho1 + 1.0 / rho2      # ||H2||^2 of the scaled coupling
        prior = alpha * L / eps ** 2
        assert 2 * h2 + prior <= 1 / (2 * lam) * (1 + 1e-12)
        assert 3 * gam * (h2 + 1 / lam + prior) < 1
        assert 0 < k1 < rho1 and 0 < k2 < rho2


def _fft_ops(h, ny, nx):
    hp = np.zeros((ny, nx))
    kh, kw = h.shape
    for a in range(kh):
        for b in range(kw):
            hp[(a - kh // 2) % ny, (b - kw // 2) % nx] += h[a, b]
    F = np.fft.fft2(hp)
    Hf = lambda v: np.real(np.fft.ifft2(np.fft.fft2(v) * F))
    Ht = lambda v: np.real(np.fft.ifft2(np.fft.fft2(v) * np.conj(F)))
    return Hf, Ht


def test_noise_free_fixed_point_is_the_augmented_minimiser(orc):
    ny = nx = 6
    # a mild blur (DFT magnitudes in [0.6, 1]) keeps the deconvolution well
    # conditioned, so the noise-free iteration converges within the loop
    h = np.full((3, 3), 0.025)
    h[1, 1] = 0.8
    eta, rho1, rho2 = 4.0, 1.0, 0.5
    rng = np.random.default_rng(3)
    xbar = rng.uniform(0.3, 1.0, (ny, nx))
    Hf, Ht = _fft_ops(h, ny, nx)
    y = rng.poisson(eta * Hf(xbar)).astype(np.float64)
    # isolated zero counts between bright pixels: the unconstrained
    # deconvolution goes negative there, so the R+ constraint on z2 and the
    # balance of the two coupling gradients both shape the minimiser
    y[1, 1] = y[4, 2] = y[2, 4] = 0.0
    lam, gam, k1, k2 = orc.poisson_stepsizes(1.0, eta, rho1, rho2, 0.0, 1.0, 0.0)
    p = orc.PoissonProblem(y, h, eta, rho1, rho2, k1, k2, 0.0, 1.0, -1.0, gam, 9, noise=False)
    x = np.full((ny, nx), 0.5)
    z1 = eta * Hf(x)
    z2 = x.copy()
    for t in range(20000):
        x, z1, z2 = orc.poisson_step(p, x, z1, z2, t)

    n = ny * nx

    def phi(v):
        xv, a, b = v[:n].reshape(ny, nx), v[n:2 * n].reshape(ny, nx), v[2 * n:].reshape(ny, nx)
        r1 = a - eta * Hf(xv)
        f = np.sum(a - y * np.log(a)) + np.sum(r1 ** 2) / (2 * rho1) + np.sum((b - xv) ** 2) / (2 * rho2)
        gx = -(eta / rho1) * Ht(r1) - (b - xv) / rho2
        ga = 1 - y / a + r1 / rho1
        gb = (b - xv) / rho2
        return f, np.concatenate([gx.ravel(), ga.ravel(), gb.ravel()])

    v0 = np.concatenate([np.full(n, 0.5), np.full(n, eta * 0.5), np.full(n, 0.5)])
    bounds = [(None, None)] * n + [(1e-9, None)] * n + [(0.0, None)] * n
    res = scipy_opt.minimize(phi, v0, jac=True, method="L-BFGS-B", bounds=bounds,
                             options={"ftol": 1e-15, "gtol": 1e-11, "maxiter": 20000})
    xs = res.x[:n].reshape(ny, nx)
    z1s = res.x[n:2 * n].reshape(ny, nx)
    z2s = res.x[2 * n:].reshape(ny, nx)
    assert np.abs(x - xs).max() <= 1e-5 * np.abs(xs).max()
    assert np.abs(z1 - z1s).max() <= 1e-5 * np.abs(z1s).max()
    assert np.abs(z2 - z2s).max() <= 1e-5 * max(np.abs(z2s).max(), 1.0)
