"""Pins of the oracle's inpainting transition (Sec. IV-A: Gaussian noise,
H = diag(mask) with mask in {0, 1}), independent of the oracle's arithmetic:

* with noise, prior and projection off, every observed pixel follows
  x_t = y + (1 - gamma / sigma^2)^t (x_0 - y) and every unobserved pixel keeps
  x_0 (closed form of the scalar linear recursion);
* with the prior and projection off the chain is ULA on a product of
  independent scalar Gaussians: an observed pixel's stationary law is
  N(y, sigma^2 / (1 - gamma / (2 sigma^2))), an unobserved pixel is a random
  walk with variance 2 gamma t (moments over 4096 pixels);
* with a linear "denoiser" G = w (*) . the noise-free fixed point solves
  (M / sigma^2 + alpha W / eps^2) x = M y / sigma^2 (dense library solve, W
  from a library convolution), so treating a missing pixel as observed
  (or dropping the data term) moves it.
"""
import numpy as np
import torch
import torch.nn.functional as Fnn

import synth


def _mask(shape, frac, seed):
    return (np.random.default_rng(seed).random(shape) < frac).astype(np.float64)


def test_masked_recursion_closed_form(orc):
    ny, nx = 9, 11
    m = _mask((ny, nx), 0.3, 1)
    rng = np.random.default_rng(2)
    y = m * rng.uniform(0, 1, (ny, nx))
    x0 = rng.uniform(-0.5, 1.5, (ny, nx))
    sigma, gamma = 0.2, 0.01
    p = orc.Problem(y, None, sigma, alpha=0.0, eps=1.0, lam=0.0, gamma=gamma, seed=0, noise=False,
                    mask=m)
    x = x0.copy()
    for t in range(7):
        x = orc.langevin_step(p, x, t)
    q = (1 - gamma / sigma ** 2) ** 7
    expect = np.where(m > 0, y + q * (x0 - y), x0)
    np.testing.assert_allclose(x, expect, rtol=0, atol=1e-13)


def test_stationary_law_per_pixel(orc):
    ny, nx = 64, 128
    m = np.zeros((ny, nx))
    m[:, :64] = 1.0                      # left half observed, right half not
    c = 0.37
    y = m * c
    sigma = 0.1
    gamma = 0.4 * sigma ** 2             # gamma / sigma^2 = 0.4: fast mixing
    p = orc.Problem(y, None, sigma, alpha=0.0, eps=1.0, lam=0.0, gamma=gamma, seed=11, mask=m)
    T = 60
    x = np.zeros((ny, nx))
    for t in range(T):
        x = orc.langevin_step(p, x, t)
    obs, free = x[:, :64].ravel(), x[:, 64:].ravel()
    n = obs.size
    v_obs = sigma ** 2 / (1 - gamma / (2 * sigma ** 2))
    assert abs(obs.mean() - c) < 4 * np.sqrt(v_obs / n)
    assert abs(obs.var() / v_obs - 1) < 4 * np.sqrt(2 / n)
    v_free = 2 * gamma * T
    assert abs(free.mean()) < 4 * np.sqrt(v_free / n)
    assert abs(free.var() / v_free - 1) < 4 * np.sqrt(2 / n)


def test_masked_linear_prior_fixed_point(orc):
    ny, nx = 7, 6
    n = ny * nx
    m = _mask((ny, nx), 0.5, 3)
    w = np.array([[0, 1, 0], [1, 4, 1], [0, 1, 0]], dtype=np.float64)[None, None] / 8.0
    rng = np.random.default_rng(4)
    y = m * rng.random((ny, nx))
    sigma, alpha, eps = 0.2, 1.0, 0.3
    E = np.eye(n).reshape(n, ny, nx)
    Wm = Fnn.conv2d(torch.from_numpy(E[:, None]), torch.from_numpy(w), padding=1)[:, 0]
    Wm = Wm.numpy().reshape(n, n).T
    A = np.diag(m.ravel()) / sigma ** 2 + alpha / eps ** 2 * Wm
    xstar = np.linalg.solve(A, m.ravel() * y.ravel() / sigma ** 2).reshape(ny, nx)
    gamma = 1.0 / np.linalg.eigvalsh((A + A.T) / 2).max()
    net = orc.Net([w], [np.zeros(1)])
    p = orc.Problem(y, None, sigma, alpha=alpha, eps=eps, lam=0.0, gamma=gamma, seed=0, net=net,
                    noise=False, mask=m)
    got = orc.run_chain(p, np.zeros((ny, nx)), 6000, burn_in=6000)["x"]
    np.testing.assert_allclose(got, xstar, rtol=0, atol=1e-9)


def test_all_observed_mask_equals_identity_blur(orc):
    """mask = 1 everywhere is H = Id: the same chain as the 1 x 1 unit kernel."""
    rng = np.random.default_rng(6)
    y = rng.random((10, 12))
    kw = dict(alpha=0.0, eps=1.0, lam=0.1, gamma=0.004, seed=3)
    a = orc.Problem(y, np.ones((1, 1)), 0.2, **kw)
    b = orc.Problem(y, None, 0.2, mask=np.ones(y.shape), **kw)
    xa = xb = np.full(y.shape, 0.5)
    for t in range(5):
        xa, xb = orc.langevin_step(a, xa, t), orc.langevin_step(b, xb, t)
    np.testing.assert_array_equal(xa, xb)


def test_inpainting_inputs(orc):
    """Generator: 30 % observed, SNR from the observed pixels, y zero where
    unobserved; the initialisation interpolates y (equal at observed pixels)."""
    prob = synth.make_inpainting_problem(96, 80, 0.3, 15.0, 7)
    m = prob.mask > 0
    assert abs(m.mean() - 0.3) < 0.02
    assert not prob.y[~m].any()
    xo = prob.xbar[m]
    snr = 10 * np.log10(xo.var() / prob.sigma ** 2)
    assert abs(snr - 15.0) < 1e-5
    np.testing.assert_allclose(prob.x0[m], prob.y[m], rtol=0, atol=1e-6)
    assert np.isfinite(prob.x0).all()
