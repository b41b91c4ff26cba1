"""Pins for the oracle's PnP-ULA transition (Eq. 8, x-update of Algorithm 1),
its step sizes (Eq. 10) and its moment accumulation.

Each term of the update is pinned by a closed form that does not reuse the
oracle's own code:
  * likelihood gradient: with the noise, prior and projection off the chain is
    the linear recursion x+ = x - gamma (Q x - b), Q = H^T H / sigma^2, solved
    per DFT frequency;
  * noise term: with the prior and projection off the chain is ULA on a
    Gaussian whose stationary law is N(mu, S), S = Q^-1 (I - gamma Q / 2)^-1,
    diagonal in the DFT basis (Monte Carlo over independent chains);
  * projection term: the deterministic iteration is gradient descent on
    f + dist^2(., C) / (2 lambda) whose minimiser is known per pixel;
  * prior term: a linear "denoiser" G = w (*) . gives the fixed point
    (Q + alpha W / eps^2) x = b, solved with a dense library solver, W built
    from a library convolution.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import synth


def kernel_dft(h, shape):
    ny, nx = shape
    kh, kw = h.shape
    hp = np.zeros(shape)
    for a in range(kh):
        for b in range(kw):
            hp[(a - kh // 2) % ny, (b - kw // 2) % nx] += h[a, b]
    return np.fft.fft2(hp)


WELL_CONDITIONED = np.array([[0.0, 0.1, 0.0], [0.1, 0.6, 0.1], [0.0, 0.1, 0.0]])


def test_gradient_recursion_closed_form(orc):
    ny, nx = 12, 10
    h = synth.motion_kernel(5, 0.4)
    rng = np.random.default_rng(0)
    y = rng.random((ny, nx))
    x0 = rng.random((ny, nx))
    sigma, gamma, T = 0.2, 0.01, 40
    p = orc.Problem(y, h, sigma, alpha=0.0, eps=1.0, lam=0.0, gamma=gamma, seed=1, noise=False)
    got = orc.run_chain(p, x0, T, burn_in=T)["x"]
    Hf = kernel_dft(h, (ny, nx))
    a = 1.0 - gamma * np.abs(Hf) ** 2 / sigma ** 2
    c = gamma * np.conj(Hf) * np.fft.fft2(y) / sigma ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        geo = np.where(np.abs(1 - a) > 1e-14, (1 - a ** T) / (1 - a), T)
    xt = np.real(np.fft.ifft2(a ** T * np.fft.fft2(x0) + geo * c))
    np.testing.assert_allclose(got, xt, rtol=0, atol=1e-11)


@pytest.mark.slow
def test_stationary_law_of_gaussian_ula(orc):
    ny = nx = 8
    h = WELL_CONDITIONED
    rng = np.random.default_rng(42)
    y = rng.random((ny, nx))
    sigma = 0.1
    gamma = 0.5 * sigma ** 2
    p = orc.Problem(y, h, sigma, alpha=0.0, eps=1.0, lam=0.0, gamma=gamma, seed=2024, noise=True)
    chains, T = 1024, 600   # slowest mode contracts by 0.98 per step
    xs = np.stack([orc.run_chain(p, np.zeros((ny, nx)), T, burn_in=T, chain=c)["x"]
                   for c in range(chains)])
    Hf = kernel_dft(h, (ny, nx))
    q = np.abs(Hf) ** 2 / sigma ** 2
    mu = np.real(np.fft.ifft2(np.conj(Hf) * np.fft.fft2(y) / sigma ** 2 / q))
    s = 1.0 / (q * (1 - gamma * q / 2))                  # eigenvalues of S
    cov0 = np.real(np.fft.ifft2(s))                        # cov[x_i, x_{i+k}] = cov0[k]
    # the mean: within 4 standard errors per pixel
    se = np.sqrt(cov0[0, 0] / chains)
    assert np.abs(xs.mean(0) - mu).max() < 4.5 * se
    # the variance and the first off-diagonals: within 5 standard errors
    d = xs - mu
    v = (d ** 2).mean(0)
    assert np.abs(v - cov0[0, 0]).max() < 5 * cov0[0, 0] * np.sqrt(2 / chains)
    c01 = (d * np.roll(d, -1, axis=2)).mean(0)
    se01 = np.sqrt((cov0[0, 0] ** 2 + cov0[0, 1] ** 2) / chains)
    assert np.abs(c01 - cov0[0, 1]).max() < 5 * se01
    # chi-square aggregate: chains * e^T S^-1 e ~ chi2(N) for the mean error e
    n = ny * nx
    idx = np.arange(n)
    di = (idx[None, :] // nx - idx[:, None] // nx) % ny
    dj = (idx[None, :] % nx - idx[:, None] % nx) % nx
    S = cov0[di, dj]
    e = (xs.mean(0) - mu).ravel()
    chi2 = chains * e @ np.linalg.solve(S, e)
    assert n - 5 * np.sqrt(2 * n) < chi2 < n + 5 * np.sqrt(2 * n)


def test_projection_term_fixed_point(orc):
    """H = Id: minimiser of (x-y)^2/(2 sigma^2) + dist^2(x, [0,1])/(2 lambda)."""
    rng = np.random.default_rng(5)
    y = rng.uniform(-0.8, 1.8, (6, 7))
    sigma, lam = 0.3, 0.05
    gamma = 0.5 / (1 / sigma ** 2 + 1 / lam)
    p = orc.Problem(y, np.ones((1, 1)), sigma, alpha=0.0, eps=1.0, lam=lam, gamma=gamma, seed=0,
                    noise=False)
    got = orc.run_chain(p, np.full(y.shape, 0.5), 400, burn_in=400)["x"]
    w = 1 / sigma ** 2
    expect = np.where(y > 1, (w * y + 1 / lam) / (w + 1 / lam),
                      np.where(y < 0, w * y / (w + 1 / lam), y))
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12)


def test_linear_prior_fixed_point(orc):
    """One linear layer G v = w (*) v (zero padding): the prior term is -(alpha/eps^2) W x."""
    ny, nx = 7, 6
    n = ny * nx
    h = WELL_CONDITIONED
    w = np.array([[0, 1, 0], [1, 4, 1], [0, 1, 0]], dtype=np.float64)[None, None] / 8.0
    rng = np.random.default_rng(9)
    y = rng.random((ny, nx))
    sigma, alpha, eps = 0.2, 1.0, 0.3
    # dense matrices from independent implementations
    E = np.eye(n).reshape(n, ny, nx)
    Hm = np.stack([synth.fft_circular_blur(e, h).ravel() for e in E], axis=1)
    Wm = Fnn.conv2d(torch.from_numpy(E[:, None]), torch.from_numpy(w), padding=1)[:, 0]
    Wm = Wm.numpy().reshape(n, n).T
    A = Hm.T @ Hm / sigma ** 2 + alpha / eps ** 2 * Wm
    xstar = np.linalg.solve(A, Hm.T @ y.ravel() / sigma ** 2).reshape(ny, nx)
    gamma = 1.0 / np.linalg.eigvalsh((A + A.T) / 2).max()
    net = orc.Net([w], [np.zeros(1)])
    p = orc.Problem(y, h, sigma, alpha=alpha, eps=eps, lam=0.0, gamma=gamma, seed=0, net=net,
                    noise=False)
    got = orc.run_chain(p, np.zeros((ny, nx)), 3000, burn_in=3000)["x"]
    np.testing.assert_allclose(got, xstar, rtol=0, atol=1e-9)


def test_welford_matches_two_pass_and_library(orc):
    d = synth.denoiser_weights(2, 4, seed=2)
    y = synth.ground_truth(9, 11, seed=1)
    h = synth.gaussian_kernel(5, 1.0)
    lam, gam = orc.stepsizes(1.0, 0.05, 1.0, 0.05, 0.9)
    p = orc.Problem(y, h, 0.05, 1.0, 0.05, lam, gam, seed=3, net=orc.Net.from_weights(d))
    res = orc.run_chain(p, np.zeros_like(y), 30, burn_in=10, store_samples=True)
    assert res["n"] == 20
    m2p, v2p = orc.moments_two_pass(res["samples"])
    np.testing.assert_allclose(res["mean"], m2p, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(res["m2"] / (res["n"] - 1), v2p, rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(m2p, res["samples"].mean(0), rtol=1e-12)
    np.testing.assert_allclose(v2p, res["samples"].var(0, ddof=1), rtol=1e-9, atol=1e-16)
    np.testing.assert_array_equal(res["samples"][-1], res["x"])


def test_chain_resume_is_exact(orc):
    """Counter-based draws make a chain split in two runs equal the single run."""
    y = synth.ground_truth(8, 8, seed=4)
    h = synth.uniform_kernel(3)
    lam, gam = orc.stepsizes(1.0, 0.1, 0.0, 1.0, 0.0)
    p = orc.Problem(y, h, 0.1, 0.0, 1.0, lam, gam, seed=77)
    full = orc.run_chain(p, np.zeros_like(y), 12, burn_in=0)["x"]
    half = orc.run_chain(p, np.zeros_like(y), 5, burn_in=0)["x"]
    rest = orc.run_chain(p, half, 7, burn_in=0, t0=5)["x"]
    np.testing.assert_array_equal(full, rest)


@pytest.mark.parametrize("hnorm,sigma,alpha,eps,lip", [
    (1.0, 0.01, 1.0, 0.01, 0.9), (1.0, 0.1, 0.0, 1.0, 0.9), (0.7, 0.03, 2.0, 0.05, 3.0)])
def test_stepsizes_satisfy_conditions(orc, hnorm, sigma, alpha, eps, lip):
    """Eq. 10 with H_2 = 0: 2L + a L_eps/eps^2 <= 1/(2 lambda) and
    3 gamma (L + 1/lambda + a L_eps/eps^2) < 1, with L = ||H||^2 / sigma^2."""
    lam, gam = orc.stepsizes(hnorm, sigma, alpha, eps, lip)
    L = hnorm ** 2 / sigma ** 2
    prior = alpha * lip / eps ** 2
    assert 2 * L + prior <= 1 / (2 * lam)
    assert 3 * gam * (L + 1 / lam + prior) < 1
    # the paper's factor 0.99 in both rules
    assert abs(lam * (4 * L + 2 * prior) - 0.99) < 1e-12
    assert abs(3 * gam * (L + 1 / lam + prior) - 0.99) < 1e-12
