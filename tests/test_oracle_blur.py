"""Pins for the oracle's blur operator H and its adjoint H^T (Sec. III-A2).

H is a circular 2-D convolution; the pins are the DFT convolution theorem
(numpy.fft, a library routine), the adjoint identity, shift kernels (which fix
convolution vs correlation) and the operator norm of a normalised
non-negative kernel.
"""
import numpy as np
import pytest

import synth


def fft_conv(x, h, adjoint=False):
    ny, nx = x.shape
    kh, kw = h.shape
    hp = np.zeros((ny, nx))
    for a in range(kh):
        for b in range(kw):
            hp[(a - kh // 2) % ny, (b - kw // 2) % nx] += h[a, b]
    H = np.fft.fft2(hp)
    if adjoint:
        H = np.conj(H)
    return np.real(np.fft.ifft2(np.fft.fft2(x) * H))


SHAPES = [(8, 8, 3, 3), (7, 13, 5, 5), (16, 9, 7, 3), (5, 5, 9, 9), (1, 6, 1, 3), (32, 24, 13, 13)]


@pytest.mark.parametrize("ny,nx,kh,kw", SHAPES)
def test_blur_matches_dft_convolution(orc, ny, nx, kh, kw):
    rng = np.random.default_rng(ny * 100 + nx)
    x = rng.standard_normal((ny, nx))
    h = rng.standard_normal((kh, kw))           # not symmetric: fixes the orientation
    np.testing.assert_allclose(orc.blur(x, h), fft_conv(x, h), rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.blur_adj(x, h), fft_conv(x, h, adjoint=True), rtol=0, atol=1e-12)


@pytest.mark.parametrize("ny,nx,kh,kw", SHAPES)
def test_adjoint_identity(orc, ny, nx, kh, kw):
    rng = np.random.default_rng(7 + ny + nx)
    x = rng.standard_normal((ny, nx))
    r = rng.standard_normal((ny, nx))
    h = rng.random((kh, kw))
    lhs = np.vdot(orc.blur(x, h), r)
    rhs = np.vdot(x, orc.blur_adj(r, h))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_shift_kernel_is_convolution(orc):
    """A kernel with a single 1 at (a, b) shifts the image by (a - r, b - r):
    (h * x)[i, j] = x[i - (a - r), j - (b - r)]  (a true convolution)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((9, 11))
    for a, b in [(0, 0), (0, 4), (3, 1), (4, 4)]:
        h = np.zeros((5, 5))
        h[a, b] = 1.0
        np.testing.assert_array_equal(orc.blur(x, h), np.roll(x, (a - 2, b - 2), axis=(0, 1)))
        np.testing.assert_array_equal(orc.blur_adj(x, h), np.roll(x, (2 - a, 2 - b), axis=(0, 1)))


def test_operator_norm_of_normalised_kernel(orc):
    """For h >= 0 with sum 1, ||H||_2 = max |DFT(h)| = 1 (power iteration on H^T H)."""
    rng = np.random.default_rng(11)
    for h in (synth.gaussian_kernel(7, 1.5), synth.uniform_kernel(9), synth.motion_kernel(13, 0.7)):
        x = rng.standard_normal((24, 20))
        for _ in range(200):
            x = orc.blur_adj(orc.blur(x, h), h)
            x /= np.linalg.norm(x)
        lam = np.vdot(x, orc.blur_adj(orc.blur(x, h), h))
        assert abs(np.sqrt(lam) - 1.0) < 1e-6


def test_blur_of_constant_image(orc):
    """Circular blur preserves the mean: H 1 = (sum h) 1."""
    h = synth.motion_kernel(11, 1.1)
    out = orc.blur(np.full((10, 12), 0.37), h)
    np.testing.assert_allclose(out, 0.37 * h.sum(), rtol=1e-13)
