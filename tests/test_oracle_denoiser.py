"""Pins for the oracle's DnCNN-form denoiser (Sec. II-B, Example 1) and its
block-wise evaluation (Defs. 1-2, Sec. II-B2).

Pins: torch.nn.functional.conv2d in FP64 on the CPU (a library routine) for
every layer and for the composed network; D = Id - G (zero network gives the
identity); block-wise = whole image exactly when the halo covers the
receptive field (K pixels for K 3x3 layers) and not when it falls one short;
the Lipschitz bound of Id - D.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import synth


def torch_layer(inp, w, b, relu):
    out = Fnn.conv2d(torch.from_numpy(inp)[None], torch.from_numpy(w), torch.from_numpy(b),
                     padding=w.shape[2] // 2)[0]
    return torch.relu(out).numpy() if relu else out.numpy()


def torch_denoise(v, dw):
    a = v[None]
    for k, (w, b) in enumerate(zip(dw.weights, dw.biases)):
        a = torch_layer(a, w, b, k < len(dw.weights) - 1)
    return v - a[0]


@pytest.mark.parametrize("cin,cout,ny,nx,ks,relu", [
    (1, 4, 9, 7, 3, True), (3, 5, 12, 16, 3, False), (8, 8, 5, 6, 3, True),
    (2, 3, 10, 11, 5, True), (16, 1, 7, 9, 3, False), (4, 4, 1, 1, 3, True)])
def test_conv_layer_matches_library(orc, cin, cout, ny, nx, ks, relu):
    rng = np.random.default_rng(cin * 31 + cout)
    inp = rng.standard_normal((cin, ny, nx))
    w = rng.standard_normal((cout, cin, ks, ks))
    b = rng.standard_normal(cout)
    np.testing.assert_allclose(orc.conv_layer(inp, w, b, relu), torch_layer(inp, w, b, relu),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("K,F", [(4, 16), (8, 8), (1, 1)])
def test_denoiser_matches_library_composition(orc, K, F):
    dw = synth.denoiser_weights(K, F, seed=5 + K)
    v = synth.ground_truth(23, 17, seed=9)
    net = orc.Net.from_weights(dw)
    np.testing.assert_allclose(orc.denoise(v, net), torch_denoise(v, dw), rtol=0, atol=1e-12)


def test_zero_network_is_identity(orc):
    dw = synth.denoiser_weights(3, 4, seed=1)
    dw.weights = [np.zeros_like(w) for w in dw.weights]
    dw.biases = [np.zeros_like(b) for b in dw.biases]
    v = synth.ground_truth(12, 12, seed=2)
    np.testing.assert_array_equal(orc.denoise(v, orc.Net.from_weights(dw)), v)


@pytest.mark.parametrize("ny,nx,by,bx", [(32, 32, 2, 2), (37, 29, 3, 2), (40, 24, 4, 1), (20, 20, 1, 1)])
def test_blockwise_equals_whole_when_halo_covers_receptive_field(orc, ny, nx, by, bx):
    K = 4
    dw = synth.denoiser_weights(K, 8, seed=3)
    net = orc.Net.from_weights(dw)
    v = synth.ground_truth(ny, nx, seed=ny + nx)
    whole = orc.denoise(v, net)
    for halo in (K, K + 3):
        blk = orc.denoise_blockwise(v, net, by, bx, halo)
        np.testing.assert_allclose(blk, whole, rtol=0, atol=1e-14)


def test_blockwise_short_halo_differs_at_block_edges(orc):
    """Negative control: a halo of K - 1 leaves errors next to inner block edges only."""
    K = 4
    dw = synth.denoiser_weights(K, 8, seed=3)
    net = orc.Net.from_weights(dw)
    v = synth.ground_truth(32, 32, seed=4)
    whole = orc.denoise(v, net)
    blk = orc.denoise_blockwise(v, net, 2, 2, K - 1)
    err = np.abs(blk - whole)
    assert err.max() > 1e-6
    # the error is confined to pixels adjacent to the inner edges (rows/cols 15, 16)
    mask = np.zeros_like(err, dtype=bool)
    mask[15:17, :] = True
    mask[:, 15:17] = True
    assert err[~mask].max() < 1e-14


def test_lipschitz_bound_of_residual(orc):
    """|| G(a) - G(b) || <= L_eps || a - b || with G = Id - D (ReLU is 1-Lipschitz
    and every layer's spectral norm is 0.9^(1/K))."""
    dw = synth.denoiser_weights(4, 16, seed=8)
    net = orc.Net.from_weights(dw)
    rng = np.random.default_rng(0)
    for _ in range(6):
        a = rng.random((20, 20))
        b = a + 0.1 * rng.standard_normal((20, 20))
        ga = a - orc.denoise(a, net)
        gb = b - orc.denoise(b, net)
        assert np.linalg.norm(ga - gb) <= dw.lipschitz * np.linalg.norm(a - b) * (1 + 1e-9)


def test_blockwise_rejects_bad_arguments(orc):
    dw = synth.denoiser_weights(2, 2, seed=1)
    net = orc.Net.from_weights(dw)
    with pytest.raises(ValueError):
        orc.denoise_blockwise(np.zeros((4, 4)), net, 5, 1, 2)
