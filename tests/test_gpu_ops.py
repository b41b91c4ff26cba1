"""GPU parity of the operator entry points against the FP64 oracle.

Every call goes through the C ABI (libpnp.so) via the thin binding; inputs are
seeded synthetic data; the oracle computes the same quantities on the CPU.
Tolerances (FP32 path): the blur/adjoint are sums of at most 441 FP32
products of magnitude <= max|x| |h|, so 2e-6 relative to max|output| bounds
the rounding; the denoiser accumulates 576 products per layer over K layers,
bounded by 1e-5 relative to max|G|.
"""
import numpy as np
import pytest

import synth

# BF16 denoiser error bound, relative to max|G| (G = x - D(x)): seven layers
# take BF16 operands, each rounding its input activations and weights to 8
# significant bits (unit roundoff u = 2^-9), with FP32 accumulation. The 14
# roundings are independent and the 0.9-Lipschitz layers do not amplify them,
# so they add like a random walk: sqrt(14) u = 7.3e-3 of the activation
# scale (the worst case, all aligned, is 14 u = 2.7e-2). Measured: 3-6e-3.
BF16_G_TOL = 1e-2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_00870_b300 as P
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


BLUR_CASES = [(7, 13, 3, 3), (64, 64, 7, 7), (37, 130, 9, 9), (130, 257, 13, 13), (33, 31, 21, 21),
              (256, 200, 5, 15)]


@pytest.mark.parametrize("ny,nx,kh,kw", BLUR_CASES)
def test_blur_and_adjoint(P, orc, ny, nx, kh, kw):
    rng = np.random.default_rng(ny * 7 + nx)
    x = rng.random((2, ny, nx)).astype(np.float32)
    y = rng.random((ny, nx)).astype(np.float32)
    h = synth.motion_kernel(max(kh, kw), 0.3)[:kh, :kw].astype(np.float32)
    h = (rng.random((kh, kw)) * (h + 0.01)).astype(np.float32)
    r = torch.empty((2, ny, nx), device="cuda")
    P.pnp_blur(dev(x), dev(y), dev(h), r)
    g = torch.empty_like(r)
    P.pnp_blur_adjoint(r, dev(h), g, scale=0.5)
    torch.cuda.synchronize()
    for c in range(2):
        rr = orc.blur(x[c], h) - y
        np.testing.assert_allclose(r[c].cpu().numpy(), rr, rtol=0, atol=2e-6 * np.abs(rr).max())
        gg = 0.5 * orc.blur_adj(r[c].cpu().numpy().astype(np.float64), h)
        np.testing.assert_allclose(g[c].cpu().numpy(), gg, rtol=0, atol=2e-6 * np.abs(gg).max())


def test_normals_match_oracle(P, orc):
    """x = 0, y = 0, no prior, no projection: x+ = sqrt(2 gamma) xi, so the GPU's
    xi can be read back and compared with the oracle's Philox/Box-Muller draws,
    including widths that are not multiples of 4 and several chains.

    Bound: the GPU forms -2 ln u from __logf and a series, and sin / cos of
    2 pi u from __sincosf, with the error bounds CUDA documents for them. The
    relative error of rad = sqrt(-2 ln u) stays below 2.5e-7 for u < 1/2
    (rad <= 5.9) and 1.7e-6 for u in [1/2, 7/8] (rad <= 1.18); sin and cos are
    off by at most 5.7e-7. So |dz| <= max(5.9 * 3.7e-7, 1.18 * 1.8e-6)
    + 5.9 * 5.7e-7 < 5.5e-6, plus 6e-7 for the FP32 x+ = sqrt(2 gamma) xi and
    its readback: 7e-6 (measured over 2.7e8 draws: 1.9e-6)."""
    for ny, nx, nch in [(8, 8, 3), (5, 7, 2), (33, 129, 1)]:
        h = dev(np.ones((1, 1)))
        x = torch.zeros((nch, ny, nx), device="cuda")
        r = torch.zeros_like(x)
        gamma = 0.125
        seed = 0xABCDEF0123456789
        P.pnp_langevin_update(x, r, None, h, sigma=1.0, alpha=0.0, eps=1.0, lam=0.0, gamma=gamma,
                              seed=seed, t=9, noise=True)
        xi = (x / np.sqrt(2 * gamma)).cpu().numpy().astype(np.float64)
        for c in range(nch):
            ref = orc.normals(seed, 9, c, ny * nx).reshape(ny, nx)
            np.testing.assert_allclose(xi[c], ref, rtol=0, atol=7e-6)


def _net(K, F, seed=11):
    return synth.denoiser_weights(K, F, seed=seed)


@pytest.mark.parametrize("K,F,ny,nx", [(4, 16, 72, 72), (4, 16, 37, 53), (8, 64, 40, 136),
                                       (3, 32, 17, 9), (8, 64, 130, 140)])
def test_denoise_fp32(P, orc, K, F, ny, nx):
    dw = _net(K, F)
    den = P.Denoiser.from_weights(dw)
    net = orc.Net.from_weights(dw)
    rng = np.random.default_rng(5)
    x = rng.random((2, ny, nx)).astype(np.float32)
    d = den.denoise(dev(x)).cpu().numpy()
    for c in range(2):
        ref = orc.denoise(x[c], net)
        G = x[c] - ref
        np.testing.assert_allclose(x[c] - d[c], G, rtol=0, atol=1e-5 * np.abs(G).max() + 1e-7)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_blockwise_halo_equals_whole(P, prec):
    """Sec. II-B2 / E11: with halo >= K the block-with-halo result is the
    whole-image result (bitwise: same fixed-order sums); halo = K-1 is not."""
    K, F = (8, 64)
    dw = _net(K, F)
    den = P.Denoiser.from_weights(dw)
    x = dev(synth.ground_truth(96, 80, seed=3)[None])
    whole = den.denoise(x, precision=prec)
    blk = den.denoise(x, precision=prec, blocks=(3, 2), halo=K)
    torch.cuda.synchronize()
    assert torch.equal(whole, blk)
    short = den.denoise(x, precision=prec, blocks=(3, 2), halo=K - 1)
    assert (short - whole).abs().max().item() > 0


@pytest.mark.parametrize("ny,nx", [(64, 64), (37, 200), (130, 257), (8, 8)])
def test_denoise_bf16_close_to_oracle(P, orc, ny, nx):
    """BF16 operands with FP32 accumulation: the residual G = x - D(x) is
    within a BF16-level error of the FP64 oracle."""
    K, F = 8, 64
    dw = _net(K, F)
    den = P.Denoiser.from_weights(dw)
    net = orc.Net.from_weights(dw)
    x = synth.ground_truth(ny, nx, seed=ny + nx).astype(np.float32)
    d = den.denoise(dev(x[None]), precision="bf16").cpu().numpy()[0]
    G = x - orc.denoise(x, net)
    err = np.abs((x - d) - G)
    print("bf16 denoiser %dx%d: max|dG| / max|G| = %.3e" % (ny, nx, err.max() / np.abs(G).max()))
    assert err.max() <= BF16_G_TOL * np.abs(G).max(), (err.max(), np.abs(G).max())


def test_denoise_bf16_matches_fp32_path(P):
    """Same network, BF16 vs FP32 GPU path on a larger image (several strips,
    a ragged tail, many CTAs)."""
    dw = _net(8, 64)
    den = P.Denoiser.from_weights(dw)
    x = dev(synth.ground_truth(300, 333, seed=9)[None])
    d32 = den.denoise(x, precision="fp32")
    d16 = den.denoise(x, precision="bf16")
    G = (x - d32).abs().max().item()
    print("bf16 vs fp32 denoiser 300x333: max|dG| / max|G| = %.3e" % ((d16 - d32).abs().max().item() / G))
    assert (d16 - d32).abs().max().item() <= BF16_G_TOL * G
