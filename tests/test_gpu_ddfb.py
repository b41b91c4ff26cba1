"""GPU parity of the DDFB denoiser (Sec. II-B, Example 2) and of the sampler
with the DDFB prior against the FP64 oracle.

Bounds: the denoiser output lies in [0, 1] and each dual variable in
[-ht, ht], so FP32 sums of P x 9 products keep |D_gpu - D_oracle| <= 1e-5;
the one-step x-update within 1e-5 * max|x+| as for the other priors.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_00870_b300 as P
    return P


def _nets(P, orc, K, Pc, seed=11, ht=0.05):
    dw = synth.ddfb_weights(K, Pc, seed, ht)
    return P.Denoiser.ddfb(dw.filters, dw.gammas, dw.ht), orc.Ddfb(dw.filters, dw.gammas, dw.ht), dw


@pytest.mark.parametrize("ny,nx,K,Pc", [(37, 70, 4, 16), (128, 96, 4, 64), (9, 200, 3, 32),
                                        (64, 64, 6, 64)])
def test_denoiser_against_oracle(P, orc, ny, nx, K, Pc):
    den, onet, _ = _nets(P, orc, K, Pc)
    rng = np.random.default_rng(ny + nx)
    x = np.clip(0.5 + 0.3 * rng.standard_normal((2, ny, nx)), -0.2, 1.2).astype(np.float32)
    out = den.denoise(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    for c in range(2):
        ref = orc.ddfb_denoise(x[c].astype(np.float64), onet)
        np.testing.assert_allclose(out[c].cpu().numpy(), ref, rtol=0, atol=1e-5)


def test_one_step_with_ddfb_prior(P, orc):
    """Ragged 72 x 136, uniform 5 x 5 blur, DDFB K = 4, P = 64 in the x-update."""
    prob = synth.make_problem(72, 136, synth.uniform_kernel(5), 20.0, 515)
    den, onet, _ = _nets(P, orc, 4, 64)
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed)
    prm = gp.params()
    op = orc.Problem(prob.y, prob.h, prob.sigma, prm["alpha"], prm["eps"], prm["lam"],
                     prm["gamma"], prob.seed, ddfb=onet)
    x0 = np.clip(prob.y + 0.02, 0, 1).astype(np.float32)
    for t in (0, 5):
        gp.set_state(x0, t)
        gp.step(1)
        xn, _ = gp.state()
        ref = orc.langevin_step(op, x0.astype(np.float64), t)
        assert np.abs(xn[0] - ref).max() <= 1e-5 * np.abs(ref).max(), t


def test_graph_eager_and_batch_with_ddfb(P, orc):
    prob = synth.make_problem(96, 128, synth.gaussian_kernel(7, 1.5), 25.0, 516)
    den, _, _ = _nets(P, orc, 4, 64)
    out = []
    for graph in (True, False):
        P.pnp_set_graph_mode(graph)
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=8, burn_in=2)
        gp.run_chain(9, 2)
        out.append((gp.state()[0], gp.moments(want_var=True)[1]))
    P.pnp_set_graph_mode(True)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    other = synth.make_problem(64, 80, synth.uniform_kernel(5), 25.0, 517)
    b = P.Batch([dict(y=prob.y, h=prob.h, sigma=prob.sigma, seed=8, burn_in=2),
                 dict(y=other.y, h=other.h, sigma=other.sigma, seed=9)], den, precision="fp32")
    b.run(9, 2)
    np.testing.assert_array_equal(b.job(0).state()[0], out[0][0])


def test_full_size_sampled(P, orc):
    """1024 x 1024 (the deconv1024 image and blur) with the DDFB prior: x+ at
    sampled pixels from crops (blur radius 2r wrapped; the DDFB receptive
    field 2K unwrapped with zero padding)."""
    prob = synth.workload_problem(2)
    den, onet, _ = _nets(P, orc, 4, 64)
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed)
    prm = gp.params()
    rng = np.random.default_rng(2)
    x0 = np.clip(prob.y + 0.05 * rng.standard_normal(prob.shape), -0.1, 1.1).astype(np.float32)
    t = 123
    gp.set_state(x0, t)
    gp.step(1)
    xn, _ = gp.state()
    x = x0.astype(np.float64)
    n = 1024
    rr = prob.h.shape[0] // 2
    R = 2 * 4          # DDFB receptive radius: 2 per operator pair, K = 4
    xi = orc.normals(prob.seed, t, 0, n * n).reshape(n, n)
    pix = [(0, 0), (1023, 1023), (0, 700), (511, 512)] + [tuple(v) for v in rng.integers(0, n, (6, 2))]
    gam, c_prior = prm["gamma"], prm["alpha"] * prm["gamma"] / prm["eps"] ** 2
    worst = 0.0
    for (i, j) in pix:
        xc = np.take(np.take(x, np.arange(i - 2 * rr, i + 2 * rr + 1) % n, 0),
                     np.arange(j - 2 * rr, j + 2 * rr + 1) % n, 1)
        yc = np.take(np.take(prob.y, np.arange(i - 2 * rr, i + 2 * rr + 1) % n, 0),
                     np.arange(j - 2 * rr, j + 2 * rr + 1) % n, 1)
        g = orc.blur_adj(orc.blur(xc, prob.h) - yc, prob.h)[2 * rr, 2 * rr] / prob.sigma ** 2
        i0, i1, j0, j1 = max(0, i - R), min(n, i + R + 1), max(0, j - R), min(n, j + R + 1)
        d = orc.ddfb_denoise(x[i0:i1, j0:j1], onet)[i - i0, j - j0]
        xv = x[i, j]
        v = xv - gam * g + c_prior * (d - xv) + gam / prm["lam"] * (min(max(xv, 0.0), 1.0) - xv)
        v += np.sqrt(2 * gam) * xi[i, j]
        worst = max(worst, abs(xn[0][i, j] - v))
    assert worst <= 1e-5 * np.abs(xn[0]).max(), worst
