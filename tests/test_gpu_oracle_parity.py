"""GPU chain against the FP64 oracle's own transition, at the workloads' sizes.

* BF16 precision form, whole chain: the MMSE PSNR of a BF16 GPU chain is
  within 0.1 dB of the FP64 oracle chain's on the same inputs and Philox
  stream (128 x 128, 8 layers x 64 channels, 64 iterations, 16 burn-in); the
  FP32 chain's difference is reported beside it.
* FP32 plain path at 1024 x 1024 (9 x 9 uniform blur, prior on): one step from
  an injected state, every element against ora_langevin_step on the whole
  image, within 1e-5 max|x+|.
* 8192 x 8192 precision workload (13 x 13 Gaussian blur, 16 x 16 blocks, the
  benchmark's direct layout): one step from injected states at two t values,
  at windows on the corners, the last row and column, block and column-strip
  edges and the interior, against ora_langevin_step_window. FP32: within
  1e-5 max|x+|; BF16: the prior term's BF16 error c_prior |G_bf16 - G| on top
  (bound in BF16_G_TOL).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# BF16 denoiser error bound, relative to max|G| (G = x - D(x)): seven layers
# take BF16 operands (activations and weights rounded to 8 significant bits,
# unit roundoff u = 2^-9) with FP32 accumulation; the 14 roundings are
# independent and the 0.9-Lipschitz layers do not amplify them, so they add
# like a random walk, sqrt(14) u = 7.3e-3 (worst case 14 u = 2.7e-2; measured
# 3-6e-3 on the denoiser tests).
BF16_G_TOL = 1e-2


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_00870_b300 as P
    return P


def _oracle(orc, prob, prm, net):
    return orc.Problem(prob.y, prob.h, prob.sigma, prm["alpha"], prm["eps"], prm["lam"],
                       prm["gamma"], prob.seed, net=net)


def _psnr(m, xbar):
    return 10.0 * np.log10(1.0 / np.mean((np.asarray(m, np.float64) - xbar) ** 2))


def test_bf16_chain_psnr_vs_oracle_chain(P, orc):
    prob = synth.workload_problem(2, shrink=8)          # 128 x 128, uniform 9 x 9, 20 dB
    dw = synth.workload_denoiser(2)                     # K = 8, F = 64
    den = P.Denoiser.from_weights(dw)
    T, TB = 64, 16
    ps, prm = {}, None
    for prec in ("bf16", "fp32"):
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed, burn_in=TB, precision=prec)
        prm = gp.params()
        gp.run_chain(T, TB)
        mm, _, n = gp.moments()
        assert n == T - TB
        ps[prec] = _psnr(mm, prob.xbar)
    ro = orc.run_chain(_oracle(orc, prob, prm, orc.Net.from_weights(dw)), np.zeros(prob.shape), T, TB)
    assert ro["n"] == T - TB
    ps["oracle"] = _psnr(ro["mean"], prob.xbar)
    print("MMSE PSNR oracle %.4f dB, bf16 %.4f (%+.4f), fp32 %.4f (%+.4f)" % (
        ps["oracle"], ps["bf16"], ps["bf16"] - ps["oracle"], ps["fp32"], ps["fp32"] - ps["oracle"]))
    assert abs(ps["bf16"] - ps["oracle"]) <= 0.1
    assert abs(ps["fp32"] - ps["oracle"]) <= 0.1


def test_config2_whole_image_one_step_fp32(P, orc):
    prob = synth.workload_problem(2)
    dw = synth.workload_denoiser(2)
    gp = P.Problem(prob.y, prob.h, prob.sigma, P.Denoiser.from_weights(dw), blocks=prob.blocks,
                   halo=0, seed=prob.seed, burn_in=prob.burn_in)
    prm = gp.params()
    rng = np.random.default_rng(12)
    x0 = np.clip(prob.y + 0.05 * rng.standard_normal(prob.shape), -0.1, 1.1).astype(np.float32)
    t = 777
    gp.set_state(x0, t)
    gp.step(1)
    xg, tt = gp.state()
    assert tt == t + 1
    ref = orc.langevin_step(_oracle(orc, prob, prm, orc.Net.from_weights(dw)),
                            x0.astype(np.float64), t)
    err = np.abs(xg[0] - ref).max()
    print("1024^2 whole-image one-step max|dx| %.3e (bound %.3e)" % (err, 1e-5 * np.abs(ref).max()))
    assert err <= 1e-5 * np.abs(ref).max()


@pytest.fixture(scope="module")
def cfg3():
    return synth.workload_problem(3)   # 8192 x 8192, Gaussian 13 x 13 s = 3, 30 dB


W = 4
WINDOWS = [(0, 0), (0, 8192 - W), (8192 - W, 0), (8192 - W, 8192 - W),   # corners
           (8192 - W, 3001), (2000, 8192 - W),                               # last row / column
           (510, 510), (4094, 1022), (1022, 7166), (6142, 4094),            # 512-px block edges
           (777, 126), (3000, 2046)]                                         # 128-px strip edges
WINDOWS += [tuple(int(v) for v in w) for w in np.random.default_rng(3).integers(0, 8192 - W, (4, 2))]


def _g_scale(orc, net, x, K):
    """max |G| = max |x - D(x)| over the windows (oracle denoiser on crops)."""
    ny, nx = x.shape
    gmax = 0.0
    for (i0, j0) in WINDOWS:
        a0, a1 = max(0, i0 - K), min(ny, i0 + W + K)
        b0, b1 = max(0, j0 - K), min(nx, j0 + W + K)
        c = x[a0:a1, b0:b1]
        G = c - orc.denoise(c, net)
        gmax = max(gmax, np.abs(G[i0 - a0:i0 - a0 + W, j0 - b0:j0 - b0 + W]).max())
    return gmax


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_config3_8192_sampled_one_step(P, orc, cfg3, prec):
    prob = cfg3
    dw = synth.workload_denoiser(3)
    net = orc.Net.from_weights(dw)
    gp = P.Problem(prob.y, prob.h, prob.sigma, P.Denoiser.from_weights(dw), blocks=prob.blocks,
                   halo=0, seed=prob.seed, burn_in=prob.burn_in, precision=prec)
    prm = gp.params()
    op = _oracle(orc, prob, prm, net)
    c_prior = prm["alpha"] * prm["gamma"] / prm["eps"] ** 2
    rng = np.random.default_rng(30)
    for t in (0, 999):
        x0 = np.clip(prob.y + 0.05 * rng.standard_normal(prob.shape, dtype=np.float32),
                     -0.1, 1.1).astype(np.float32)
        gp.set_state(x0, t)
        gp.step(1)
        xg, tt = gp.state()
        assert tt == t + 1
        x64 = x0.astype(np.float64)
        bound = 1e-5 * np.abs(xg[0]).max()
        if prec == "bf16":
            bound += c_prior * BF16_G_TOL * _g_scale(orc, net, x64, dw.K)
        worst = 0.0
        for (i0, j0) in WINDOWS:
            ref = orc.langevin_step_window(op, x64, t, i0, j0, W, W)
            worst = max(worst, np.abs(xg[0][i0:i0 + W, j0:j0 + W] - ref).max())
        print("8192^2 %s t=%d: max|dx| %.3e, bound %.3e" % (prec, t, worst, bound))
        assert worst <= bound, (t, worst, bound)
    gp.close()
