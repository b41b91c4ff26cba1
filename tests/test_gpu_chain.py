"""GPU chain parity against the FP64 oracle, through the problem API of the C ABI.

One-step bound (FP32 plain path): from the same state x^(t), the GPU's x^(t+1)
is within 1e-5 * max|x^(t+1)| of the oracle's. Chains are compared by
injecting the GPU state into the oracle at every t, because ULA need not
contract and free-running trajectories drift apart at FP32 rounding.
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


def oracle_problem(orc, prob, params, net=None, noise=True):
    return orc.Problem(prob.y, prob.h, prob.sigma, params["alpha"] if net else 0.0, params["eps"],
                       params["lam"], params["gamma"], prob.seed, net=net, noise=noise)


def test_config1_chain_one_step_bound_every_t(P, orc):
    prob = synth.workload_problem(1)
    dw = synth.workload_denoiser(1)
    den = P.Denoiser.from_weights(dw)
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=prob.blocks, halo=prob.halo,
                   seed=prob.seed, burn_in=prob.burn_in)
    prm = gp.params()
    op = oracle_problem(orc, prob, prm, orc.Net.from_weights(dw))
    worst = 0.0
    traj = []
    x_prev, _ = gp.state()
    for t in range(prob.T):
        gp.step(1)
        x_new, tt = gp.state()
        assert tt == t + 1
        ref = orc.langevin_step(op, x_prev[0].astype(np.float64), t)
        err = np.abs(x_new[0] - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        traj.append(x_new[0].astype(np.float64))
        x_prev = x_new
    assert worst <= 1e-5, worst
    # moments: the GPU's FP32 Welford vs FP64 two-pass over the same trajectory
    kept = np.stack(traj[prob.burn_in:])
    mm, var, n = gp.moments(want_var=True)
    assert n == prob.T - prob.burn_in
    m_ref, v_ref = orc.moments_two_pass(kept)
    np.testing.assert_allclose(mm, m_ref, rtol=0, atol=1e-6 * np.abs(m_ref).max())
    np.testing.assert_allclose(var, v_ref, rtol=1e-3, atol=1e-6 * v_ref.max())
    mm2, sd, _ = gp.moments(want_var=False)
    np.testing.assert_allclose(sd, np.sqrt(var), rtol=1e-12)


def test_free_running_trajectory_error_is_reported(P, orc):
    """Free-running GPU vs oracle chains on config 1 (reported, loosely bounded)."""
    prob = synth.workload_problem(1)
    dw = synth.workload_denoiser(1)
    gp = P.Problem(prob.y, prob.h, prob.sigma, P.Denoiser.from_weights(dw), seed=prob.seed,
                   burn_in=prob.burn_in)
    op = oracle_problem(orc, prob, gp.params(), orc.Net.from_weights(dw))
    gp.run_chain(prob.T, prob.burn_in)
    xg, _ = gp.state()
    ro = orc.run_chain(op, np.zeros(prob.shape), prob.T, prob.burn_in)
    err = np.abs(xg[0] - ro["x"]).max()
    print(f"config-1 free-running trajectory max|dx| after {prob.T} steps: {err:.3e}")
    assert err < 1e-3


def test_graph_replay_equals_eager(P):
    prob = synth.workload_problem(1, shrink=2)
    dw = synth.workload_denoiser(1)
    den = P.Denoiser.from_weights(dw)
    out = []
    for graph in (True, False):
        P.pnp_set_graph_mode(graph)
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=5, burn_in=3)
        gp.run_chain(12, 3)
        out.append((gp.state()[0], gp.moments(want_var=True)))
    P.pnp_set_graph_mode(True)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1][0], out[1][1][0])
    np.testing.assert_array_equal(out[0][1][1], out[1][1][1])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_block_split_invariance(P, prec):
    """E11: the chain is the same for any block split (counter-based RNG and
    fixed-order sums make it bitwise for both precisions)."""
    prob = synth.workload_problem(2, shrink=8)      # 128 x 128, 8L x 64ch
    dw = synth.workload_denoiser(2)
    den = P.Denoiser.from_weights(dw)
    res = []
    for blocks, halo in [((1, 1), 0), ((4, 4), 8), ((2, 3), 8)]:
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=blocks, halo=halo, seed=7,
                       burn_in=2, precision=prec)
        gp.run_chain(6, 2)
        res.append(gp.state()[0])
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], res[2])


def test_resume_is_bitwise(P):
    prob = synth.workload_problem(1, shrink=2)
    dw = synth.workload_denoiser(1)
    den = P.Denoiser.from_weights(dw)
    a = P.Problem(prob.y, prob.h, prob.sigma, den, seed=9)
    a.run_chain(10, 0)
    xa, _ = a.state()
    b = P.Problem(prob.y, prob.h, prob.sigma, den, seed=9)
    b.run_chain(4, 0)
    xb, tb = b.state()
    c = P.Problem(prob.y, prob.h, prob.sigma, den, seed=9)
    c.set_state(xb, tb)
    c.run_chain(6, 0)
    np.testing.assert_array_equal(c.state()[0], xa)


def test_chains_are_independent_streams(P):
    prob = synth.workload_problem(1, shrink=4)
    gp = P.Problem(prob.y, prob.h, prob.sigma, None, seed=1, nchain=3)
    gp.run_chain(5, 0)
    x, _ = gp.state()
    assert not np.array_equal(x[0], x[1]) and not np.array_equal(x[1], x[2])
    # chain c of a 3-chain problem equals chain c run alone? (same counters: chain index)
    solo = P.Problem(prob.y, prob.h, prob.sigma, None, seed=1, nchain=1)
    solo.run_chain(5, 0)
    np.testing.assert_array_equal(solo.state()[0][0], x[0])


def test_stationary_law_gpu(P):
    """Noise on, no prior, projection off: ULA on a Gaussian; the empirical law
    of 4096 independent GPU chains matches N(mu, Q^-1 (I - gamma Q/2)^-1)."""
    ny = nx = 8
    h = np.array([[0.0, 0.1, 0.0], [0.1, 0.6, 0.1], [0.0, 0.1, 0.0]], np.float32)
    rng = np.random.default_rng(42)
    y = rng.random((ny, nx)).astype(np.float32)
    sigma = 0.1
    gamma = 0.5 * sigma ** 2
    nch = 4096
    x = torch.zeros((nch, ny, nx), device="cuda")
    r = torch.empty_like(x)
    yd, hd = torch.from_numpy(y).cuda(), torch.from_numpy(h).cuda()
    for t in range(600):
        P.pnp_blur(x, yd, hd, r)
        P.pnp_langevin_update(x, r, None, hd, sigma=sigma, alpha=0.0, eps=1.0, lam=0.0,
                              gamma=gamma, seed=2024, t=t)
    xs = x.cpu().numpy().astype(np.float64)
    hp = np.zeros((ny, nx))
    for a in range(3):
        for b in range(3):
            hp[(a - 1) % ny, (b - 1) % nx] += h[a, b]
    Hf = np.fft.fft2(hp)
    q = np.abs(Hf) ** 2 / sigma ** 2
    mu = np.real(np.fft.ifft2(np.conj(Hf) * np.fft.fft2(y) / sigma ** 2 / q))
    cov0 = np.real(np.fft.ifft2(1.0 / (q * (1 - gamma * q / 2))))
    se = np.sqrt(cov0[0, 0] / nch)
    assert np.abs(xs.mean(0) - mu).max() < 4.5 * se
    v = ((xs - mu) ** 2).mean(0)
    assert np.abs(v - cov0[0, 0]).max() < 5 * cov0[0, 0] * np.sqrt(2 / nch)


def test_config2_full_size_sampled_one_step(P, orc):
    """1024 x 1024, 9x9 uniform blur, 8L x 64ch FP32, 4 x 4 blocks: one-step
    bound at windows (corners, borders, block edges, interior) for injected
    states at several t, in the launch configuration the benchmark times,
    against the oracle's transition evaluated on those windows."""
    prob = synth.workload_problem(2)
    dw = synth.workload_denoiser(2)
    den = P.Denoiser.from_weights(dw)
    net = orc.Net.from_weights(dw)
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=prob.blocks, halo=0, seed=prob.seed,
                   burn_in=prob.burn_in)
    prm = gp.params()
    op = oracle_problem(orc, prob, prm, net)
    rng = np.random.default_rng(0)
    w = 3
    wins = [(0, 0), (0, 1021), (1021, 510), (254, 255), (255, 254), (510, 511), (766, 2),
            (100, 1000)] + [tuple(v) for v in rng.integers(0, 1021, size=(8, 2))]
    for t in (0, 1, 499, 1999):
        x0 = np.clip(prob.y + 0.05 * rng.standard_normal(prob.shape), -0.1, 1.1).astype(np.float32)
        gp.set_state(x0, t)
        gp.step(1)
        xn, _ = gp.state()
        x64 = x0.astype(np.float64)
        err = max(np.abs(xn[0][i:i + w, j:j + w] -
                         orc.langevin_step_window(op, x64, t, i, j, w, w)).max() for i, j in wins)
        assert err <= 1e-5 * np.abs(xn[0]).max(), (t, err)


def test_bf16_mmse_psnr_matches_fp32(P):
    """Precision form: the BF16 denoiser chain gives the FP32 chain's MMSE PSNR
    within 0.1 dB (256 x 256, 8L x 64ch, 200 iterations, 50 burn-in)."""
    prob = synth.workload_problem(2, shrink=4)
    dw = synth.workload_denoiser(2)
    den = P.Denoiser.from_weights(dw)
    ps = {}
    for prec in ("fp32", "bf16"):
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed, precision=prec)
        gp.run_chain(200, 50)
        mm, _, _ = gp.moments()
        ps[prec] = 10 * np.log10(1.0 / np.mean((mm - prob.xbar) ** 2))
    print("MMSE PSNR fp32 %.3f dB  bf16 %.3f dB" % (ps["fp32"], ps["bf16"]))
    assert abs(ps["fp32"] - ps["bf16"]) <= 0.1


@pytest.mark.parametrize("blocks,halo", [((1, 1), 0), ((2, 2), 8)])
def test_bf16_one_step_against_oracle(P, orc, blocks, halo):
    """One BF16 step from an injected state against the FP64 oracle, in the
    direct and the block + halo layouts: the difference is the prior term's
    BF16 error, c_prior |G_bf16 - G|, bounded like the denoiser tests (1 % of
    max |G|), on a ragged 72 x 136 image."""
    prob = synth.make_problem(72, 136, synth.uniform_kernel(5), 25.0, 909)
    dw = synth.workload_denoiser(2)
    den = P.Denoiser.from_weights(dw)
    net = orc.Net.from_weights(dw)
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=blocks, halo=halo, seed=prob.seed,
                   burn_in=0, precision="bf16")
    prm = gp.params()
    x0 = np.clip(prob.y + 0.03, 0, 1).astype(np.float64)
    gp.set_state(x0, 3)
    gp.step(1)
    x1, _ = gp.state()
    op = oracle_problem(orc, prob, prm, net)
    ref = orc.langevin_step(op, x0, 3)
    G = x0 - orc.denoise(x0, net)
    c_prior = prm["alpha"] * prm["gamma"] / prm["eps"] ** 2
    bound = c_prior * 1e-2 * np.abs(G).max() + 1e-5 * np.abs(ref).max()
    assert np.abs(x1[0] - ref).max() <= bound, (np.abs(x1[0] - ref).max(), bound)
