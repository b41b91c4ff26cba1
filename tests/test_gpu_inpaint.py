"""GPU parity of the inpainting sampler (Sec. IV-A: H = diag(mask), Gaussian
noise, x initialised by interpolating y) against the FP64 oracle.

One-step bound (FP32 path): from the same x^(t), max|x_gpu - x_oracle| <=
1e-5 * max|x_oracle|, as for deconvolution. The masked update has no stencil:
the data term is x - y at observed pixels and 0 at missing ones.
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


def _gpu_problem(P, prob, den, **kw):
    kw.setdefault("x0", prob.x0)
    return P.Problem(prob.y, None, prob.sigma, den, mask=prob.mask, seed=prob.seed, **kw)


def _oracle(orc, prob, prm, net, noise=True):
    return orc.Problem(prob.y, None, prob.sigma, prm["alpha"] if net else 0.0, prm["eps"],
                       prm["lam"], prm["gamma"], prob.seed, net=net, noise=noise, mask=prob.mask)


@pytest.mark.parametrize("shape", [(64, 64), (37, 53)])
def test_operator_against_oracle(P, orc, shape):
    """pnp_inpaint_update on device buffers, 2 chains, moments on; the 37 x 53
    image (plane not a multiple of 4) takes the scalar path."""
    prob = synth.make_inpainting_problem(*shape, 0.3, 15.0, 21)
    sigma, lam, gam = prob.sigma, 0.0, 0.2 * prob.sigma ** 2
    y_obs = np.where(prob.mask > 0, prob.y, np.nan).astype(np.float32)
    rng = np.random.default_rng(3)
    x0 = np.stack([prob.x0, prob.x0 + 0.05 * rng.standard_normal(shape)]).astype(np.float32)
    x = torch.from_numpy(x0.copy()).cuda()
    yd = torch.from_numpy(y_obs).cuda()
    mean = torch.zeros_like(x)
    m2 = torch.zeros_like(x)
    P.pnp_inpaint_update(x, yd, None, sigma, 0.0, 1.0, lam, gam, prob.seed, 9, mean=mean, m2=m2,
                         n_kept=1)
    torch.cuda.synchronize()
    op = orc.Problem(prob.y, None, sigma, 0.0, 1.0, lam, gam, prob.seed, mask=prob.mask)
    for c in range(2):
        ref = orc.langevin_step(op, x0[c].astype(np.float64), 9, chain=c)
        got = x[c].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
        np.testing.assert_array_equal(mean[c].cpu().numpy(), got)   # first sample: mean = x
        assert not m2[c].cpu().numpy().any()


def test_one_step_fp32_with_prior(P, orc):
    """Ragged 72 x 136, FP32 denoiser, several t, mask 30 %, the chain started
    at the spline initialisation; every step compared from the GPU's state,
    then the FP32 Welford moments against FP64 two-pass over that trajectory."""
    prob = synth.make_inpainting_problem(72, 136, 0.3, 15.0, 33)
    dw = synth.workload_denoiser(1)
    gp = _gpu_problem(P, prob, P.Denoiser.from_weights(dw), burn_in=2)
    prm = gp.params()
    op = _oracle(orc, prob, prm, orc.Net.from_weights(dw))
    x_prev, t0 = gp.state()
    assert t0 == 0
    np.testing.assert_array_equal(x_prev[0], prob.x0.astype(np.float32))
    traj = []
    for t in range(6):
        gp.step(1)
        x_new, tt = gp.state()
        assert tt == t + 1
        ref = orc.langevin_step(op, x_prev[0].astype(np.float64), t)
        assert np.abs(x_new[0] - ref).max() <= 1e-5 * np.abs(ref).max(), t
        traj.append(x_new[0].astype(np.float64))
        x_prev = x_new
    mm, var, n = gp.moments(want_var=True)
    assert n == 4
    m_ref, v_ref = orc.moments_two_pass(np.stack(traj[2:]))
    np.testing.assert_allclose(mm, m_ref, rtol=0, atol=1e-6 * np.abs(m_ref).max())
    np.testing.assert_allclose(var, v_ref, rtol=1e-3, atol=1e-6 * v_ref.max())


def test_graph_eager_blocks_and_batch(P):
    """Graph replay = eager, any block split, batch = alone: bitwise."""
    prob = synth.make_inpainting_problem(128, 96, 0.3, 15.0, 44)
    dw = synth.workload_denoiser(2)
    den = P.Denoiser.from_weights(dw)
    res = []
    for graph, blocks, halo in [(True, (1, 1), 0), (False, (1, 1), 0), (True, (4, 4), 8),
                                (True, (2, 3), 8)]:
        P.pnp_set_graph_mode(graph)
        gp = _gpu_problem(P, prob, den, blocks=blocks, halo=halo, burn_in=1, precision="bf16")
        gp.run_chain(7, 1)
        res.append((gp.state()[0], gp.moments(want_var=True)[1]))
    P.pnp_set_graph_mode(True)
    for r in res[1:]:
        np.testing.assert_array_equal(res[0][0], r[0])
        np.testing.assert_array_equal(res[0][1], r[1])
    probs = [prob, synth.make_inpainting_problem(64, 80, 0.3, 15.0, 45)]
    jobs = [dict(y=p.y, h=None, sigma=p.sigma, mask=p.mask, x0=p.x0, seed=p.seed, burn_in=1)
            for p in probs]
    b = P.Batch(jobs, den, precision="bf16")
    b.run(7, 1)
    np.testing.assert_array_equal(b.job(0).state()[0], res[0][0])
    solo = _gpu_problem(P, probs[1], den, burn_in=1, precision="bf16")
    solo.run_chain(7, 1)
    np.testing.assert_array_equal(b.job(1).state()[0], solo.state()[0])


def test_full_size_sampled_bf16(P, orc):
    """1024 x 1024, 30 % mask, 8L x 64ch BF16 denoiser, direct layout (the
    benchmark's launch configuration): x+ at sampled pixels, the oracle's
    denoiser on unwrapped crops with K pixels of margin. Bound: the BF16 prior
    error c_prior 1 % max|G| (as for deconvolution) plus the FP32 bound."""
    prob = synth.make_inpainting_problem(1024, 1024, 0.3, 15.0, 1250)
    dw = synth.workload_denoiser(2)
    net = orc.Net.from_weights(dw)
    gp = _gpu_problem(P, prob, P.Denoiser.from_weights(dw), precision="bf16")
    prm = gp.params()
    K = net.K
    rng = np.random.default_rng(5)
    pix = [(0, 0), (0, 1023), (1023, 0), (1023, 1023), (511, 512), (3, 700)] + \
        [tuple(v) for v in rng.integers(0, 1024, size=(6, 2))]
    x = prob.x0.astype(np.float32)
    # max |G| on a 128 x 128 corner stands in for the whole image's in the bound
    gcrop = np.abs(x[:128, :128] - orc.denoise(x[:128, :128].astype(np.float64), net)).max()
    for t in (0, 999):
        gp.set_state(x, t)
        gp.step(1)
        xn, _ = gp.state()
        xi = orc.normals(prob.seed, t, 0, 1024 * 1024).reshape(1024, 1024)
        gam, c_prior = prm["gamma"], prm["alpha"] * prm["gamma"] / prm["eps"] ** 2
        got, ref, gmax = [], [], 0.0
        for (i, j) in pix:
            i0, i1, j0, j1 = max(0, i - K), min(1024, i + K + 1), max(0, j - K), min(1024, j + K + 1)
            xv = float(x[i, j])
            G = xv - orc.denoise(x[i0:i1, j0:j1].astype(np.float64), net)[i - i0, j - j0]
            gmax = max(gmax, abs(G))
            g = (xv - prob.y[i, j]) if prob.mask[i, j] > 0 else 0.0
            v = xv - gam * g / prob.sigma ** 2 - c_prior * G
            v += gam / prm["lam"] * (min(max(xv, 0.0), 1.0) - xv) + np.sqrt(2 * gam) * xi[i, j]
            got.append(xn[0][i, j])
            ref.append(v)
        got, ref = np.array(got), np.array(ref)
        bound = c_prior * 1e-2 * max(gmax, gcrop) + 1e-5 * np.abs(xn[0]).max()
        assert np.abs(got - ref).max() <= bound, (t, np.abs(got - ref).max(), bound)
