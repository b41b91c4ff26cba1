"""Large blur kernels (the paper's 65^2-129^2 motion blurs, Sec. IV-A) on the
wide-window stencil, against the FP64 oracle's direct circular sums.

Bounds: r = Hx - y and H^T r within 2e-6 * max|ref| (FP32 sums of up to a few
thousand taps of a normalised kernel); the one-step x-update within
1e-5 * max|x+| as for small kernels. The problem API (host-built list of
nonzero taps) and the operator entry points (walk of h skipping zeros) use
the same order, so they agree bitwise.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _kernel(kind, L, seed=0):
    if kind == "motion":
        return synth.motion_kernel(L, 0.3 + 0.4 * seed)
    rng = np.random.default_rng(seed)
    h = rng.random((L, L + 2))            # dense, non-square, not rank one
    return h / h.sum()


@pytest.mark.parametrize("ny,nx,kind,L", [(150, 210, "motion", 65), (97, 131, "dense", 33),
                                          (256, 256, "motion", 129), (130, 140, "motion", 129)])
def test_blur_and_adjoint_against_oracle(P, orc, ny, nx, kind, L):
    h = _kernel(kind, L, 1).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(ny)
    x = rng.random((2, ny, nx))
    y = rng.random((ny, nx))
    r = torch.empty((2, ny, nx), device="cuda")
    g = torch.empty_like(r)
    P.pnp_blur(dev(x), dev(y), dev(h), r)
    P.pnp_blur_adjoint(r, dev(h), g, scale=0.5)
    torch.cuda.synchronize()
    for c in range(2):
        xf = x[c].astype(np.float32).astype(np.float64)
        rr = orc.blur(xf, h) - y.astype(np.float32)
        got = r[c].cpu().numpy()
        np.testing.assert_allclose(got, rr, rtol=0, atol=2e-6 * np.abs(rr).max())
        gg = 0.5 * orc.blur_adj(got.astype(np.float64), h)
        np.testing.assert_allclose(g[c].cpu().numpy(), gg, rtol=0, atol=2e-6 * np.abs(gg).max())


def test_problem_step_equals_operators_and_oracle(P, orc):
    """Ragged 200 x 300, motion 65, FP32 denoiser: the problem's step equals
    pnp_blur + pnp_langevin_update on the same state bitwise (prior off), and
    the oracle's within 1e-5 (prior on)."""
    prob = synth.make_problem(200, 300, synth.motion_kernel(65, 0.7), 25.0, 77)
    x0 = np.clip(prob.y + 0.02, 0, 1).astype(np.float32)
    # prior off: problem vs operators
    gp = P.Problem(prob.y, prob.h, prob.sigma, None, seed=prob.seed)
    prm = gp.params()
    gp.set_state(x0, 4)
    gp.step(1)
    xp, _ = gp.state()
    x = dev(x0[None])
    r = torch.empty_like(x)
    P.pnp_blur(x, dev(prob.y), dev(prob.h), r)
    P.pnp_langevin_update(x, r, None, dev(prob.h), prob.sigma, 0.0, prm["eps"], prm["lam"],
                          prm["gamma"], prob.seed, 4)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy()[0], xp[0])
    op0 = orc.Problem(prob.y, prob.h, prob.sigma, 0.0, prm["eps"], prm["lam"], prm["gamma"],
                      prob.seed)
    ref0 = orc.langevin_step(op0, x0.astype(np.float64), 4)
    assert np.abs(xp[0] - ref0).max() <= 1e-5 * np.abs(ref0).max()
    # prior on
    dw = synth.workload_denoiser(1)
    gq = P.Problem(prob.y, prob.h, prob.sigma, P.Denoiser.from_weights(dw), seed=prob.seed,
                   burn_in=0)
    prq = gq.params()
    gq.set_state(x0, 11)
    gq.step(1)
    xq, _ = gq.state()
    op = orc.Problem(prob.y, prob.h, prob.sigma, prq["alpha"], prq["eps"], prq["lam"],
                     prq["gamma"], prob.seed, net=orc.Net.from_weights(dw))
    ref = orc.langevin_step(op, x0.astype(np.float64), 11)
    assert np.abs(xq[0] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_graph_eager_and_batch_with_wide_kernels(P):
    prob = synth.make_problem(160, 192, synth.motion_kernel(65, 1.1), 25.0, 78)
    dw = synth.workload_denoiser(2)
    den = P.Denoiser.from_weights(dw)
    out = []
    for graph in (True, False):
        P.pnp_set_graph_mode(graph)
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=3, burn_in=2, precision="bf16")
        gp.run_chain(9, 2)
        out.append((gp.state()[0], gp.moments(want_var=True)[1]))
    P.pnp_set_graph_mode(True)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    b = P.Batch([dict(y=prob.y, h=prob.h, sigma=prob.sigma, seed=3, burn_in=2),
                 dict(y=prob.y[:96, :128], h=synth.uniform_kernel(9), sigma=prob.sigma, seed=4)],
                den, precision="bf16")
    b.run(9, 2)
    np.testing.assert_array_equal(b.job(0).state()[0], out[0][0])


@pytest.mark.parametrize("n,L,nwin", [(2048, 65, 8), (4096, 129, 4)])
def test_paper_scale_sampled_bf16(P, orc, n, L, nwin):
    """The paper's sizes (2048^2 with 65^2, 4096^2 with 129^2 motion blur),
    BF16 denoiser, direct layout: x+ at windows (corners, a border, the
    interior) against the oracle's transition evaluated on those windows; the
    bound adds the prior term's BF16 error c_prior 1 % max|G| (oracle G on
    crops around the windows) to the FP32 one-step bound."""
    prob = synth.make_problem(n, n, synth.motion_kernel(L, 0.9), 25.0, 4000 + L)
    dw = synth.workload_denoiser(2)
    net = orc.Net.from_weights(dw)
    gp = P.Problem(prob.y, prob.h, prob.sigma, P.Denoiser.from_weights(dw), seed=prob.seed,
                   precision="bf16")
    prm = gp.params()
    op = orc.Problem(prob.y, prob.h, prob.sigma, prm["alpha"], prm["eps"], prm["lam"],
                     prm["gamma"], prob.seed, net=net)
    rng = np.random.default_rng(L)
    w = 2
    wins = [(0, 0), (n - w, n - w), (n // 2, 3)][:nwin] + \
        [tuple(int(v) for v in rng.integers(0, n - w, size=2)) for _ in range(max(nwin - 3, 1))]
    x0 = np.clip(prob.y + 0.05 * rng.standard_normal(prob.shape), -0.1, 1.1).astype(np.float32)
    t = 17
    gp.set_state(x0, t)
    gp.step(1)
    xn, _ = gp.state()
    K = net.K
    c_prior = prm["alpha"] * prm["gamma"] / prm["eps"] ** 2
    x64 = x0.astype(np.float64)
    err, gmax = 0.0, 0.0
    for (i, j) in wins:
        ref = orc.langevin_step_window(op, x64, t, i, j, w, w)
        err = max(err, np.abs(xn[0][i:i + w, j:j + w] - ref).max())
        a0, a1, b0, b1 = max(0, i - K), min(n, i + w + K), max(0, j - K), min(n, j + w + K)
        c = x64[a0:a1, b0:b1]
        gmax = max(gmax, np.abs((c - orc.denoise(c, net))[i - a0:i - a0 + w, j - b0:j - b0 + w]).max())
    gcrop = np.abs(x64[:96, :96] - orc.denoise(x64[:96, :96], net)).max()
    bound = c_prior * 1e-2 * max(gmax, gcrop) + 1e-5 * np.abs(xn[0]).max()
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("ny,nx,L,prior", [(256, 256, 65, False), (256, 512, 129, True),
                                           (512, 128, 65, True)])
def test_spectral_gradient_matches_direct_and_oracle(P, orc, ny, nx, L, prior):
    """Power-of-two images take the spectral gradient (FFT of x, |H^|^2,
    inverse FFT) instead of the direct wide stencil. One step from the same
    state with each, and the oracle's direct FP64 sums: both within
    1e-5 max|x+| of the oracle (the FP32 FFT's rounding, a few 1e-7 of the
    gradient's scale times gamma / sigma^2, stays far below it)."""
    prob = synth.make_problem(ny, nx, synth.motion_kernel(L, 0.45), 25.0, 90 + L)
    dw = synth.workload_denoiser(1)
    den = P.Denoiser.from_weights(dw) if prior else None
    x0 = np.clip(prob.y + 0.03 * np.random.default_rng(L).standard_normal(prob.shape), -0.1,
                 1.1).astype(np.float32)
    out = {}
    try:
        for spectral in (True, False):
            P.pnp_set_spectral(spectral)
            gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed, burn_in=0)
            prm = gp.params()
            gp.set_state(x0, 5)
            gp.step(1)
            out[spectral] = gp.state()[0][0]
    finally:
        P.pnp_set_spectral(True)
    alpha = prm["alpha"] if prior else 0.0
    op = orc.Problem(prob.y, prob.h, prob.sigma, alpha, prm["eps"], prm["lam"], prm["gamma"],
                     prob.seed, net=orc.Net.from_weights(dw) if prior else None)
    ref = orc.langevin_step(op, x0.astype(np.float64), 5)
    bound = 1e-5 * np.abs(ref).max()
    e_sp, e_dir = np.abs(out[True] - ref).max(), np.abs(out[False] - ref).max()
    print("%dx%d L=%d: spectral %.3e, direct %.3e, |spectral - direct| %.3e (bound %.3e)" % (
        ny, nx, L, e_sp, e_dir, np.abs(out[True] - out[False]).max(), bound))
    assert e_sp <= bound and e_dir <= bound
