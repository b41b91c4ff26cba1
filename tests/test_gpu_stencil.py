"""Stencil tile shapes: every shape the autotuner can pick gives bitwise the
same r = Hx - y, H^T r and x-update (each output is the same fixed-order FP32
sum), so the timing-based choice never changes a chain. Cases cover ragged
tiles, widths that are not multiples of 4, non-square kernels and the smallest
and largest kernel widths; parity with the oracle is in test_gpu_ops and the
chain tests.
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
    yield P
    P.pnp_set_stencil_tile(-1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


CASES = [(33, 300, 7, 7), (128, 128, 9, 9), (100, 72, 5, 13), (40, 40, 31, 31), (17, 9, 3, 1),
         (70, 130, 21, 3), (64, 64, 1, 1)]


@pytest.mark.parametrize("ny,nx,kh,kw", CASES)
def test_blur_adjoint_same_for_every_tile(P, orc, ny, nx, kh, kw):
    rng = np.random.default_rng(ny + 1000 * kw)
    x = dev(rng.standard_normal((2, ny, nx)))
    y = dev(rng.standard_normal((ny, nx)))
    h = rng.random((kh, kw))
    h = dev(h / h.sum())
    outs = []
    for k in range(P.pnp_stencil_tile_count()):
        P.pnp_set_stencil_tile(k)
        r = torch.empty((2, ny, nx), device="cuda")
        g = torch.empty_like(r)
        P.pnp_blur(x, y, h, r)
        P.pnp_blur_adjoint(r, h, g, scale=0.25)
        torch.cuda.synchronize()
        outs.append((r.cpu().numpy(), g.cpu().numpy()))
    P.pnp_set_stencil_tile(-1)
    for r, g in outs[1:]:
        np.testing.assert_array_equal(r, outs[0][0])
        np.testing.assert_array_equal(g, outs[0][1])
    hh = h.cpu().numpy().astype(np.float64)
    rr = orc.blur(x[1].cpu().numpy().astype(np.float64), hh) - y.cpu().numpy()
    np.testing.assert_allclose(outs[0][0][1], rr, rtol=0, atol=2e-6 * np.abs(rr).max())


@pytest.mark.parametrize("ny,nx,kh,kw", CASES[:4])
def test_update_same_for_every_tile(P, ny, nx, kh, kw):
    rng = np.random.default_rng(7 * ny + kw)
    x0 = rng.random((3, ny, nx)).astype(np.float32)
    r = dev(rng.standard_normal((3, ny, nx)))
    d = dev(rng.random((3, ny, nx)))
    h = rng.random((kh, kw))
    h = dev(h / h.sum())
    m0 = rng.random((3, ny, nx)).astype(np.float32)
    outs = []
    for k in range(P.pnp_stencil_tile_count()):
        P.pnp_set_stencil_tile(k)
        x = dev(x0)
        mean, m2 = dev(m0), dev(m0 * 0.5)
        P.pnp_langevin_update(x, r, d, h, sigma=0.1, alpha=1.0, eps=0.1, lam=0.5, gamma=1e-3,
                              seed=1234 + ny, t=5, noise=True, mean=mean, m2=m2, n_kept=3)
        torch.cuda.synchronize()
        outs.append([a.cpu().numpy() for a in (x, mean, m2)])
    P.pnp_set_stencil_tile(-1)
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_chain_same_for_every_tile(P, prec):
    """Forced shapes and the autotuned choice step identical chains (the update's
    last block also advances the device step counter: t must reach 6)."""
    den = P.Denoiser.from_weights(synth.workload_denoiser(1 if prec == "fp32" else 2))
    prob = synth.make_problem(96, 136, synth.gaussian_kernel(7, 1.5), 30.0, 515)
    res = []
    for k in [-1] + list(range(P.pnp_stencil_tile_count())):
        P.pnp_set_stencil_tile(k)
        p = P.Problem(prob.y, prob.h, prob.sigma, den, seed=99, burn_in=2, precision=prec)
        if k == -1:
            bt, ut, _ = p.stencil_tiles()
            assert 0 <= bt < P.pnp_stencil_tile_count() and 0 <= ut < P.pnp_stencil_tile_count()
        p.run_chain(6, 2)
        x, t = p.state()
        assert t == 6
        res.append((x, p.moments()[0]))
    P.pnp_set_stencil_tile(-1)
    for x, m in res[1:]:
        np.testing.assert_array_equal(x, res[0][0])
        np.testing.assert_array_equal(m, res[0][1])


@pytest.mark.parametrize("kind", ["gaussian", "uniform", "motion", "uniform15", "gaussian17"])
def test_separable_and_direct_one_step_match_oracle(P, orc, kind):
    """Rank-one kernels of up to 15 taps take the one-pass gradient
    (H^T H) x - H^T y over separable taps of H^T H (up to 29 taps), larger
    rank-one kernels the two-pass separable residual and adjoint, others the
    2-D stencils; every way one FP32 step (no prior) is within 1e-5 of the
    oracle's H^T (H x - y) form, on a ragged 77 x 133 image, from states at two
    step parities (the one-pass form alternates two state buffers)."""
    h = {"gaussian": synth.gaussian_kernel(9, 2.0), "uniform": synth.uniform_kernel(7),
         "motion": synth.motion_kernel(11, 0.7), "uniform15": synth.uniform_kernel(15),
         "gaussian17": synth.gaussian_kernel(17, 3.0)}[kind]
    prob = synth.make_problem(77, 133, h, 25.0, 321)
    gp = P.Problem(prob.y, prob.h, prob.sigma, None, seed=prob.seed, burn_in=0)
    assert gp.stencil_tiles()[2] == (kind != "motion")
    prm = gp.params()
    rng = np.random.default_rng(5)
    x0 = rng.random(prob.shape).astype(np.float32)
    for t in (0, 3, 4):
        gp.set_state(x0, t)
        gp.step(1)
        x1, _ = gp.state()
        op = orc.Problem(prob.y, prob.h, prob.sigma, 0.0, prm["eps"], prm["lam"], prm["gamma"],
                         prob.seed)
        ref = orc.langevin_step(op, x0.astype(np.float64), t)
        assert np.abs(x1[0] - ref).max() <= 1e-5 * np.abs(ref).max()
