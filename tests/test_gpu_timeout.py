"""Bounded device-side waits: a tensor-core layer whose wait runs out reports
PNP_ETIMEOUT to the host instead of hanging the GPU, and the device stays
usable.

The fault is made deliberately and safely through a one-shot test hook
(pnp_debug_inject_tc_timeout): CTA 0 of the next F -> F layer skips issuing
its second row load, so nothing is in flight for that row, and the launch's
waits give up after 1e6 SM cycles (about 0.5 ms) instead of about two
seconds. The CTA waiting for the missing row then aborts: its producer and MMA
threads wait for their own copies and MMAs already in flight, the CTA frees
its tensor memory and sets the caller's timeout flag. No wait is left without
a limit and nothing faults; the next normal call must give bitwise the result
of a fresh run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BUDGET = 1_000_000


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_00870_b300 as P
    return P


def test_problem_reports_timeout_then_recovers_bitwise(P):
    prob = synth.make_problem(64, 64, synth.uniform_kernel(5), 25.0, 77)
    den = P.Denoiser.from_weights(synth.workload_denoiser(2))      # K = 8, F = 64
    x0 = np.clip(prob.y + 0.02, 0, 1).astype(np.float32)
    P.pnp_set_graph_mode(False)            # the hook only reaches eager launches
    try:
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed, precision="bf16")
        gp.set_state(x0, 0)
        P.pnp_debug_inject_tc_timeout(0, 1, BUDGET)
        gp.step(1)
        with pytest.raises(P.PnpError) as e:
            gp.sync()
        assert e.value.status == 5 and "bounded wait" in str(e.value)
        gp.sync()                          # reported once, then cleared
        gp.set_state(x0, 0)
        gp.step(2)
        got, t = gp.state()
        fresh = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed, precision="bf16")
        fresh.set_state(x0, 0)
        fresh.step(2)
        want, _ = fresh.state()
        assert t == 2
        np.testing.assert_array_equal(got, want)
    finally:
        P.pnp_set_graph_mode(True)


def test_denoise_status_reports_timeout_then_recovers_bitwise(P):
    den = P.Denoiser.from_weights(synth.denoiser_weights(8, 64, seed=21))
    x = torch.from_numpy(synth.ground_truth(96, 130, seed=8).astype(np.float32))[None].cuda()
    want = den.denoise(x, precision="bf16")
    den.status()
    P.pnp_debug_inject_tc_timeout(0, 1, BUDGET)
    den.denoise(x, precision="bf16")
    with pytest.raises(P.PnpError) as e:
        den.status()
    assert e.value.status == 5
    den.status()
    got = den.denoise(x, precision="bf16")
    den.status()
    assert torch.equal(got, want)


def test_inject_hook_validates_its_arguments(P):
    for args in ((-1, 0, BUDGET), (0, -1, BUDGET), (0, 0, 10)):
        with pytest.raises(P.PnpError):
            P.pnp_debug_inject_tc_timeout(*args)
        with pytest.raises(P.PnpError):
            P.pnp_debug_inject_update_timeout(*args)


def test_pipelined_update_reports_timeout_then_recovers_bitwise(P):
    """The one-pass update's TMA-filled windows complete on mbarriers with
    bounded waits. CTA 0 skips issuing the window of its first tile (nothing is
    in flight for it), its wait gives up after BUDGET cycles, it reports
    PNP_ETIMEOUT and still arrives on the step counter (t advances); after
    pnp_set_state the chain steps bitwise as a fresh problem does."""
    prob = synth.make_problem(256, 256, synth.gaussian_kernel(7, 1.5), 25.0, 79)   # one-pass form
    x0 = np.clip(prob.y + 0.02, 0, 1).astype(np.float32)
    P.pnp_set_graph_mode(False)            # the hook only reaches eager launches
    try:
        gp = P.Problem(prob.y, prob.h, prob.sigma, None, seed=prob.seed)
        gp.set_state(x0, 0)
        P.pnp_debug_inject_update_timeout(0, 0, BUDGET)
        gp.step(1)
        with pytest.raises(P.PnpError) as e:
            gp.sync()
        assert e.value.status == 5 and "bounded wait" in str(e.value)
        gp.sync()                          # reported once, then cleared
        assert gp.state()[1] == 1          # every CTA arrived: t advanced once
        gp.set_state(x0, 0)
        gp.step(2)
        got, t = gp.state()
        fresh = P.Problem(prob.y, prob.h, prob.sigma, None, seed=prob.seed)
        fresh.set_state(x0, 0)
        fresh.step(2)
        want, _ = fresh.state()
        assert t == 2
        np.testing.assert_array_equal(got, want)
    finally:
        P.pnp_set_graph_mode(True)
