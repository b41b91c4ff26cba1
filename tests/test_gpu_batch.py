"""Batched and served forms (continuous batching) through the C ABI.

The defining property: a job's chain does not depend on the other jobs it is
batched with. Every job's state / moments in a batch or under the server
equal those of the same problem run alone, bitwise (same kernels, same
per-pixel summation order, per-job Philox stream and step counter).
"""
import time

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


@pytest.fixture(scope="module")
def den(P):
    return P.Denoiser.from_weights(synth.workload_denoiser(2))


def mixed_jobs(n=5, seed=11):
    rng = np.random.default_rng(seed)
    sizes = [(96, 80), (130, 257), (64, 64), (200, 150), (33, 300), (256, 256)][:n]
    jobs = []
    for k, (ny, nx) in enumerate(sizes):
        h, _ = synth.random_blur(rng)
        if h.shape[0] > min(ny, nx):
            h = synth.uniform_kernel(5)
        prob = synth.make_problem(ny, nx, h, float(rng.uniform(15, 40)), 7000 + k)
        jobs.append(dict(y=prob.y, h=prob.h, sigma=prob.sigma, seed=prob.seed, burn_in=3))
    return jobs


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batch_jobs_equal_alone(P, den, prec):
    jobs = mixed_jobs()
    b = P.Batch(jobs, den, precision=prec)
    b.run(10, 3)
    for k, jb in enumerate(jobs):
        alone = P.Problem(jb["y"], jb["h"], jb["sigma"], den, seed=jb["seed"], burn_in=3,
                          precision=prec)
        alone.run_chain(10, 3)
        xa, ta = alone.state()
        xb, tb = b.job(k).state()
        assert ta == tb == 10
        np.testing.assert_array_equal(xa, xb)
        ma, va, na = alone.moments(want_var=True)
        mb, vb, nb = b.job(k).moments(want_var=True)
        assert na == nb == 7
        np.testing.assert_array_equal(ma, mb)
        np.testing.assert_array_equal(va, vb)


def test_batch_launches_are_grouped(P, den):
    """One batch iteration launches one first layer, the shared conv layers and
    one residual / update launch per (stencil width, form), not one per job."""
    jobs = mixed_jobs(6) + mixed_jobs(6, seed=12)
    widths = {np.asarray(j["h"]).shape for j in jobs}
    b = P.Batch(jobs, den, precision="bf16")
    b.step(2)
    P.pnp_kernel_timer(True)            # eager launches, counted
    n0 = P.pnp_launch_count()
    b.step(1)
    b.sync()
    n = P.pnp_launch_count() - n0
    P.pnp_kernel_timer(False)
    K = 8
    assert n <= 2 * len(widths) + K, (n, len(widths))
    assert n < 3 * len(jobs) + K - 1


def test_batch_job_stepped_alone_between_batch_steps(P, den):
    """A batch job stepped through its own handle between batch steps keeps the
    same chain as the job run alone for the same total number of steps."""
    jobs = mixed_jobs(3)
    b = P.Batch(jobs, den, precision="fp32")
    b.step(3)
    b.job(1).step(1)
    b.step(2)
    b.sync()
    jb = jobs[1]
    alone = P.Problem(jb["y"], jb["h"], jb["sigma"], den, seed=jb["seed"], burn_in=3,
                      precision="fp32")
    alone.step(6)
    np.testing.assert_array_equal(b.job(1).state()[0], alone.state()[0])


def test_batch_one_step_parity_with_oracle(P, den, orc):
    """A batched job's one-step x+ matches the FP64 oracle (FP32 path)."""
    jobs = mixed_jobs(3)
    b = P.Batch(jobs, den, precision="fp32")
    j = 1
    jb = jobs[j]
    prm = b.job(j).params()
    x0 = np.clip(jb["y"], 0, 1).astype(np.float32)
    for k in range(len(jobs)):
        b.job(k).set_state(np.clip(jobs[k]["y"], 0, 1), 0)
    b.step(1)
    b.sync()
    x1, _ = b.job(j).state()
    op = orc.Problem(jb["y"], jb["h"], jb["sigma"], prm["alpha"], prm["eps"], prm["lam"],
                     prm["gamma"], jb["seed"], net=orc.Net.from_weights(synth.workload_denoiser(2)))
    ref = orc.langevin_step(op, x0.astype(np.float64), 0)
    assert np.abs(x1[0] - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_server_results_equal_alone(P, den, prec):
    jobs = mixed_jobs()
    Ts = [12, 7, 20, 9, 15]
    srv = P.Server(den, precision=prec, hbm_budget_bytes=8 << 30, round_iters=4)
    ids = []
    for k, jb in enumerate(jobs):
        ids.append(srv.submit(jb["y"], jb["h"], jb["sigma"], Ts[k], 2, seed=jb["seed"]))
        time.sleep(0.01 * (k % 2))          # staggered arrivals join running jobs
    for jid in ids:
        assert srv.wait(jid, 300) == "done"
    for k, jb in enumerate(jobs):
        st, mm, sd = srv.poll(ids[k])
        assert st == "done"
        alone = P.Problem(jb["y"], jb["h"], jb["sigma"], den, seed=jb["seed"], burn_in=2,
                          precision=prec)
        alone.run_chain(Ts[k], 2)
        ma, sa, _ = alone.moments()
        np.testing.assert_array_equal(mm, ma)
        np.testing.assert_array_equal(sd, sa)
        t = srv.times(ids[k])
        assert 0 <= t["submit"] <= t["admit"] <= t["done"]
    srv.close()


def test_server_admission_respects_budget(P, den):
    """A budget that fits about two jobs: the rest queue, usage never exceeds it,
    and every job still finishes with its alone result."""
    jobs = [dict(y=synth.make_problem(160, 160, synth.gaussian_kernel(7, 1.5), 30.0, 8000 + k).y,
                 h=synth.gaussian_kernel(7, 1.5).astype(np.float32), sigma=0.01, seed=8000 + k)
            for k in range(5)]
    one = 160 * 160 * (4 + 20) + 256 * 160 * 160 + 4096 + 49 * 4 + 4096
    budget = int(2.5 * one)
    srv = P.Server(den, precision="bf16", hbm_budget_bytes=budget, round_iters=2)
    ids = [srv.submit(jb["y"], jb["h"], jb["sigma"], 6, 1, seed=jb["seed"]) for jb in jobs]
    peak = 0
    while True:
        s = srv.stats()
        peak = max(peak, s["used_bytes"])
        assert s["active"] <= 2
        if all(srv.poll(i, fetch=False)[0] == "done" for i in ids):
            break
        time.sleep(0.002)
    assert peak <= budget
    # a job that can never fit is refused at submission
    big = synth.make_problem(512, 512, synth.uniform_kernel(5), 20.0, 1).y
    with pytest.raises(P.PnpError) as e:
        srv.submit(big, synth.uniform_kernel(5), 0.05, 5, 1)
    assert e.value.status == 3   # PNP_EBUSY
    srv.close()


def test_server_cancel_leaves_others_unchanged(P, den):
    jobs = mixed_jobs(4)
    srv = P.Server(den, precision="bf16", hbm_budget_bytes=8 << 30, round_iters=2)
    ids = [srv.submit(jb["y"], jb["h"], jb["sigma"], 30, 5, seed=jb["seed"]) for jb in jobs]
    srv.cancel(ids[1])
    for k, jid in enumerate(ids):
        st = srv.wait(jid, 300)
        assert st == ("cancelled" if k == 1 else "done")
    for k in (0, 2, 3):
        jb = jobs[k]
        alone = P.Problem(jb["y"], jb["h"], jb["sigma"], den, seed=jb["seed"], burn_in=5,
                          precision="bf16")
        alone.run_chain(30, 5)
        np.testing.assert_array_equal(srv.poll(ids[k])[1], alone.moments()[0])
    srv.close()
