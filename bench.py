#!/usr/bin/env python3
"""Throughput benchmark of the PnP-ULA sampler on B300.

Default (``--workload serve``, the headline): the serving form. A seeded
Poisson stream of sampling jobs (20 jobs/s; sizes uniform over {512, 1024,
2048, 4096}^2; blur and noise drawn as in the batched workload; 200 burn-in +
800 kept iterations; MMSE and std returned) is continuously batched by the
library's server with the BF16 denoiser. A step is one job of the stream:
``--steps K`` jobs are timed (at most 64), after ``--warmup W`` iterations on
every distinct job size. value = the stream's pixel-iterations / the server's
device time (CUDA events around each round's launches); e2e = the same
pixel-iterations / wall time from the first submission to the last completion
(host inputs in, host MMSE/std out). Beside it: p50/p99 job latency, the FP32
one-job-at-a-time baseline (FP32 iteration time measured per size over 50
iterations, FIFO over the same arrivals: modelled), MMSE PSNR of a served BF16
job against its FP32 plain chain, the tensor-core conv roofline from a timed
batch pass over the stream's jobs, the FP64 oracle on the host cores, and the
single-job 1024^2 and 8192^2 workloads nested as extra keys.

A step of every other workload is one full x-update of the chain (Eq. 8 /
Algorithm 1 x-part): blur residual, block-wise DnCNN-form denoiser, fused
Langevin update with Philox noise and Welford moments. Metric:
Mpixel-iterations/s = pixels x iterations / time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload serve|deconv1024|deconv8192|deconv128|motion2048|motion4096|
                                   inpaint1024|poisson1024|ddfb1024|batch48]
                       [--no-quality] [--no-nested] [--jobs M]
deconv1024: 1024 x 1024 Gaussian deconvolution, 9 x 9 uniform blur, 20 dB
BSNR, 8-layer 64-channel seeded denoiser, 4 x 4 blocks (BF16, with the FP32
plain form, the FP8 variant and the MMSE PSNR of each beside it).
ddfb1024: the deconv1024 posterior with the DDFB denoiser (Sec. II-B, Example
2: K = 4 unrolled dual forward-backward layers, P = 64 filters) in FP32.
inpaint1024: Gaussian-noise inpainting (Sec. IV-A: H = diag(mask), 30 % of the
pixels observed, 15 dB input SNR, x started at the cubic interpolant of y).
poisson1024: the Poisson-noise sampler (Sec. IV-B: AXDA split, x-update with
the coupling gradients, PSGLA updates of z1 and z2) on 1024 x 1024 counts at
peak eta = 250, same blur and denoiser as deconv1024.
Multi-GPU (torchrun): every rank runs an independent replica of the workload
(independent chains, no data-path collective); value = all ranks' pixel-
iterations / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "PnP-ULA Mpixel-iters/s (BF16 serve vs FP32 plain) at equal PSNR; p50/p99 latency"
UNIT = "Mpixel-iters/s"

WORKLOADS = {
    "deconv1024": 2,   # 1024^2, uniform 9x9, 20 dB, K=8 F=64, 4x4 blocks, 2000 it (500 burn-in)
    "deconv8192": 3,   # 8192^2, Gaussian 13x13 s=3, 30 dB, K=8 F=64, 16x16 blocks
    "deconv128": 1,    # 128^2, Gaussian 7x7 s=1.5, 30 dB, K=4 F=16, 2x2 blocks
    "batch48": 4,      # 48 problems, sizes log-uniform 256..2048, blur/BSNR mix, BF16
    "serve": 5,        # Poisson arrivals (20/s), sizes {512..4096}^2, 200 + 800 iterations
    "poisson1024": 2,  # Poisson counts, eta = 250, rho1 = 10, rho2 = 1e-3; blur/denoiser of deconv1024
    "inpaint1024": 2,  # 30 % observed pixels, 15 dB input SNR, spline start; denoiser of deconv1024
    "ddfb1024": 2,     # the deconv1024 posterior with the DDFB prior (K=4, P=64), FP32
    "motion2048": 6,   # 2048^2, 65x65 motion blur, 25 dB, K=8 F=64 (paper scale)
    "motion4096": 7,   # 4096^2, 129x129 motion blur, 25 dB, K=8 F=64 (paper scale)
}
POISSON = dict(eta=250.0, rho1=10.0, rho2=1e-3)


def poisson_problem(rank=0):
    """Counts y ~ Poisson(eta H xbar) on the deconv1024 image and blur."""
    w = synth.WORKLOADS[2]
    return synth.make_poisson_problem(w["ny"], w["nx"], synth.blur_from_spec(w["blur"]),
                                      POISSON["eta"], synth.gt_seed(2, rank) + 50)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    sm_max=d.get("sm_max_mhz", 2032.0), src="measured")
    return dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, sm_max=2032.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
                    samples=len(self.rows))


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Replicas: every rank runs its own independent problems (no data-path
# collective); timing is bracketed by barriers and the whole-job rate is all
# ranks' pixel-iterations over the slowest rank's time.
def rank_barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _rank_reduce(v, ws, op, device):
    if ws == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return t.item()


def rank_max(v, ws, device="cuda"):
    import torch.distributed as dist
    return _rank_reduce(v, ws, dist.ReduceOp.MAX if ws > 1 else None, device)


def rank_sum(v, ws, device="cuda"):
    import torch.distributed as dist
    return _rank_reduce(v, ws, dist.ReduceOp.SUM if ws > 1 else None, device)


def replica_rate(pix_iters, seconds, ws, device="cuda"):
    """(Mpixel-iters/s of the whole job, slowest rank's seconds)."""
    tot = rank_sum(pix_iters, ws, device)
    slow = rank_max(seconds, ws, device)
    return tot / slow / 1e6, slow


def inpainting_problem(rank=0):
    w = synth.WORKLOADS[2]
    return synth.make_inpainting_problem(w["ny"], w["nx"], 0.3, 15.0, synth.gt_seed(2, rank) + 50)


def ddfb_net(P_=None):
    dd = synth.ddfb_weights(4, 64, 11)
    return dd


def _oracle_setup(cfg_id, crop, poisson=False, inpaint=False, ddfb=False):
    import oracle
    if inpaint:
        prob = inpainting_problem()
        dw = synth.workload_denoiser(cfg_id)
        crop = min(crop, prob.shape[0], prob.shape[1])
        lam, gam = oracle.stepsizes(1.0, prob.sigma, 1.0, prob.sigma, dw.lipschitz)
        op = oracle.Problem(prob.y[:crop, :crop], None, prob.sigma, 1.0, prob.sigma, lam, gam,
                            prob.seed, net=oracle.Net.from_weights(dw),
                            mask=prob.mask[:crop, :crop])
        return oracle, prob, op, crop
    if poisson:
        prob = poisson_problem()
        dw = synth.workload_denoiser(cfg_id)
        crop = min(crop, prob.shape[0], prob.shape[1])
        lam, gam, k1, k2 = oracle.poisson_stepsizes(float(np.abs(prob.h).sum()), prob.eta,
                                                    POISSON["rho1"], POISSON["rho2"], 1.0, 0.05,
                                                    dw.lipschitz)
        op = oracle.PoissonProblem(prob.y[:crop, :crop], prob.h, prob.eta, POISSON["rho1"],
                                   POISSON["rho2"], k1, k2, 1.0, 0.05, lam, gam, prob.seed,
                                   net=oracle.Net.from_weights(dw))
        return oracle, prob, op, crop
    if cfg_id == 4:
        prob = synth.batched_problems(1, seed=4000)[0]
    elif cfg_id == 5:
        sp = synth.serving_jobs(1, seed=5000)[0]
        prob = synth.make_problem(sp["size"], sp["size"], sp["h"], sp["bsnr"], sp["gt_seed"])
    else:
        prob = synth.workload_problem(cfg_id)
    dw = synth.workload_denoiser(cfg_id)
    # the crop holds at least two kernel widths (the paper's 129 x 129 blur)
    crop = min(max(crop, 2 * prob.h.shape[0]), prob.shape[0], prob.shape[1])
    y = prob.y[:crop, :crop]
    lam, gam = oracle.stepsizes(float(np.abs(prob.h).sum()), prob.sigma, 1.0, prob.sigma,
                                dw.lipschitz)
    if ddfb:
        dd = ddfb_net()
        lam, gam = oracle.stepsizes(float(np.abs(prob.h).sum()), prob.sigma, 1.0, prob.sigma, 1.0)
        op = oracle.Problem(y, prob.h, prob.sigma, 1.0, prob.sigma, lam, gam, prob.seed,
                            ddfb=oracle.Ddfb(dd.filters, dd.gammas, dd.ht))
        return oracle, prob, op, crop
    op = oracle.Problem(y, prob.h, prob.sigma, 1.0, prob.sigma, lam, gam, prob.seed,
                        net=oracle.Net.from_weights(dw))
    return oracle, prob, op, crop


class _OracleChain:
    """One oracle iteration at a time on the crop: the Gaussian x-update, or
    the Poisson x-update followed by the z-updates."""

    def __init__(self, oracle, op, crop, poisson, x0=None):
        self.o, self.op, self.poisson = oracle, op, poisson
        self.x = np.zeros((crop, crop)) if x0 is None else np.array(x0[:crop, :crop], np.float64)
        self.z1 = np.zeros((crop, crop))
        self.z2 = np.zeros((crop, crop))

    def step(self, t):
        if self.poisson:
            self.x, self.z1, self.z2 = self.o.poisson_step(self.op, self.x, self.z1, self.z2, t)
        else:
            self.x = self.o.langevin_step(self.op, self.x, t)


def oracle_baseline(cfg_id, budget_s=20.0, crop=128, poisson=False, inpaint=False, ddfb=False):
    """The FP64 oracle as it stands, on a bounded sample of the workload:
    whole iterations on a crop of the image (same blur, noise level and
    network), on this host's cores."""
    oracle, prob, op, crop = _oracle_setup(cfg_id, crop, poisson, inpaint, ddfb)
    ny, nx = prob.shape
    ch = _OracleChain(oracle, op, crop, poisson, prob.x0 if inpaint else None)
    t0 = time.perf_counter()
    it = 0
    while True:
        ch.step(it)
        it += 1
        if time.perf_counter() - t0 > budget_s or it >= 64:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(value=crop * crop * it / dt / 1e6, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{it} FP64 oracle iterations on a {crop}x{crop} crop of the "
                       f"{ny}x{nx} workload (same blur, noise, network)")


def run_reference(args):
    """Reference arm: the FP64 oracle; one step = one oracle iteration on a crop
    of the workload, the crop sized so that the whole run stays within minutes."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    cfg_id = WORKLOADS[args.workload]
    steps = max(1, args.steps)
    n = args.warmup + steps
    crop = 128 if n <= 60 else (64 if n <= 250 else 32)
    poisson = args.workload == "poisson1024"
    inpaint = args.workload == "inpaint1024"
    oracle, prob, op, crop = _oracle_setup(cfg_id, crop, poisson, inpaint,
                                           args.workload == "ddfb1024")
    ch = _OracleChain(oracle, op, crop, poisson, prob.x0 if inpaint else None)
    for it in range(args.warmup):
        ch.step(it)
    t0 = time.perf_counter()
    for it in range(args.warmup, n):
        ch.step(it)
    dt = time.perf_counter() - t0
    val = crop * crop * steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"each step one FP64 oracle iteration on a {crop}x{crop} crop of the "
              f"{prob.shape[0]}x{prob.shape[1]} workload (same blur, noise, network)")
    if cfg_id == 5:
        sample += "; the image is the first job of the serving stream"
        wname = "serve"
    elif cfg_id == 4:
        wname = "batch48"
    else:
        wname = (args.workload if poisson or inpaint or args.workload == "ddfb1024"
                 else synth.WORKLOADS[cfg_id]["name"])
    line = dict(metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus, steps=steps,
                warmup=args.warmup, ms_per_step=1e3 * dt / steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=f"{wname} (oracle, bounded crop sample)"),
                cpu_baseline=dict(kind="oracle", cores=cores, sample=sample, value=val, unit=UNIT),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def _percentile(v, q):
    v = sorted(v)
    if not v:
        return None
    k = (len(v) - 1) * q / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def _fp32_iter_time(P, torch, den, prob, stream, iters=50):
    """Device time of one FP32 plain iteration (graph replay, CUDA events on
    the problem's stream, mean over `iters` iterations after 3 warm-up ones)."""
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, seed=prob.seed, precision="fp32",
                   stream=stream.cuda_stream)
    gp.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gp.step(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    gp.close()
    return e0.elapsed_time(e1) / iters / 1e3


KTIMERS = ("blur", "update", "conv_fp32", "conv_tc", "conv_edge", "conv_last", "zupdate")


def _source_sha(kernel):
    """Short hash of the CUDA source a kernel is built from (ties a committed
    ncu traffic figure to the kernel version it was measured on)."""
    import hashlib
    name = ("k_conv_tc.cu" if kernel.startswith("k_conv_tc") or kernel.startswith("k_first_tc")
            else "k_ddfb.cu" if kernel.startswith("k_ddfb")
            else "k_update_os.cu" if kernel.startswith("k_update_os")
            else "k_spectral.cu" if kernel.startswith("k_sp_") else "k_stencil.cu")
    path = os.path.join(ROOT, "paper_2511_00870_b300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:12]


def ncu_traffic(kernel, workload, precision, npix=None):
    """(DRAM bytes per launch, note) of `kernel` from the committed ncu summary,
    only when the line was captured on the current kernel source. Without a
    line for this workload, a line of the same kernel and precision that
    records the pixels of its captured launch is scaled to `npix` pixels (the
    kernel's traffic grows in proportion to the pixels it processes)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None, "no ncu capture committed"
    cur = _source_sha(kernel.split(" ")[0])
    scaled = None
    for line in open(path):
        f = line.split()
        if len(f) < 5 or f[0].startswith("#") or f[0] != kernel.split(" ")[0] or f[2] != precision:
            continue
        fresh = len(f) >= 6 and f[5] == cur
        if f[1] == workload:
            if fresh:
                return int(f[3]) + int(f[4]), f"profiles/ncu_traffic.txt, ncu capture of source {cur}"
            return None, "kernel source changed since the committed ncu capture"
        if fresh and len(f) >= 7 and npix and scaled is None:
            b = (int(f[3]) + int(f[4])) * npix / int(f[6])
            scaled = (int(round(b)), f"profiles/ncu_traffic.txt: the {f[1]} capture ({int(f[6])} "
                                     f"pixels per launch, source {cur}) scaled to {npix} pixels")
    if scaled:
        return scaled
    return None, "no ncu capture of this kernel on the current source committed"


def _tc_roofline(peaks, prec, flop, avg_ms, kernel, workload):
    """Tensor-core conv roofline for a kernel timed alone by per-launch CUDA
    events in a short eager pass: the burst peak (FP8: x nominal ratio 2)."""
    achieved = flop / (avg_ms * 1e-3) / 1e12
    pk = peaks["bf16"] * (2 if prec == "fp8" else 1)
    traffic, tnote = ncu_traffic(kernel, workload, prec, npix=int(round(flop / 73728.0)))
    return dict(bound="tensor", achieved=round(achieved, 2), peak=pk, unit="TFLOP/s",
                frac=round(achieved / pk, 4), traffic=traffic, traffic_source=tnote, kernel=kernel,
                flop_per_launch=flop, avg_launch_ms=round(avg_ms, 5),
                peak_kind=f"{prec} burst ({peaks['src']}"
                          + (", bf16 x nominal ratio 2" if prec == "fp8" else "")
                          + "): kernel timed alone by per-launch CUDA events in a short eager pass")


def run_batch(args, P, torch, stream, ws, rank, local):
    """Batched form: 48 independent problems, one tensor-core launch per layer
    over all of them, one CUDA graph per iteration."""
    peaks = load_peaks()
    probs = synth.batched_problems(48, seed=4000 + 17 * rank)
    den = P.Denoiser.from_weights(synth.workload_denoiser(2))
    # timed in the sampling regime (burn-in 0: the Welford accumulation runs)
    jobs = [dict(y=p.y, h=p.h, sigma=p.sigma, seed=p.seed, burn_in=0) for p in probs]
    npix = sum(p.y.size for p in probs)
    out = {}
    for prec in ("bf16", "fp32"):
        steps = args.steps if prec == "bf16" else min(args.steps, 20)
        b = P.Batch(jobs, den, precision=prec, stream=stream.cuda_stream)
        b.step(args.warmup)
        torch.cuda.synchronize()
        rank_barrier(ws)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier(ws)
        ck = sampler.stop()
        rate, slow = replica_rate(npix * steps, e0.elapsed_time(e1) / 1e3, ws)
        out[prec] = dict(ms=slow * 1e3, steps=steps, value=rate, clocks=ck)
        if prec == "bf16":
            kb, kc = _timed_kernels(P, torch, b.step, 10)
            out[prec]["conv_tc_avg_ms"] = kb["conv_tc"] / max(kc["conv_tc"], 1)
            out[prec]["launches_per_iter"] = sum(kc.values()) / 10
            out[prec]["kb"], out[prec]["kc"] = kb, kc
        b.close()
    if rank != 0:
        return
    roof = _tc_roofline(peaks, "bf16", 2.0 * 64 * 64 * 9 * npix, out["bf16"]["conv_tc_avg_ms"],
                        "k_conv_tc<0,0> (48-job table)", "batch48")
    sizes = [p.y.shape[0] for p in probs]
    line = dict(
        metric=METRIC, value=round(out["bf16"]["value"], 3), unit=UNIT, n_gpus=ws,
        steps=args.steps, warmup=args.warmup, ms_per_step=round(out["bf16"]["ms"] / args.steps, 4),
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="bf16", data="synthetic",
        config=dict(workload=f"batch48: 48 problems, sizes log-uniform 256..2048 (min {min(sizes)}, "
                             f"max {max(sizes)}, {npix / 1e6:.1f} Mpixel total), blur mix, BSNR "
                             f"15-40 dB, K=8 F=64 BF16, one launch per layer over all jobs",
                    precision="bf16", graph="one CUDA graph per batch iteration",
                    l2="working set per step > 126 MB L2"),
        roofline=roof,
        fp32_plain=dict(value=round(out["fp32"]["value"], 3), unit=UNIT, steps=out["fp32"]["steps"],
                        speedup_bf16=round(out["bf16"]["value"] / out["fp32"]["value"], 3)),
        gpu_launches=int(round(out["bf16"]["launches_per_iter"])) * args.steps,
        launches_per_iter=out["bf16"]["launches_per_iter"],
        clocks=out["bf16"]["clocks"],
        kernel_breakdown_ms=dict(bf16=out["bf16"]["kb"], launches=out["bf16"]["kc"], iterations=10),
        stencil_roofline=_stencil_roofline(peaks, dict(breakdown=out["bf16"]["kb"],
                                                       counts=out["bf16"]["kc"]), npix, iters=10),
        latency=dict(p50_s=None, p99_s=None, note="batch of 48 jobs stepped together"),
    )
    print(json.dumps(line), flush=True)


def _pow2_side(n):
    return 64 <= n <= 4096 and (n & (n - 1)) == 0


def _stencil_roofline(peaks, kern, npix, poisson=False, wide_h=None, iters=None, spectral=False):
    """Stencils against HBM from the eager per-kernel timing: algorithmic bytes
    per pixel (r = Hx - y: read x, y, write r: 12 B; update while sampling:
    read r, x, d, mean, m2, write x, mean, m2: 32 B, Poisson + z2: 36 B;
    Poisson z-update: read x, z1, z2, y, write z1, z2: 24 B) x the pixels of
    one iteration (npix, all jobs) x iterations / the kernel's total time
    (iters = None: one launch per iteration). Large (wide) kernels add their
    FMA rate against the FP32 FFMA peak. With the spectral gradient the "blur"
    timer holds the row FFTs (read x, write the half spectrum: 4 + 4 B) and
    the column pass (read and write the half spectrum, read |H^|^2: 4 + 4 + 2 B),
    and the "update" timer the inverse row FFTs fused with the update (half
    spectrum 4 B + 32 B)."""
    out = {}
    kinds = ((("blur", 18), ("update", 36)) if spectral else
             (("blur", 12), ("update", 36 if poisson else 32), ("zupdate", 24)))
    for kname, bpp in kinds:
        n = kern["counts"].get(kname, 0)
        if not n:
            continue
        avg = kern["breakdown"][kname] / n
        it = n if iters is None else iters
        gbs = bpp * npix * it / (kern["breakdown"][kname] * 1e-3) / 1e9
        out[kname] = dict(avg_us=round(avg * 1e3, 2), bytes_per_pixel=bpp,
                          achieved_gbs=round(gbs, 1), frac=round(gbs / peaks["hbm"], 4))
        if spectral:
            out[kname]["form"] = "spectral (FFT) gradient"
        elif wide_h is not None and kname != "zupdate":
            nnz = int(np.count_nonzero(wide_h.astype(np.float32)))
            tf = 2.0 * nnz * npix * it / (kern["breakdown"][kname] * 1e-3) / 1e12
            alu = 148 * 128 * 2 * peaks["sm_max"] / 1e6
            out[kname].update(nonzero_taps=nnz, achieved_tflops=round(tf, 2),
                              alu_frac=round(tf / alu, 4), alu_peak_tflops=round(alu, 1))
    if out:
        out["peak_gbs"] = peaks["hbm"]
        out["peak_kind"] = f"HBM copy ({peaks['src']})"
    return out


def _timed_kernels(P, torch, run, n_timed):
    """Per-kernel device time of `n_timed` eager iterations (CUDA events
    around every launch): {name: ms}, {name: launches}."""
    P.pnp_kernel_timer(True)
    run(n_timed)
    torch.cuda.synchronize()
    tot = {k: P.pnp_kernel_timer_read(k) for k in KTIMERS}
    P.pnp_kernel_timer(False)
    return ({k: v[0] for k, v in tot.items()}, {k: v[1] for k, v in tot.items()})


def run_serve(args, P, torch, stream, ws, rank, local):
    """Serving form (the headline): a seeded Poisson stream of sampling jobs
    (20 jobs/s), each 200 burn-in + 800 kept iterations, continuously batched
    by the server; a bounded run of the first K arrivals (K = --steps, at most
    64). The FP32 one-job-at-a-time baseline is modelled from FP32 iteration
    times measured per image size on the same GPU."""
    import threading as th
    peaks = load_peaks()
    n = max(1, min(args.jobs if args.jobs else args.steps, 64))
    specs = synth.serving_jobs(n, seed=5000 + 31 * rank)
    arrivals = synth.poisson_arrivals(n, 20.0, seed=5000 + 31 * rank)
    probs = [synth.make_problem(sp["size"], sp["size"], sp["h"], sp["bsnr"], sp["gt_seed"])
             for sp in specs]
    den = P.Denoiser.from_weights(synth.workload_denoiser(2))
    T, TB = 1000, 200
    # warm-up: every distinct (size, blur size) runs W iterations once, so the
    # per-size one-time work (stencil tile timing, lazy kernel setup) is done
    warm = {}
    for p in probs:
        warm.setdefault((p.y.shape, p.h.shape), p)
    for p in warm.values():
        gw = P.Problem(p.y, p.h, p.sigma, den, seed=p.seed, precision="bf16",
                       stream=stream.cuda_stream)
        gw.step(args.warmup)
        gw.sync()
        gw.close()
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    srv = P.Server(den, precision="bf16", hbm_budget_bytes=int(0.8 * free), round_iters=8)
    ids = [None] * n
    t_start = 0.0

    def submitter():
        for k in range(n):
            dt = arrivals[k] - (time.perf_counter() - t_start)
            if dt > 0:
                time.sleep(dt)
            p = probs[k]
            ids[k] = srv.submit(p.y, p.h, p.sigma, T, TB, seed=p.seed)

    rank_barrier(ws)
    launches0 = P.pnp_launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    t_start = time.perf_counter()
    thr = th.Thread(target=submitter)
    thr.start()
    thr.join()
    for jid in ids:
        srv.wait(jid, 3600)
    t_end = time.perf_counter()
    ck = sampler.stop()
    launches = P.pnp_launch_count() - launches0
    dev_s = srv.device_seconds()
    times = [srv.times(j) for j in ids]
    lat = [t["done"] - t["submit"] for t in times]
    span = max(t["done"] for t in times) - min(t["submit"] for t in times)
    pix_iters = sum(p.y.size for p in probs) * T
    value, _ = replica_rate(pix_iters, dev_s, ws)
    e2e_value, _ = replica_rate(pix_iters, span, ws)
    # quality at equal PSNR on the smallest job: BF16 served vs its FP32 plain chain
    kq = min(range(n), key=lambda k: probs[k].y.size)
    q = probs[kq]
    _, mm16, _ = srv.poll(ids[kq])
    srv.close()
    g32 = P.Problem(q.y, q.h, q.sigma, den, seed=q.seed, burn_in=TB, precision="fp32",
                    stream=stream.cuda_stream)
    g32.run_chain(T, TB)
    mm32, _, _ = g32.moments()
    g32.close()
    psnr = lambda m: 10 * math.log10(1.0 / float(np.mean((m - q.xbar) ** 2)))
    # roofline: the tensor-core conv over a table of the stream's jobs (one
    # launch per layer over all of them, as in the server's rounds), timed alone
    sub = probs[:min(n, 8)]
    b = P.Batch([dict(y=p.y, h=p.h, sigma=p.sigma, seed=p.seed, burn_in=0) for p in sub], den,
                precision="bf16", stream=stream.cuda_stream)
    b.step(3)
    kb, kc = _timed_kernels(P, torch, b.step, 10)
    b.close()
    npix_b = sum(p.y.size for p in sub)
    roof = _tc_roofline(peaks, "bf16", 2.0 * 64 * 64 * 9 * npix_b, kb["conv_tc"] / max(kc["conv_tc"], 1),
                        "k_conv_tc<0,0>", "serve")
    roof["units_per_launch"] = f"{npix_b} pixels of {len(sub)} served jobs x 73728 FLOP"
    # FP32 one-job-at-a-time: measured per-size iteration time, FIFO over the same arrivals
    per_size = {}
    for p in probs:
        key = (p.y.shape[0], p.h.shape)
        if key not in per_size:
            per_size[key] = _fp32_iter_time(P, torch, den, p, stream, iters=50)
    finish, lat32 = 0.0, []
    for k, p in enumerate(probs):
        start = max(arrivals[k], finish)
        finish = start + T * per_size[(p.y.shape[0], p.h.shape)]
        lat32.append(finish - arrivals[k])
    value32 = pix_iters / (finish - arrivals[0]) / 1e6
    if rank != 0:
        return None
    sizes = [p.y.shape[0] for p in probs]
    h2d = sum(p.y.size * 4 + p.h.size * 4 for p in probs)
    d2h = sum(2 * p.y.size * 8 for p in probs)
    line = dict(
        metric=METRIC, value=round(value, 3), unit=UNIT, n_gpus=ws, steps=n, warmup=args.warmup,
        ms_per_step=round(1e3 * span / n, 3), higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="bf16", data="synthetic",
        config=dict(workload=f"serve: the first {n} jobs of a seeded Poisson stream at 20 jobs/s, "
                             f"sizes {sorted(set(sizes))} (uniform over 512..4096 squared), blur and "
                             "BSNR drawn as in the batched workload, 200 burn-in + 800 kept "
                             "iterations, MMSE + std maps; K=8 F=64 DnCNN-form denoiser in BF16; "
                             "continuous batching with HBM-budget admission",
                    step="one job of the stream (1000 iterations)",
                    value="stream pixel-iterations / server device time (CUDA events around every "
                          "round's launches)",
                    precision="bf16", l2="working set per round > 126 MB L2"),
        roofline=roof,
        e2e=dict(value=round(e2e_value, 3), unit=UNIT, h2d_bytes_per_step=h2d / n,
                 d2h_bytes_per_step=d2h / n,
                 note="wall time from the first submission to the last completion: host y and h "
                      "copied in at admission, FP64 MMSE and std maps copied out at retirement"),
        latency=dict(p50_s=round(_percentile(lat, 50), 3), p99_s=round(_percentile(lat, 99), 3),
                     unit="s", definition="completion - submission", jobs=n),
        fp32_plain=dict(value=round(value32, 3), unit=UNIT,
                        p50_s=round(_percentile(lat32, 50), 3), p99_s=round(_percentile(lat32, 99), 3),
                        kind="modelled",
                        note="one job at a time, FIFO over the same arrivals; FP32 plain iteration "
                             "time measured on this GPU per image and blur size (50 iterations, "
                             "graph replay) times T = 1000",
                        per_size_ms={f"{k[0]}x{k[0]} h{k[1][0]}": round(1e3 * v, 4)
                                     for k, v in per_size.items()}),
        speedup_bf16=round(value / value32, 3),
        e2e_speedup_bf16=round(e2e_value / value32, 3),
        quality=dict(job=f"{q.y.shape[0]}x{q.y.shape[1]}", psnr_bf16_served_db=round(psnr(mm16), 4),
                     psnr_fp32_plain_db=round(psnr(mm32), 4),
                     delta_db=round(psnr(mm16) - psnr(mm32), 4)),
        gpu_launches=int(launches),
        clocks=ck,
        kernel_breakdown_ms=dict(batch_pass=kb, launches=kc, iterations=10, jobs=len(sub)),
        stencil_roofline=_stencil_roofline(peaks, dict(breakdown=kb, counts=kc), npix_b, iters=10),
        server=dict(device_s=round(dev_s, 3), wall_s=round(span, 3), timed_region_s=round(t_end - t_start, 3)),
    )
    return line


def measure_single(args, P, torch, stream, ws, rank, local, workload, precs, steps, warmup,
                   quality=True, cpu_baseline=True):
    """One workload's single-job line: device-timed graph replay (value), the
    same K iterations end to end through the public API with host buffers
    (e2e), per-kernel eager timing (roofline, stencils), MMSE PSNR per
    precision and the FP64 oracle on the host cores. Returns the line (rank 0)
    or None."""
    cfg_id = WORKLOADS[workload]
    w = synth.WORKLOADS[cfg_id]
    poisson = workload == "poisson1024"
    inpaint = workload == "inpaint1024"
    ddfb = workload == "ddfb1024"
    prob = (poisson_problem(rank) if poisson else inpainting_problem(rank) if inpaint
            else synth.workload_problem(cfg_id, job=rank))
    if getattr(args, "size", 0) and not (poisson or inpaint):
        # the same posterior (blur, BSNR, denoiser) on an n x n image: profiling runs
        n = args.size
        prob = synth.make_problem(n, n, synth.blur_from_spec(w["blur"]), w["bsnr"],
                                  synth.gt_seed(cfg_id, rank), name=f"{w['name']}@{n}",
                                  blocks=w["blocks"], halo=w["halo"], T=w["T"], burn_in=w["burn_in"])
    dw = synth.workload_denoiser(cfg_id)
    if ddfb:
        dd = ddfb_net()
        den = P.Denoiser.ddfb(dd.filters, dd.gammas, dd.ht)
    else:
        den = P.Denoiser.from_weights(dw)
    ny, nx = prob.shape
    npix = ny * nx
    peaks = load_peaks()
    precs = list(precs)
    if w["F"] != 64 or ddfb:
        precs = ["fp32"]

    def make_problem(prec, burn_in):
        kw = dict(blocks=w["blocks"], halo=0, seed=prob.seed, burn_in=burn_in, precision=prec,
                  stream=stream.cuda_stream)
        if poisson:
            return P.Problem(prob.y, prob.h, 0.0, den, noise_model="poisson", eta=prob.eta,
                             rho1=POISSON["rho1"], rho2=POISSON["rho2"], **kw)
        if inpaint:
            return P.Problem(prob.y, None, prob.sigma, den, mask=prob.mask, x0=prob.x0, **kw)
        return P.Problem(prob.y, prob.h, prob.sigma, den, **kw)

    results = {}
    clocks = None
    for prec in precs:
        # the timed iterations sample (burn-in 0): the Welford accumulation runs,
        # as in 80 % of a chain's iterations, and the stencil moves 32 B/pixel
        gp = make_problem(prec, 0)
        st = steps if prec == precs[0] else min(steps, 200)
        gp.step(warmup)
        gp.prepare_graphs()
        torch.cuda.synchronize()
        rank_barrier(ws)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gp.step(st)
        e1.record(stream)
        torch.cuda.synchronize()
        rank_barrier(ws)
        ck = sampler.stop()
        rate, slow = replica_rate(npix * st, e0.elapsed_time(e1) / 1e3, ws)
        results[prec] = dict(ms=slow * 1e3, steps=st, value=rate)
        if prec == precs[0]:
            clocks = ck
        # per-kernel timing: the same iterations launched eagerly with CUDA events
        n_timed = max(5, min(steps, 20))
        kb, kc = _timed_kernels(P, torch, gp.step, n_timed)
        name = "conv_fp32" if prec == "fp32" else "conv_tc"
        results[prec]["kernel"] = dict(name=name, avg_ms=kb[name] / max(kc[name], 1),
                                       launches=kc[name], breakdown=kb, counts=kc,
                                       launches_per_iter=sum(kc.values()) / n_timed)
        gp.close()

    # end-to-end through the public API with host buffers: create (H2D of y, h),
    # run K iterations, read MMSE + std back (D2H)
    prec0 = precs[0]
    torch.cuda.synchronize()
    rank_barrier(ws)
    t0 = time.perf_counter()
    gp = make_problem(prec0, 0)
    gp.run_chain(steps, 0)
    mm, sd, _ = gp.moments()
    e2e_rate, _ = replica_rate(npix * steps, time.perf_counter() - t0, ws)
    gp.close()
    e2e = dict(value=e2e_rate, unit=UNIT,
               h2d_bytes_per_step=(prob.y.size * 4 + (prob.mask.size * 4 + prob.x0.size * 4 if inpaint
                                                       else prob.h.size * 4)) / steps,
               d2h_bytes_per_step=2 * npix * 8 / steps)

    # quality at equal PSNR: the full chain of the workload for each precision
    qual = None
    if quality and rank == 0 and cfg_id in (1, 2):
        qual = {}
        for prec in precs:
            gq = make_problem(prec, w["burn_in"])
            gq.run_chain(w["T"], w["burn_in"])
            mq, _, _ = gq.moments()
            qual[f"psnr_{prec}_db"] = round(10 * math.log10(1.0 / float(np.mean((mq - prob.xbar) ** 2))), 4)
            gq.close()
        if "bf16" in precs and "fp32" in precs:
            qual["delta_db"] = round(qual["psnr_bf16_db"] - qual["psnr_fp32_db"], 4)
        if "fp8" in precs and "fp32" in precs:
            qual["delta_fp8_db"] = round(qual["psnr_fp8_db"] - qual["psnr_fp32_db"], 4)
        qual["chain"] = f"{w['T']} iterations, {w['burn_in']} burn-in"
    if rank != 0:
        return None

    head = results[precs[0]]
    kern = head["kernel"]
    K, F = w["K"], w["F"]
    if kern["name"] == "conv_tc":
        ktag = "k_conv_tc<0,1>" if precs[0] == "fp8" else "k_conv_tc<0,0>"
        roof = _tc_roofline(peaks, precs[0], 2.0 * F * F * 9 * npix, kern["avg_ms"], ktag, workload)
    elif ddfb:
        # a dual layer (the conv_fp32 timer; the first layer and the output run
        # under conv_edge) streams the P-channel dual variable: read v and u, write u
        bpp = 4 + 8 * 64
        gbs = bpp * npix / (kern["avg_ms"] * 1e-3) / 1e9
        traffic, tnote = ncu_traffic("k_ddfb<64,0>", workload, "fp32")
        roof = dict(bound="hbm", achieved=round(gbs, 1), peak=peaks["hbm"], unit="GB/s",
                    frac=round(gbs / peaks["hbm"], 4), traffic=traffic, traffic_source=tnote,
                    kernel="k_ddfb<64,0>", bytes_per_pixel=bpp, peak_kind=f"HBM copy ({peaks['src']})")
    else:
        flop = 2.0 * F * F * 9 * npix
        achieved = flop / (kern["avg_ms"] * 1e-3) / 1e12
        alu_peak = 148 * 128 * 2 * peaks["sm_max"] / 1e6
        roof = dict(bound="alu", achieved=round(achieved, 2), peak=round(alu_peak, 2),
                    unit="TFLOP/s", frac=round(achieved / alu_peak, 4), traffic=None,
                    kernel="k_conv3x3<64,64>", peak_kind="FP32 FFMA: 148 SM x 128 lanes x 2 x max clock")
    wide = prob.h if (not poisson and not inpaint and max(prob.h.shape) > 31) else None
    spectral = (wide is not None and not args.no_spectral and _pow2_side(prob.y.shape[0]) and
                _pow2_side(prob.y.shape[1]))
    stencils = _stencil_roofline(peaks, kern, npix, poisson=poisson, wide_h=wide, spectral=spectral)
    cpu = None
    if cpu_baseline:
        try:
            cpu = oracle_baseline(cfg_id, budget_s=15.0, poisson=poisson, inpaint=inpaint, ddfb=ddfb)
        except Exception as ex:  # report, never fake
            cpu = dict(value=None, unit=UNIT, cores=None, kind="oracle", sample=f"failed: {ex}")
    if poisson:
        wl = (f"poisson1024: {ny}x{nx} Poisson counts, peak eta={prob.eta:g}, rho1={POISSON['rho1']:g}, "
              f"rho2={POISSON['rho2']:g}, AXDA + PSGLA, blur {w['blur'][0]} {w['blur'][1]}x{w['blur'][1]}, ")
    elif inpaint:
        wl = (f"inpaint1024: {ny}x{nx} grayscale, 30 % of the pixels observed, 15 dB input SNR, "
              "cubic-interpolant start, ")
    elif ddfb:
        wl = (f"ddfb1024: {ny}x{nx} grayscale, {w['bsnr']} dB BSNR, DDFB prior K=4 P=64 (FP32), "
              f"blur {w['blur'][0]} {w['blur'][1]}x{w['blur'][1]}, ")
    else:
        wl = (f"{w['name']}{' resized' if getattr(args, 'size', 0) else ''}: {ny}x{nx} grayscale, "
              f"{w['bsnr']} dB BSNR, blur {w['blur'][0]} {w['blur'][1]}x{w['blur'][1]}, ")
    wl += ("" if ddfb else f"DnCNN-form K={K} F={F}, ") + \
        f"{w['blocks'][0]}x{w['blocks'][1]} blocks (halo-exchange-free), 1 chain per GPU"
    line = dict(
        metric=METRIC, value=round(head["value"], 3), unit=UNIT, n_gpus=ws, steps=steps,
        warmup=warmup, ms_per_step=round(head["ms"] / steps, 4), higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype=("bf16" if precs[0] == "bf16" else
                                                 "fp8" if precs[0] == "fp8" else "f32"),
        data="synthetic",
        config=dict(workload=wl, precision=precs[0],
                    l2="working set per step > 126 MB L2 (activation planes)",
                    graph="one CUDA graph per iteration",
                    stencil_tile=("forced %d" % args.stencil_tile if args.stencil_tile >= 0
                                  else "autotuned"),
                    wide_gradient=(None if wide is None else
                                   "spectral (FFT)" if spectral else "direct wide stencil")),
        roofline=roof,
        cpu_baseline=cpu,
        e2e=e2e,
        gpu_launches=int(round(kern["launches_per_iter"])) * steps,
        clocks=clocks,
        kernel_breakdown_ms={p: results[p]["kernel"]["breakdown"] for p in results},
        stencil_roofline=stencils,
    )
    if "fp32" in results and precs[0] != "fp32":
        line["fp32_plain"] = dict(value=round(results["fp32"]["value"], 3), unit=UNIT,
                                  ms_per_step=round(results["fp32"]["ms"] / results["fp32"]["steps"], 4),
                                  steps=results["fp32"]["steps"],
                                  speedup_bf16=round(head["value"] / results["fp32"]["value"], 3))
    if "fp8" in results and precs[0] != "fp8":
        r8 = results["fp8"]
        r8roof = _tc_roofline(peaks, "fp8", 2.0 * F * F * 9 * npix, r8["kernel"]["avg_ms"],
                              "k_conv_tc<0,1>", workload)
        line["fp8_variant"] = dict(
            value=round(r8["value"], 3), unit=UNIT, ms_per_step=round(r8["ms"] / r8["steps"], 4),
            steps=r8["steps"], speedup_vs_bf16=round(r8["value"] / head["value"], 3),
            conv_tc_tflops=r8roof["achieved"], conv_tc_frac=r8roof["frac"],
            peak_kind=r8roof["peak_kind"],
            note="E4M3 weights (per-output-channel scales) and activations (per-layer static scales)")
    if qual:
        line["quality"] = qual
    line["latency"] = dict(p50_s=None, p99_s=None, note="single-job workload")
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="serve", choices=sorted(WORKLOADS))
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-nested", action="store_true",
                    help="serve: skip the nested single-job deconv1024 / deconv8192 lines")
    ap.add_argument("--precisions", default="bf16,fp32,fp8")
    ap.add_argument("--jobs", type=int, default=0, help="serve: number of arrivals (default: --steps)")
    ap.add_argument("--size", type=int, default=0,
                    help="single-job Gaussian workloads: the same posterior on a size x size image")
    ap.add_argument("--no-spectral", action="store_true",
                    help="wide blurs: the direct stencil instead of the spectral (FFT) gradient")
    ap.add_argument("--stencil-tile", type=int, default=-1,
                    help="force stencil tile shape k for every launch (profiling; default: autotuned)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2511_00870_b300 as P
    from paper_2511_00870_b300 import build
    if rank == 0 and build.needs_build():
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    if args.stencil_tile >= 0:
        P.pnp_set_stencil_tile(args.stencil_tile)
    if args.no_spectral:
        P.pnp_set_spectral(False)
    # a dedicated stream: the problems enqueue on it and the events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    if args.workload == "batch48":
        run_batch(args, P, torch, stream, ws, rank, local)
    elif args.workload == "serve":
        line = run_serve(args, P, torch, stream, ws, rank, local)
        cpu = None
        if rank == 0 and not args.no_cpu_baseline:
            try:
                cpu = oracle_baseline(5, budget_s=15.0)
            except Exception as ex:  # report, never fake
                cpu = dict(value=None, unit=UNIT, cores=None, kind="oracle", sample=f"failed: {ex}")
        nested = {}
        if not args.no_nested:
            for wl, precs, q in (("deconv1024", ("bf16", "fp32", "fp8"), not args.no_quality),
                                 ("deconv8192", ("bf16",), False)):
                nested[wl] = measure_single(args, P, torch, stream, ws, rank, local, wl, precs,
                                            args.steps, args.warmup, quality=q, cpu_baseline=False)
        if rank == 0:
            line["cpu_baseline"] = cpu
            for wl, sub in nested.items():
                line[f"single_job_{wl}"] = {k: sub[k] for k in (
                    "value", "unit", "ms_per_step", "steps", "dtype", "config", "roofline", "e2e",
                    "gpu_launches", "clocks", "kernel_breakdown_ms", "stencil_roofline",
                    "fp32_plain", "fp8_variant", "quality") if k in sub}
            print(json.dumps(line), flush=True)
    else:
        line = measure_single(args, P, torch, stream, ws, rank, local, args.workload,
                              [p for p in args.precisions.split(",") if p], args.steps,
                              args.warmup, quality=not args.no_quality,
                              cpu_baseline=not args.no_cpu_baseline)
        if rank == 0:
            print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
