#!/usr/bin/env python3
"""Throughput benchmark of the PnP-ULA Gaussian-deconvolution sampler on B300.

A step is one full x-update of the chain (Eq. 8 / Algorithm 1 x-part): blur
residual, block-wise DnCNN-form denoiser, fused Langevin update with Philox
noise and Welford moments. Metric: Mpixel-iterations/s = pixels x iterations /
time. Default workload: 1024 x 1024 Gaussian deconvolution, 9 x 9 uniform
blur, 20 dB BSNR, 8-layer 64-channel seeded denoiser, 4 x 4 blocks; the
headline value is the BF16 denoiser form, with the FP32 plain form and the
MMSE PSNR of both reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload deconv1024|deconv8192|deconv128] [--no-quality]
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
}


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


def _oracle_setup(cfg_id, crop):
    import oracle
    prob = synth.workload_problem(cfg_id)
    dw = synth.workload_denoiser(cfg_id)
    crop = min(crop, prob.shape[0], prob.shape[1])
    y = prob.y[:crop, :crop]
    lam, gam = oracle.stepsizes(float(np.abs(prob.h).sum()), prob.sigma, 1.0, prob.sigma,
                                dw.lipschitz)
    op = oracle.Problem(y, prob.h, prob.sigma, 1.0, prob.sigma, lam, gam, prob.seed,
                        net=oracle.Net.from_weights(dw))
    return oracle, prob, op, crop


def oracle_baseline(cfg_id, budget_s=20.0, crop=128):
    """The FP64 oracle as it stands, on a bounded sample of the workload:
    whole iterations on a crop of the image (same blur, noise level and
    network), on this host's cores."""
    oracle, prob, op, crop = _oracle_setup(cfg_id, crop)
    ny, nx = prob.shape
    x = np.zeros((crop, crop))
    t0 = time.perf_counter()
    it = 0
    while True:
        x = oracle.langevin_step(op, x, it)
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
    w = synth.WORKLOADS[cfg_id]
    steps = max(1, args.steps)
    n = args.warmup + steps
    crop = 128 if n <= 60 else (64 if n <= 250 else 32)
    oracle, prob, op, crop = _oracle_setup(cfg_id, crop)
    x = np.zeros((crop, crop))
    for it in range(args.warmup):
        x = oracle.langevin_step(op, x, it)
    t0 = time.perf_counter()
    for it in range(args.warmup, n):
        x = oracle.langevin_step(op, x, it)
    dt = time.perf_counter() - t0
    val = crop * crop * steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"each step one FP64 oracle iteration on a {crop}x{crop} crop of the "
              f"{prob.shape[0]}x{prob.shape[1]} workload (same blur, noise, network)")
    line = dict(metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus, steps=steps,
                warmup=args.warmup, ms_per_step=1e3 * dt / steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=f"{w['name']} (oracle, bounded crop sample)"),
                cpu_baseline=dict(kind="oracle", cores=cores, sample=sample, value=val, unit=UNIT),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="deconv1024", choices=sorted(WORKLOADS))
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precisions", default="bf16,fp32")
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

    cfg_id = WORKLOADS[args.workload]
    w = synth.WORKLOADS[cfg_id]
    prob = synth.workload_problem(cfg_id, job=rank)
    dw = synth.workload_denoiser(cfg_id)
    den = P.Denoiser.from_weights(dw)
    ny, nx = prob.shape
    npix = ny * nx
    # a dedicated stream: the problems enqueue on it and the events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    peaks = load_peaks()
    precs = [p for p in args.precisions.split(",") if p]
    if w["F"] != 64:
        precs = ["fp32"]

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        if ws == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return t.item()

    results = {}
    clocks = None
    for prec in precs:
        gp = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=w["blocks"], halo=0,
                       seed=prob.seed, burn_in=w["burn_in"], precision=prec,
                       stream=stream.cuda_stream)
        steps = args.steps if prec == precs[0] else min(args.steps, 200)
        gp.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gp.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck = sampler.stop()
        ms = e0.elapsed_time(e1)
        ms_max = max_over_ranks(ms)
        results[prec] = dict(ms=ms_max, steps=steps, value=ws * npix * steps / (ms_max * 1e3))
        if prec == precs[0]:
            clocks = ck
        # dominant-kernel timing: same iterations launched eagerly with CUDA events
        P.pnp_kernel_timer(True)
        gp.step(max(5, min(args.steps, 20)))
        torch.cuda.synchronize()
        name = "conv_tc" if prec == "bf16" else "conv_fp32"
        kms, kn = P.pnp_kernel_timer_read(name)
        tot = {k: P.pnp_kernel_timer_read(k) for k in ("blur", "update", "conv_fp32", "conv_tc",
                                                        "conv_edge")}
        P.pnp_kernel_timer(False)
        results[prec]["kernel"] = dict(name=name, avg_ms=kms / max(kn, 1), launches=kn,
                                       breakdown={k: v[0] for k, v in tot.items()})
        gp.close()

    # end-to-end through the public API with host buffers: create (H2D of y, h),
    # run K iterations, read MMSE + std back (D2H)
    prec0 = precs[0]
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    gp = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=w["blocks"], halo=0, seed=prob.seed,
                   burn_in=0, precision=prec0, stream=stream.cuda_stream)
    gp.run_chain(args.steps, 0)
    mm, sd, _ = gp.moments()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    gp.close()
    e2e = dict(value=ws * npix * args.steps / t_e2e / 1e6, unit=UNIT,
               h2d_bytes_per_step=(prob.y.size * 4 + prob.h.size * 4) / args.steps,
               d2h_bytes_per_step=2 * npix * 8 / args.steps)

    # quality at equal PSNR: the full chain of the workload for each precision
    quality = None
    if not args.no_quality and rank == 0 and cfg_id != 3:
        quality = {}
        for prec in precs:
            gq = P.Problem(prob.y, prob.h, prob.sigma, den, blocks=w["blocks"], halo=0,
                           seed=prob.seed, burn_in=w["burn_in"], precision=prec,
                           stream=stream.cuda_stream)
            gq.run_chain(w["T"], w["burn_in"])
            mq, _, _ = gq.moments()
            quality[f"psnr_{prec}_db"] = round(10 * math.log10(1.0 / float(np.mean((mq - prob.xbar) ** 2))), 4)
            gq.close()
        if "bf16" in precs and "fp32" in precs:
            quality["delta_db"] = round(quality["psnr_bf16_db"] - quality["psnr_fp32_db"], 4)
        quality["chain"] = f"{w['T']} iterations, {w['burn_in']} burn-in"

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    head = results[precs[0]]
    kern = head["kernel"]
    K, F = w["K"], w["F"]
    pix_per_launch = npix  # one image per replica
    if kern["name"] == "conv_tc":
        flop = 2.0 * F * F * 9 * pix_per_launch
        achieved = flop / (kern["avg_ms"] * 1e-3) / 1e12
        roof = dict(bound="tensor", achieved=round(achieved, 2),
                    peak=peaks["bf16_sus"], unit="TFLOP/s",
                    frac=round(achieved / peaks["bf16_sus"], 4), traffic=None,
                    kernel="k_conv_tc", peak_kind=f"bf16 sustained ({peaks['src']})")
    else:
        flop = 2.0 * F * F * 9 * pix_per_launch
        achieved = flop / (kern["avg_ms"] * 1e-3) / 1e12
        alu_peak = 148 * 128 * 2 * peaks["sm_max"] / 1e6
        roof = dict(bound="alu", achieved=round(achieved, 2), peak=round(alu_peak, 2),
                    unit="TFLOP/s", frac=round(achieved / alu_peak, 4), traffic=None,
                    kernel="k_conv3x3<64,64>", peak_kind="FP32 FFMA: 148 SM x 128 lanes x 2 x max clock")
    launches_per_step = (K + 3) if precs[0] == "bf16" else (K + 3)
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = oracle_baseline(cfg_id, budget_s=15.0)
        except Exception as ex:  # report, never fake
            cpu = dict(value=None, unit=UNIT, cores=None, kind="oracle", sample=f"failed: {ex}")
    line = dict(
        metric=METRIC, value=round(head["value"], 3), unit=UNIT, n_gpus=ws, steps=args.steps,
        warmup=args.warmup, ms_per_step=round(head["ms"] / args.steps, 4), higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype=("bf16" if precs[0] == "bf16" else "f32"),
        data="synthetic",
        config=dict(workload=f"{w['name']}: {ny}x{nx} grayscale, blur {w['blur'][0]} "
                             f"{w['blur'][1]}x{w['blur'][1]}, {w['bsnr']} dB BSNR, DnCNN-form "
                             f"K={K} F={F}, {w['blocks'][0]}x{w['blocks'][1]} blocks "
                             f"(halo-exchange-free), 1 chain per GPU",
                    precision=precs[0], l2="working set per step > 126 MB L2 (activation planes)",
                    graph="one CUDA graph per iteration"),
        roofline=roof,
        cpu_baseline=cpu,
        e2e=e2e,
        gpu_launches=launches_per_step * args.steps,
        clocks=clocks,
        kernel_breakdown_ms={p: results[p]["kernel"]["breakdown"] for p in results},
    )
    if "fp32" in results and precs[0] != "fp32":
        line["fp32_plain"] = dict(value=round(results["fp32"]["value"], 3), unit=UNIT,
                                  ms_per_step=round(results["fp32"]["ms"] / results["fp32"]["steps"], 4),
                                  steps=results["fp32"]["steps"],
                                  speedup_bf16=round(head["value"] / results["fp32"]["value"], 3))
    if quality:
        line["quality"] = quality
    line["latency"] = dict(p50_s=None, p99_s=None, note="single-job workload; see --workload serve")
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
