#!/usr/bin/env python
"""Throughput of the SFFT fit + subtraction on GB300: 4088 x 4088 difference images per second.

One step = fit + subtract for every pair in this rank's batch of seeded synthetic Roman-like
4088^2 float32 pairs (~3000 Moffat stars per frame, FWHM 1.8 -> 2.4 px across the frame,
Poisson sky 80 e- subtracted, 0.5% + 0.5% masked pixels; 11 x 11 delta kernel, DK=2, DB=2,
732 unknowns).  Inputs are resident in HBM before the timed region; each pair's frames
(150 MB) plus the plan's spectra (1.5 GB) exceed the 129 MB L2, so no flush is needed.

Under torchrun every rank processes its own pairs (weak scaling, no data-path collective);
rank 0 prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same workload, scaled to the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "4088² difference images/s on 1 GB300 (batched+learned vs plain), HBM roofline %"
UNIT = "difference images/s"
NY = NX = 4088
L, DK, DB = 11, 2, 2
WORKLOAD = "Roman-like 4088x4088 float32 pair, L=11, DK=2, DB=2 (732 unknowns), masked"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=4, help="pairs per step per rank")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solver", default="cholesky", choices=["cholesky", "pcg"])
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_18544_gb300 import build as sfft_build
    from paper_2509_18544_gb300 import sfft, synth

    sfft_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    pairs = []
    for i in range(args.pairs):
        S, T, M = synth.roman_pair(NY, NX, seed=1000 + 100 * rank + i)
        pairs.append((S, T, M))
    dev_pairs = [tuple(torch.from_numpy(a).to(dev) for a in p) for p in pairs]
    stream = torch.cuda.current_stream(dev)
    solver = sfft.SOLVE_PCG if args.solver == "pcg" else sfft.SOLVE_CHOLESKY
    plan = sfft.sfft_plan(sfft.make_desc(NY, NX, L, DK, DB, solver=solver), stream=stream)
    n = plan.n
    coeffs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in pairs]
    diffs = [torch.empty((NY, NX), dtype=torch.float32, device=dev) for _ in pairs]

    def step():
        for (S, T, M), th, D in zip(dev_pairs, coeffs, diffs):
            sfft.sfft_fit(plan, S, T, M, None, th, want_info=False)
            sfft.sfft_subtract(plan, S, T, th, D)

    def barrier():
        if world > 1:
            dist.barrier()

    # first call reported separately (cold), then warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(max(args.warmup - 1, 0)):
        step()
    info = sfft.sfft_fit(plan, *dev_pairs[0], None, coeffs[0], want_info=True)
    torch.cuda.synchronize()

    # ---- timed region (device events on the launching stream)
    sfft.sfft_stage_times(plan)  # reset accumulators
    sfft.sfft_profile(plan, True)
    clocks = ClockSampler(local)
    launches0 = sfft.sfft_launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = sfft.sfft_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    stages, calls = sfft.sfft_stage_times(plan)
    sfft.sfft_profile(plan, False)
    ms_max = ms
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    total_pairs = args.steps * args.pairs * world
    value = total_pairs / (ms_max / 1e3)

    # ---- end to end through the public API with pinned host buffers
    host = [tuple(torch.from_numpy(a).pin_memory() for a in p) for p in pairs]
    host_D = [torch.empty((NY, NX), dtype=torch.float32).pin_memory() for _ in pairs]
    host_th = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in pairs]
    dbuf = [tuple(torch.empty_like(t) for t in p) for p in dev_pairs]

    def e2e_step():
        for (hS, hT, hM), (dS, dT, dM), th, D, oD, oth in zip(host, dbuf, coeffs, diffs, host_D, host_th):
            dS.copy_(hS, non_blocking=True)
            dT.copy_(hT, non_blocking=True)
            dM.copy_(hM, non_blocking=True)
            sfft.sfft_fit(plan, dS, dT, dM, None, th, want_info=False)
            sfft.sfft_subtract(plan, dS, dT, th, D)
            oD.copy_(D, non_blocking=True)
            oth.copy_(th, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(2, args.steps // 2)
    f0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    if world > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = e2e_steps * args.pairs * world / (e2e_ms / 1e3)
    h2d = args.pairs * sum(t.numel() * t.element_size() for t in host[0])
    d2h = args.pairs * (host_D[0].numel() * 4 + n * 8)

    # ---- roofline of the dominant kernel (y-direction lag correlation, ALU bound)
    g_nseg = -(-NX // (256 - 2 * (L - 1)))
    nk, nb = (DK + 1) * (DK + 2) // 2, (DB + 1) * (DB + 2) // 2
    nent = nk * (nk + 1) // 2 * (2 * L - 1) + nk * (nb + 1) * L
    flops_per_launch = g_nseg * 129 * NY * nent * 8.0  # one complex multiply-add = 8 flops
    ycorr_ms_per_launch = stages["ycorr"] / max(calls, 1)
    achieved_tflops = flops_per_launch / (ycorr_ms_per_launch * 1e-3) / 1e12
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s: SMs x FP32 lanes x (mul+add) x clock
    roofline = {"bound": "alu", "kernel": "k_ycorr_f32 (y-direction lag correlation)",
                "achieved": round(achieved_tflops, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved_tflops / fp32_peak, 4), "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (MEASURED_PEAKS sm_max_mhz)" % sm_max,
                "flops_per_launch": flops_per_launch, "ms_per_launch": round(ycorr_ms_per_launch, 4)}
    seg_bytes = NY * NX * 9.0 + g_nseg * NY * 129 * 20 * 8.0  # read S,T,mask; write 20 spectra
    seg_ms = stages["segment_fft"] / max(calls, 1)
    hbm = peaks.get("hbm_gbs", 6785.5)
    stage_ms = {k: round(v / max(calls, 1), 4) for k, v in stages.items()}

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frame": "%dx%d" % (NY, NX), "L": L, "dk": DK, "db": DB,
                   "pairs_per_step_per_rank": args.pairs,
                   "mode": "plain (FP32 spectra, FP64 Cholesky)" if args.solver == "cholesky"
                   else "FP32 spectra, cluster PCG (FP32 Cholesky preconditioner, FP64 residuals)",
                   "l2": "inputs larger than L2 (150 MB frames + 1.5 GB spectra per pair); no flush",
                   "parallelism": "replicas: independent pairs per GPU" if world > 1 else "1 GPU"},
        "roofline": roofline,
        "segment_fft_hbm": {"bound": "hbm", "achieved": round(seg_bytes / (seg_ms * 1e-3) / 1e9, 1),
                            "peak": hbm, "unit": "GB/s", "frac": round(seg_bytes / (seg_ms * 1e-3) / 1e9 / hbm, 4)},
        "stages_ms_per_pair": stage_ms,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
        "first_call_ms": round(first_ms, 1),
        "fit_rel_residual": info.rel_residual,
    }
    if world > 1:
        dist.barrier()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(result), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- oracle arm
def oracle_sample(size: int, seed: int):
    """FP64 oracle fit + subtraction of one size x size pair drawn like the workload; returns
    seconds, scaled to one 4088^2 pair by pixel count (the oracle's work is linear in pixels)."""
    import oracle
    from paper_2509_18544_gb300 import synth

    S, T, M = synth.roman_pair(size, size, seed=seed)
    t0 = time.perf_counter()
    th = oracle.fit(S, T, M, L, DK, DB)
    oracle.subtract(S, T, th, L, DK, DB)
    dt = time.perf_counter() - t0
    return dt, dt * (NY * NX) / float(size * size)


def cpu_baseline(size: int = 2048):
    import oracle
    oracle.build()
    dt, per_pair = oracle_sample(size, seed=77)
    return {"value": round(1.0 / per_pair, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "one %dx%d pair of the same star/PSF/noise/mask model, L=11 DK=2 DB=2, fit + subtract in "
                      "%.1f s, scaled to 4088^2 by pixel count" % (size, size, dt)}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    size = 512
    for i in range(args.warmup):
        oracle_sample(size, seed=500 + i)
    total = 0.0
    for i in range(args.steps):
        _, per_pair = oracle_sample(size, seed=600 + i)
        total += per_pair
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frame": "%dx%d" % (NY, NX), "L": L, "dk": DK, "db": DB,
                       "sample": "%dx%d pair per step, scaled to 4088^2 by pixel count" % (size, size)},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d steps, each one %dx%d pair (fit + subtract), scaled by pixel count"
                                       % (args.steps, size, size)},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
