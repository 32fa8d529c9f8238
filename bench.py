#!/usr/bin/env python
"""Throughput of the SFFT fit + subtraction on GB300: 4088 x 4088 difference images per second.

One step = fit + subtract for every pair in this rank's batch of seeded synthetic Roman-like
4088^2 float32 pairs, in the batched + learned form (warm starts from the trained network,
all pairs in one graph-captured multi-lane batch) whose rate is `value`; the plain form (one
plan, pairs in sequence, FP64 Cholesky) is timed on the same pairs and reported beside it.
Each pair has ~3000 Moffat stars per frame, FWHM 1.8 -> 2.4 px across the frame,
Poisson sky 80 e- subtracted, 0.5% + 0.5% masked pixels; 11 x 11 delta kernel, DK=2, DB=2,
732 unknowns.  Inputs are resident in HBM before the timed region; each pair's frames
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
    ap.add_argument("--pairs", type=int, default=8, help="pairs per step per rank")
    ap.add_argument("--lanes", type=int, default=8, help="streams of the batched form (at most --pairs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-samples", type=int, default=20000, help="warm-start network training fits")
    ap.add_argument("--frame", type=int, default=NY, help="frame side (smaller frames are for profiling runs)")
    ap.add_argument("--plain-only", action="store_true", help="time the plain form only (profiling runs)")
    ap.add_argument("--train-epochs", type=int, default=8)
    ap.add_argument("--pcg-cluster", type=int, default=0, choices=[0, 8, 16],
                    help="PCG cluster size for the batched form (0: the tuner's / largest available)")
    ap.add_argument("--workload", default="roman4088",
                    choices=["roman4088", "sxt48", "learned256", "stress4088", "library"],
                    help="roman4088: the headline line; sxt48: 8 x 6 science/template pairs of uneven "
                         "cutout sizes, batched vs sequential; learned256: 256 batched 2048^2 pairs "
                         "with and without the network's warm starts; stress4088: the precision-stress "
                         "shape (L=15, DK=3, DB=2, 1e5 flux range) in SPLIT and FP64; library: the "
                         "cuFFT + cuSOLVER comparison build on the headline pairs")
    return ap.parse_args()


def pair_seeds(rank: int, pairs: int):
    """Seeds of this rank's pairs: ranks draw disjoint pairs (weak scaling, no shared data)."""
    return [1000 + 100 * rank + i for i in range(pairs)]


def pair_field(seed: int):
    """PSF fields of the pair drawn with this seed: round Moffats whose FWHM runs linearly
    1.8 -> 2.4 px across the frame, along a direction drawn per pair and per image (the pair
    with seed 1000 keeps x for the template and y for the science image), so that the
    warm-start network sees a different input for every pair."""
    import numpy as np
    from paper_2509_18544_gb300 import synth
    if seed == 1000:
        return synth.roman_field()
    th = np.random.Generator(np.random.PCG64(seed + 77)).uniform(0.0, 2.0 * np.pi, 2)
    return synth.linear_field(th[0], th[1])


def max_over_ranks(v: float, world: int, device=None) -> float:
    """Largest value over the ranks (the timed region ends when the slowest rank ends)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(steps: int, pairs: int, world: int, ms: float) -> float:
    """Whole-job difference images per second: every rank's pairs over the slowest rank's time."""
    return steps * pairs * world / (ms / 1e3)


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
    from paper_2509_18544_gb300 import learned, sfft, synth

    sfft_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    NY = NX = args.frame
    workload = WORKLOAD if args.frame == 4088 else WORKLOAD.replace("4088x4088", "%dx%d" % (NY, NX))
    seeds = pair_seeds(rank, args.pairs)
    pairs = [synth.roman_pair(NY, NX, seed=sd, field=pair_field(sd)) for sd in seeds]
    dev_pairs = [tuple(torch.from_numpy(a).to(dev) for a in p) for p in pairs]
    stream = torch.cuda.current_stream(dev)
    n = L * L * (DK + 1) * (DK + 2) // 2 + (DB + 1) * (DB + 2) // 2

    def timed(step, steps, name):
        """ms of `steps` calls of step(), CUDA events on the launching stream, barriers and
        synchronisation on both sides; the loop is an NVTX range `name` (for profilers)."""
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.nvtx.range(name):
            for _ in range(steps):
                step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), world, dev)

    # ================= plain: one plan, pairs in sequence, FP64 Cholesky
    plan = sfft.sfft_plan(sfft.make_desc(NY, NX, L, DK, DB), stream=stream)
    coeffs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in pairs]
    diffs = [torch.empty((NY, NX), dtype=torch.float32, device=dev) for _ in pairs]

    def plain_step():
        for (S, T, M), th, D in zip(dev_pairs, coeffs, diffs):
            sfft.sfft_fit(plan, S, T, M, None, th, want_info=False)
            sfft.sfft_subtract(plan, S, T, th, D)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_step()
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(max(args.warmup - 1, 0)):
        plain_step()
    info = sfft.sfft_fit(plan, *dev_pairs[0], None, coeffs[0], want_info=True)
    sfft.sfft_stage_times(plan)  # reset the accumulators
    sfft.sfft_profile(plan, True)
    plain_ms = timed(plain_step, args.steps, "plain")
    stages, calls = sfft.sfft_stage_times(plan)
    sfft.sfft_profile(plan, False)
    plain_value = weak_value(args.steps, args.pairs, world, plain_ms)
    if args.plain_only:
        # the pipeline steps around the fit on the plain fits' coefficients and differences
        steps_info = pipeline_steps(args, dev, stream, dev_pairs, seeds, coeffs, diffs, NY, NX,
                                    plain_ms / (args.steps * args.pairs))
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(plain_value, 3), "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": round(plain_ms / args.steps, 3), "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                              "config": {"workload": workload, "mode": "plain only (profiling run)",
                                         "pairs_per_step_per_rank": args.pairs},
                              "stages_ms_per_pair": {k: round(v / max(calls, 1), 4) for k, v in stages.items()},
                              "pipeline_steps": steps_info}),
                  flush=True)
        plan.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # ================= batched + learned: CNN warm starts, graph-captured PCG batch in lanes
    t0 = time.perf_counter()
    tr_stamps, tr_targets, _ = learned.make_training_set(args.train_samples, seed=1000, size=256)
    cnn, losses = learned.train(tr_stamps, tr_targets, epochs=args.train_epochs, batch=64, lr=1e-3,
                                stream=stream)
    train_s = time.perf_counter() - t0
    del tr_stamps, tr_targets
    # each pair's own PSF fields
    stamps = torch.from_numpy(np.stack([synth.psf_stamps(pair_field(sd)) for sd in seeds])).to(dev)
    bcoeffs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in pairs]
    bdiffs = [torch.empty((NY, NX), dtype=torch.float32, device=dev) for _ in pairs]
    # the network runs inside the batch: each run evaluates it on the pairs' stamps and starts
    # their PCG solves from its warm starts
    bpairs = [sfft.make_pair(S, T, M, th, D, NY, NX, stamps=stamps[k])
              for k, ((S, T, M), th, D) in enumerate(zip(dev_pairs, bcoeffs, bdiffs))]
    if args.pcg_cluster:
        tn = sfft.sfft_tuning()
        tn.pcg_cluster = args.pcg_cluster
        sfft.sfft_tuning_set(sfft.make_desc(NY, NX, L, DK, DB, solver=sfft.SOLVE_PCG), tn)
    t0 = time.perf_counter()
    batch = sfft.sfft_batch_create(sfft.make_desc(NY, NX, L, DK, DB, solver=sfft.SOLVE_PCG), bpairs,
                                   lanes=min(args.pairs, args.lanes), flags=sfft.BATCH_GRAPH | sfft.BATCH_AUTOTUNE,
                                   stream=stream, cnn=cnn)
    create_s = time.perf_counter() - t0
    tuning, _ = sfft.sfft_tuning_get(sfft.make_desc(NY, NX, L, DK, DB, solver=sfft.SOLVE_PCG))

    def batched_step():
        sfft.sfft_batch_run(batch)

    for _ in range(args.warmup):
        batched_step()
    binfos = sfft.sfft_batch_info(batch)
    clocks = ClockSampler(local)
    launches0 = sfft.sfft_launch_count()
    clocks.start()
    ms = timed(batched_step, args.steps, "batched")
    clk = clocks.stop()
    launches = sfft.sfft_launch_count() - launches0
    value = weak_value(args.steps, args.pairs, world, ms)
    binfos = sfft.sfft_batch_info(batch)

    # ---- the same batch from cold starts (no warm start): what the network contributes
    cold_pairs = [sfft.make_pair(S, T, M, th, D, NY, NX)
                  for (S, T, M), th, D in zip(dev_pairs, bcoeffs, bdiffs)]
    cold = sfft.sfft_batch_create(sfft.make_desc(NY, NX, L, DK, DB, solver=sfft.SOLVE_PCG), cold_pairs,
                                  lanes=min(args.pairs, args.lanes), flags=sfft.BATCH_GRAPH, stream=stream)
    for _ in range(args.warmup):
        sfft.sfft_batch_run(cold)
    cold_ms = timed(lambda: sfft.sfft_batch_run(cold), args.steps, "cold")
    cold_value = weak_value(args.steps, args.pairs, world, cold_ms)
    cinfos = sfft.sfft_batch_info(cold)
    cold.close()

    # ---- end to end through the public API with pinned host buffers (batched + learned): a
    # second batch whose pairs carry their host buffers, so each lane copies its pair's inputs
    # in before the fit and D and theta out after the subtraction, overlapping other lanes
    host = [dict(sci=torch.from_numpy(S).pin_memory(), tmpl=torch.from_numpy(T).pin_memory(),
                 mask=torch.from_numpy(M).pin_memory(), coeffs=torch.empty(n, dtype=torch.float64).pin_memory(),
                 diff=torch.empty((NY, NX), dtype=torch.float32).pin_memory()) for S, T, M in pairs]
    e2e_in = [tuple(torch.empty_like(t) for t in p) for p in dev_pairs]
    e2e_th = [torch.empty(n, dtype=torch.float64, device=dev) for _ in pairs]
    e2e_D = [torch.empty((NY, NX), dtype=torch.float32, device=dev) for _ in pairs]
    e2e_pairs = [sfft.make_pair(dS, dT, dM, th, D, NY, NX, host=host[k], stamps=stamps[k])
                 for k, ((dS, dT, dM), th, D) in enumerate(zip(e2e_in, e2e_th, e2e_D))]
    e2e_batch = sfft.sfft_batch_create(sfft.make_desc(NY, NX, L, DK, DB, solver=sfft.SOLVE_PCG), e2e_pairs,
                                       lanes=min(args.pairs, args.lanes), flags=sfft.BATCH_GRAPH, stream=stream,
                                       cnn=cnn)

    def e2e_step():
        sfft.sfft_batch_run(e2e_batch)

    for _ in range(2):
        e2e_step()
    e2e_steps = max(2, args.steps // 2)
    e2e_ms = timed(e2e_step, e2e_steps, "e2e")
    e2e_value = weak_value(e2e_steps, args.pairs, world, e2e_ms)
    h2d = args.pairs * sum(host[0][k].numel() * host[0][k].element_size() for k in ("sci", "tmpl", "mask"))
    d2h = args.pairs * (host[0]["diff"].numel() * 4 + n * 8)
    e2e_batch.close()

    # ---- the other GPU steps of the pipeline on the same pairs, per pair
    steps_info = pipeline_steps(args, dev, stream, dev_pairs, seeds, bcoeffs, bdiffs, NY, NX, ms / (args.steps * args.pairs))

    # ---- HBM roofline (the metric's HBM roofline %), per stage of the plain pass, from its
    # per-stage CUDA events on the plan's stream.  Algorithmic bytes: the per-pixel figures of
    # the two-pass FFT model of the hot path for the steps each stage performs (a1 + a2 row
    # pass: read S, T, m and write the spectra, 61 B/px; a2 column pass: 104 B/px; a3 + a4
    # cross-spectra and pruned inverse: 55 B/px; a7 convolve-subtract: 120 B/px), beside this
    # design's own minimum traffic (each input read once, each output written once).
    px = float(NY * NX)
    g_nseg = -(-NX // (256 - 2 * (L - 1)))
    nk, nb = (DK + 1) * (DK + 2) // 2, (DB + 1) * (DB + 2) // 2
    nrec = (2 * (DK + 1) + (DB + 1) + 1 + 1) // 2 * 2
    spec_bytes = g_nseg * NY * 129 * nrec * 8.0
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6785.5)
    calls_ = max(calls, 1)
    stage_ms = {k: round(v / calls_, 4) for k, v in stages.items()}

    def hbm_stage(name, steps, survey_bpx, own_bytes):
        t = stages[name] / calls_ * 1e-3
        a = survey_bpx * px / t / 1e9
        return {"steps": steps, "ms": round(t * 1e3, 4), "bytes": round(survey_bpx * px), "achieved": round(a, 1),
                "frac": round(a / hbm, 4), "own_bytes": round(own_bytes),
                "own_frac": round(own_bytes / t / 1e9 / hbm, 4)}

    # CTAs per frequency of the y-FFT kernel (the library's choice: the fullest last wave of
    # one CTA per SM, at least 8 (segment, block) units per CTA)
    units = g_nseg * (-(-NY // (128 - 2 * (L - 1))))
    best, y2split = -1.0, 1
    for sp in range(1, 17):
        if sp > 1 and units // sp < 8:
            break
        ctas = 129 * sp
        eff = ctas / (-(-ctas // sms) * sms)
        if eff > best + 1e-9:
            best, y2split = eff, sp
    hbm_stages = {
        "segment_fft": hbm_stage("segment_fft", "a1 + a2 row pass", 61.0, 9.0 * px + spec_bytes),
        "ycorr": hbm_stage("ycorr", "a2 column pass + a3 (+ a4 reads)", 104.0 + 55.0,
                           spec_bytes + y2split * 129 * (nk * (nk + 1) // 2 + nk * (nb + 1)) * 128 * 16.0),
        "subtract": hbm_stage("subtract", "a7 (direct route)", 120.0, 12.0 * px),
    }
    # DRAM bytes measured by ncu on one 2048^2 launch of each stage's kernel (dram__bytes_read.sum
    # + dram__bytes_write.sum, the profiles/ summaries), scaled by the pixel count; writes still
    # in L2 when a launch ends are not counted there
    for key, rd, wr in (("segment_fft", 37.878e6, 130.446e6), ("ycorr", 191.260e6, 94.586e6),
                        ("subtract", 36.672e6, 0.006e6)):
        hbm_stages[key]["traffic"] = round((rd + wr) * px / (2048.0 * 2048.0))
    pair_ms = plain_ms / (args.steps * args.pairs)
    whole = {"plain_ms_per_pair": round(pair_ms, 4), "batched_ms_per_pair": round(ms / (args.steps * args.pairs), 4),
             "bytes": round(340.0 * px),
             "plain_frac": round(340.0 * px / (pair_ms * 1e-3) / 1e9 / hbm, 4),
             "batched_frac": round(340.0 * px / (ms / (args.steps * args.pairs) * 1e-3) / 1e9 / hbm, 4)}
    # the dominant GPU-wide kernel: the y correlation (k_ycorr_fft32); DRAM bytes of one
    # launch from an ncu capture of this kernel on a 2048^2 pair (191.3 MB read + 94.6 MB
    # written), scaled to the frame by its pixel count (its traffic grows in proportion)
    yc = hbm_stages["ycorr"]
    traffic = (191.260e6 + 94.586e6) * px / (2048.0 * 2048.0)
    ycorr_flops = 129 * g_nseg * (-(-NY // 108)) * ((2 * nk + nb + 1) * 2824.0 + (nk * (nk + 1) // 2 + nk * (nb + 1)) * 128 * 8.0)
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    roofline = {"bound": "hbm", "kernel": "k_ycorr_fft32 (y correlation: block FFTs + cross-spectra)",
                "achieved": yc["achieved"], "peak": hbm, "unit": "GB/s", "frac": yc["frac"], "traffic": round(traffic),
                "bytes_per_launch": yc["bytes"], "ms_per_launch": yc["ms"],
                "peak_source": "MEASURED_PEAKS hbm_gbs (copy bandwidth)",
                "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one launch at 2048^2, scaled by pixels",
                "own_bytes_frac": yc["own_frac"],
                "alu": {"flops_per_launch": ycorr_flops, "achieved_tflops": round(ycorr_flops / (yc["ms"] * 1e-3) / 1e12, 2),
                        "peak_tflops": round(fp32_peak, 2),
                        "frac": round(ycorr_flops / (yc["ms"] * 1e-3) / 1e12 / fp32_peak, 4),
                        "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz" % (sms, peaks.get("sm_max_mhz", 2070.0))}}

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "frame": "%dx%d" % (NY, NX), "L": L, "dk": DK, "db": DB,
                   "pairs_per_step_per_rank": args.pairs,
                   "mode": "batched+learned: CNN warm starts, %d-lane CUDA-graph batch, autotuned, cluster PCG "
                           "(FP32 Cholesky preconditioner, FP64 residuals), FP32 spectra, one compensated "
                           "refinement pass" % min(args.pairs, args.lanes),
                   "l2": "inputs larger than L2 (150 MB frames + 1.5 GB spectra per pair); no flush",
                   "parallelism": "replicas: independent pairs per GPU" if world > 1 else "1 GPU"},
        "plain": {"value": round(plain_value, 3), "ms_per_step": round(plain_ms / args.steps, 3),
                  "mode": "one plan, pairs in sequence, FP64 Cholesky, one compensated refinement pass",
                  "stages_ms_per_pair": stage_ms, "first_call_ms": round(first_ms, 1),
                  "fit_rel_residual": info.rel_residual},
        "batched_over_plain": round(value / plain_value, 3),
        "learned": {"train_samples": args.train_samples, "train_epochs": args.train_epochs,
                    "train_s": round(train_s, 1), "loss_first": losses[0], "loss_last": losses[-1],
                    "warm_value": round(value, 3), "cold_value": round(cold_value, 3),
                    "warm_over_cold": round(value / cold_value, 4),
                    "pcg_iterations": [i.iterations for i in binfos],
                    "pcg_iterations_cold": [i.iterations for i in cinfos],
                    "mean_iterations_warm": sum(i.iterations for i in binfos) / len(binfos),
                    "mean_iterations_cold": sum(i.iterations for i in cinfos) / len(cinfos),
                    "start_residual": [round(i.start_residual, 4) for i in binfos],
                    "fallbacks": sum(i.fallback for i in binfos)},
        "batch": {"create_s": round(create_s, 2),
                  "tuning": {"ycorr_bins": tuning.ycorr_bins, "ycorr_split": tuning.ycorr_split,
                             "ycorr_scalar": tuning.ycorr_scalar, "subtract_ctas": tuning.subtract_ctas,
                             "pcg_cluster": tuning.pcg_cluster, "ycorr_direct": tuning.ycorr_direct,
                             "ycorr_sets": tuning.ycorr_sets, "subtract_fft": tuning.subtract_fft,
                             "note": "0 = the library's default for that field"}},
        "roofline": roofline,
        "hbm_stages": hbm_stages,
        "hbm_whole_path": whole,
        "pipeline_steps": steps_info,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if world > 1:
        dist.barrier()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(result), flush=True)
    batch.close()
    cnn.close()
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def pipeline_steps(args, dev, stream, dev_pairs, seeds, coeffs, diffs, NY, NX, fit_ms_per_pair):
    """Per-pair device time of the GPU steps around the fit (Sec. "Pipeline steps"), on the
    benchmark's own pairs: step 4 (template and mask resampled onto the science grid with a
    0.3 degree rotation, a 1e-4 scale change, a sub-pixel shift and a cubic distortion;
    Lanczos-3; the template PSF aligned), step 5 (cross-convolution with 25 x 25 stamps),
    step 7 (decorrelation kernel at the frame centre, applied to D and to the cross-convolved
    science image) and steps 8-9 (forced photometry of 500 field stars and the transient per
    pair, constant background).  Roofline per step: the own-traffic HBM fraction (each
    input read once, each output written once) for the resampler, the FP32 fraction of the
    row-segment FFT route's flops for the two convolutions."""
    import math

    import numpy as np
    import torch

    from paper_2509_18544_gb300 import sfft, synth

    P = len(dev_pairs)
    K, M = 25, 25
    fields = [pair_field(sd) for sd in seeds]
    ps = [torch.from_numpy(synth.psf_stamp_at(f, "sci", 0.0, 0.0, K)).to(dev) for f in fields]
    pt = [torch.from_numpy(synth.psf_stamp_at(f, "tmpl", 0.0, 0.0, K)).to(dev) for f in fields]
    th, sc = math.radians(0.3), 1.0001
    c, sn, x0 = sc * math.cos(th), sc * math.sin(th), (NX - 1) / 2.0
    warp = sfft.make_warp(3, [x0 + 3.37, c, -sn, 0, 0, 0, 1e-10, 0, 0, 0],
                          [x0 - 2.81, sn, c, 0, 0, 0, 0, 0, 1e-10, 0], x0, x0)
    t_al = [torch.empty_like(p[1]) for p in dev_pairs]
    m_al = [torch.empty_like(p[2]) for p in dev_pairs]
    psf_al = [torch.empty_like(x) for x in pt]
    s_cc = [torch.empty_like(p[0]) for p in dev_pairs]
    t_cc = [torch.empty_like(p[1]) for p in dev_pairs]
    phi = [torch.empty((M, M), dtype=torch.float32, device=dev) for _ in range(P)]
    psf_dec = [torch.empty((M, M), dtype=torch.float32, device=dev) for _ in range(P)]
    d_dec = [torch.empty_like(p[0]) for p in dev_pairs]
    s_dec = [torch.empty_like(p[0]) for p in dev_pairs]
    rng = np.random.default_rng(5)
    jobs = []
    for k in range(P):
        xs, ys = rng.uniform(20, NX - 20, 501), rng.uniform(20, NY - 20, 501)
        jobs += [dict(image=d_dec[k], psf=psf_dec[k], x=x, y=y) for x, y in zip(xs, ys)]
    arr = sfft.phot_jobs(jobs)
    jobs_dev = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(dev)
    res = torch.empty((len(jobs), 8), dtype=torch.float64, device=dev)

    def step4():
        for k, (S, T, Mk) in enumerate(dev_pairs):
            sfft.sfft_resample(warp, T, t_al[k], Mk, m_al[k], sfft.LANCZOS3, 0, stream=stream)
            sfft.sfft_align_psf(warp, x0, x0, pt[k], psf_al[k], stream=stream)

    def step5():
        for k, (S, T, Mk) in enumerate(dev_pairs):
            sfft.sfft_cross_convolve(NY, NX, K, S, T, ps[k], pt[k], s_cc[k], t_cc[k], stream=stream)

    def step7k():
        for k in range(P):
            sfft.sfft_decorrelation_kernel(NY, NX, L, DK, coeffs[k], x0, x0, ps[k], pt[k], 1.0, 1.0, phi[k],
                                           psf_dec[k], stream=stream)

    def step7a():
        for k in range(P):
            sfft.sfft_cross_convolve(NY, NX, M, diffs[k], s_cc[k], phi[k], phi[k], d_dec[k], s_dec[k], stream=stream)

    def step9():
        sfft.sfft_forced_photometry(jobs_dev, len(jobs), M, res, sfft.PHOT_BACKGROUND, stream=stream)

    ms = {}
    for name, fn in (("align_resample", step4), ("cross_convolve", step5), ("decorrelation_kernel", step7k),
                     ("decorrelation_apply", step7a), ("forced_photometry", step9)):
        fn()
        ms[name] = _timed_once(fn, stream, reps=5) / P
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6785.5)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32 = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    px = float(NY * NX)
    # the convolutions run on the row-segment FFT route (K >= 9): per 256-column segment and
    # image, a 256-point complex FFT (5 N log2 N flops) per two input rows (32 + K - 1 rows per
    # 32 output rows), K complex multiply-adds (8 flops) per output row and half-spectrum bin
    # (128 per U = 257 - K columns), and one inverse FFT per two output rows
    def fft_conv_flops(k):
        u, fft = 257 - k, 5.0 * 256 * 8
        per_px = (fft / 2 * (32 + k - 1) / 32 + 8.0 * k * 128 + fft / 2) / u
        return 2 * per_px * px  # two images
    conv_flops = fft_conv_flops(K)
    total = sum(ms.values()) + fit_ms_per_pair
    bad = int((res[:, 5] != 0).sum().item())
    return {
        "ms_per_pair": {k: round(v, 4) for k, v in ms.items()},
        "fit_subtract_ms_per_pair": round(fit_ms_per_pair, 4),
        "pipeline_pairs_per_s": round(1e3 / total, 2),
        "roofline": {
            "align_resample": {"bound": "hbm", "own_bytes": round(10.0 * px),
                               "frac": round(10.0 * px / (ms["align_resample"] * 1e-3) / 1e9 / hbm, 4)},
            "cross_convolve": {"bound": "alu", "route": "row-segment FFT", "flops": conv_flops,
                               "frac": round(conv_flops / (ms["cross_convolve"] * 1e-3) / fp32, 4),
                               "direct_equivalent_flops": 2 * 2.0 * K * K * px,
                               "hbm_own_frac": round(16.0 * px / (ms["cross_convolve"] * 1e-3) / 1e9 / hbm, 4)},
            "decorrelation_apply": {"bound": "alu", "flops": fft_conv_flops(M),
                                    "frac": round(fft_conv_flops(M) / (ms["decorrelation_apply"] * 1e-3) / fp32, 4),
                                    "direct_equivalent_flops": 2 * 2.0 * M * M * px},
        },
        "photometry_jobs_per_pair": 501, "photometry_unsolved": bad,
        "config": "steps 4, 5, 7, 8-9 on the benchmark's pairs: rotation 0.3 deg + 1e-4 scale + cubic "
                  "distortion, Lanczos-3 with mask; 25 x 25 stamps; M = 25 decorrelation kernel; 501 photometry "
                  "jobs per pair",
    }


# ----------------------------------------------------------------------------- oracle arm
def oracle_full_pair(seed: int):
    """FP64 oracle fit + subtraction of one full 4088^2 pair of the workload (seconds, pair)."""
    import oracle
    from paper_2509_18544_gb300 import synth

    S, T, M = synth.roman_pair(NY, NX, seed=seed)
    t0 = time.perf_counter()
    th = oracle.fit(S, T, M, L, DK, DB)
    oracle.subtract(S, T, th, L, DK, DB)
    return time.perf_counter() - t0


def cpu_baseline():
    import oracle
    oracle.build()
    dt = oracle_full_pair(seed=77)
    return {"value": round(1.0 / dt, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "one full 4088x4088 pair of the workload (seed 77), L=11 DK=2 DB=2: FP64 lag tables by "
                      "direct sums, Cholesky and difference image in %.1f s" % dt}


class OracleSlices:
    """The oracle's fit + subtraction of one 4088^2 pair cut into `k` consecutive slices: slice
    i computes the lag tables of row band i (the sums restricted to those rows, which add up to
    the full tables); the last slice also adds the bands up, assembles N and b, solves and forms
    the whole difference image.  Running every slice is exactly one full oracle pair."""

    def __init__(self, seed: int, k: int, size: int = NY):
        from paper_2509_18544_gb300 import synth
        self.S, self.T, self.M = synth.roman_pair(size, size, seed=seed)
        self.k = k
        self.edges = [round(i * size / k) for i in range(k + 1)]
        self.parts = []

    def run(self, i: int):
        import oracle
        y0, y1 = self.edges[i], self.edges[i + 1]
        self.parts.append(oracle.lag_tables_band(self.S, self.T, self.M, L, DK, DB, y0, y1))
        if i == self.k - 1:
            tab = {key: sum(p[key] for p in self.parts) for key in self.parts[0]}
            N, b = oracle.assemble(tab, L, DK, DB)
            th = oracle.cholesky_solve(N, b)
            oracle.subtract(self.S, self.T, th, L, DK, DB)
            self.parts = []


def run_reference(args, world, rank):
    """The oracle timed on this host's cores: the K timed steps together are one full 4088^2
    pair (step i = slice i of OracleSlices); the warm-up steps run slices of another pair."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    steps = max(1, args.steps)
    size = args.frame  # 4088 unless a smaller frame is asked for (quick checks)
    warm = OracleSlices(seed=999, k=steps, size=size)
    for i in range(min(args.warmup, steps)):
        warm.run(i)
    del warm
    timed = OracleSlices(seed=1000, k=steps, size=size)
    t0 = time.perf_counter()
    for i in range(steps):
        timed.run(i)
    total = time.perf_counter() - t0
    value = 1.0 / total
    sample = ("one full %dx%d pair of the workload (seed 1000) split into %d steps: step i sums the lag "
              "tables over row band i, the last step also assembles, solves (FP64 Cholesky) and forms the "
              "whole difference image; %d warm-up steps run bands of another pair" % (size, size, steps, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(total / steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if size == NY else WORKLOAD.replace("4088x4088", "%dx%d" % (size, size)),
                       "frame": "%dx%d" % (size, size), "L": L, "dk": DK, "db": DB,
                       "pairs_per_step": round(1.0 / steps, 6), "sample": sample},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- other workloads
def _timed_once(step, stream, reps=3):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_sxt48(args):
    """8 science x 6 template pairs, each a cutout of its own size from {512, 1024, 1536, 2048}^2
    (L = 11, DK = 2, DB = 1): the whole batch as one graph over 4 lanes (autotuned, PCG) against
    the 48 pairs fitted one after another on single plans (FP64 Cholesky)."""
    import torch
    from paper_2509_18544_gb300 import build as sfft_build
    from paper_2509_18544_gb300 import sfft, synth
    sfft_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n_sci, n_tmpl, Lk, dk, db = 8, 6, 11, 2, 1
    sizes = synth.cutout_sizes(n_sci * n_tmpl, seed=2000)
    pairs = [tuple(torch.from_numpy(a).to(dev) for a in synth.roman_pair(z, z, seed=2000 + k))
             for k, z in enumerate(sizes)]
    n = Lk * Lk * (dk + 1) * (dk + 2) // 2 + (db + 1) * (db + 2) // 2
    th = [torch.empty(n, dtype=torch.float64, device=dev) for _ in pairs]
    Ds = [torch.empty_like(p[0]) for p in pairs]
    plans = {z: sfft.sfft_plan(sfft.make_desc(z, z, Lk, dk, db), stream=stream) for z in set(sizes)}

    def plain_step():
        for (S, T, M), z, t, D in zip(pairs, sizes, th, Ds):
            sfft.sfft_fit(plans[z], S, T, M, None, t, want_info=False)
            sfft.sfft_subtract(plans[z], S, T, t, D)

    plain_step()
    plain_ms = _timed_once(plain_step, stream, args.steps)
    bth = [torch.empty(n, dtype=torch.float64, device=dev) for _ in pairs]
    bD = [torch.empty_like(p[0]) for p in pairs]
    bp = [sfft.make_pair(S, T, M, t, D, z, z) for (S, T, M), z, t, D in zip(pairs, sizes, bth, bD)]
    t0 = time.perf_counter()
    batch = sfft.sfft_batch_create(sfft.make_desc(512, 512, Lk, dk, db, solver=sfft.SOLVE_PCG), bp, lanes=4,
                                   flags=sfft.BATCH_GRAPH | sfft.BATCH_AUTOTUNE, stream=stream)
    create_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        sfft.sfft_batch_run(batch)
    ms = _timed_once(lambda: sfft.sfft_batch_run(batch), stream, args.steps)
    infos = sfft.sfft_batch_info(batch)
    worst = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(bth, th))
    print(json.dumps({"metric": "S x T batch throughput (difference images/s)", "value": round(48 / (ms / 1e3), 2),
                      "unit": "difference images/s", "workload": "sxt48: 8 x 6 pairs, cutouts %s px^2, L=11 DK=2 DB=1"
                      % sorted(set(sizes)), "sizes": sizes, "batched_ms": round(ms, 2),
                      "sequential_plain_ms": round(plain_ms, 2), "sequential_plain_value": round(48 / (plain_ms / 1e3), 2),
                      "batched_over_sequential": round(plain_ms / ms, 3), "create_s": round(create_s, 2),
                      "max_rel_coeff_diff_vs_sequential": worst,
                      "statuses": sorted(set(i.status for i in infos)),
                      "pcg_fallbacks": sum(i.fallback for i in infos)}), flush=True)
    batch.close()
    for p in plans.values():
        p.close()


def library_fit_subtract(S, T, M, L, dk, db):
    """The same fit and subtraction built on library routines, as a comparison baseline only:
    full-frame 2-D FFTs (cuFFT through torch.fft, FP32), every lag table from a full inverse
    FFT of its cross-spectrum, the normal matrix assembled and solved in FP64 (cuSOLVER
    Cholesky through torch.linalg), the difference image by FFT convolution.  Returns
    (theta, D)."""
    import torch
    dev = S.device
    ny, nx = S.shape
    h, G = (L - 1) // 2, L - 1
    good = (M == 0).to(torch.float32) if M is not None else torch.ones_like(S)
    Tm, Sm = torch.where(good > 0, T, torch.zeros_like(T)), torch.where(good > 0, S, torch.zeros_like(S))
    xh = torch.linspace(-1.0, 1.0, nx, device=dev, dtype=torch.float64).to(torch.float32)
    yh = torch.linspace(-1.0, 1.0, ny, device=dev, dtype=torch.float64).to(torch.float32)

    def monos(d):
        return [(deg - q, q) for deg in range(d + 1) for q in range(deg + 1)]

    mk, mb = monos(dk), monos(db)
    wmon = lambda p, q: yh[:, None] ** q * xh[None, :] ** p
    W = torch.stack([wmon(p, q) * Tm for p, q in mk])
    Psi = torch.stack([wmon(p, q) * good for p, q in mb])
    FW, FP, FS = torch.fft.rfft2(W), torch.fft.rfft2(Psi), torch.fft.rfft2(Sm)
    nk, nb = len(mk), len(mb)
    dys = torch.arange(-G, G + 1, device=dev)

    def lags(FA, FB, r):
        c = torch.fft.irfft2(torch.conj(FA) * FB, s=(ny, nx))  # C(d) = sum_u A(u) B(u + d)
        iy = (torch.arange(-r, r + 1, device=dev) % ny)[:, None]
        ix = (torch.arange(-r, r + 1, device=dev) % nx)[None, :]
        return c[iy, ix].to(torch.float64)

    ns, nker = L * L, nk * L * L
    n = nker + nb
    N = torch.empty((n, n), dtype=torch.float64, device=dev)
    bvec = torch.empty(n, dtype=torch.float64, device=dev)
    l = torch.arange(ns, device=dev)
    dyl, dxl = l // L - h, l % L - h
    ddy = (dyl[:, None] - dyl[None, :]) + G
    ddx = (dxl[:, None] - dxl[None, :]) + G
    for i in range(nk):
        for j in range(i, nk):
            C = lags(FW[i], FW[j], G)
            blk = C[ddy, ddx]  # <Phi_i,d, Phi_j,d'> = C_ij(d - d')
            N[i * ns:(i + 1) * ns, j * ns:(j + 1) * ns] = blk
            N[j * ns:(j + 1) * ns, i * ns:(i + 1) * ns] = blk.T
        for r in range(nb):
            v = lags(FW[i], FP[r], h).reshape(-1)
            N[i * ns:(i + 1) * ns, nker + r] = v
            N[nker + r, i * ns:(i + 1) * ns] = v
        bvec[i * ns:(i + 1) * ns] = lags(FW[i], FS, h).reshape(-1)
    P64 = Psi.to(torch.float64)
    N[nker:, nker:] = torch.einsum("ayx,byx->ab", P64, P64)
    bvec[nker:] = torch.einsum("ayx,yx->a", P64, Sm.to(torch.float64))
    theta = torch.cholesky_solve(bvec[:, None], torch.linalg.cholesky(N))[:, 0]
    # D = S - sum_pq (kernel_pq * (w_pq T)) - background, the kernels as cyclic images
    model = torch.zeros((ny, nx // 2 + 1), dtype=torch.complex64, device=dev)
    for i, (p, q) in enumerate(mk):
        kimg = torch.zeros((ny, nx), dtype=torch.float32, device=dev)
        kimg[dyl % ny, dxl % nx] = theta[i * ns:(i + 1) * ns].to(torch.float32)
        model += torch.fft.rfft2(wmon(p, q) * T) * torch.fft.rfft2(kimg)
    D = S - torch.fft.irfft2(model, s=(ny, nx))
    for r, (p, q) in enumerate(mb):
        D -= theta[nker + r].to(torch.float32) * wmon(p, q)
    return theta, D


def run_library(args):
    """Comparison baseline: `library_fit_subtract` (cuFFT + cuSOLVER) on the headline pairs,
    timed like the plain form, with its agreement with libsfft's coefficients."""
    import torch
    from paper_2509_18544_gb300 import build as sfft_build
    from paper_2509_18544_gb300 import sfft, synth
    sfft_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    npairs = min(args.pairs, 4)
    seeds = pair_seeds(0, npairs)
    data = [tuple(torch.from_numpy(a).to(dev) for a in synth.roman_pair(NY, NX, seed=sd, field=pair_field(sd)))
            for sd in seeds]
    with torch.no_grad():
        for S, T, M in data[:1]:
            library_fit_subtract(S, T, M, L, DK, DB)
        ms = _timed_once(lambda: [library_fit_subtract(S, T, M, L, DK, DB) for S, T, M in data], stream, 1)
        th_lib = [library_fit_subtract(S, T, M, L, DK, DB)[0] for S, T, M in data]
    n = L * L * (DK + 1) * (DK + 2) // 2 + (DB + 1) * (DB + 2) // 2
    with sfft.sfft_plan(sfft.make_desc(NY, NX, L, DK, DB), stream=stream) as plan:
        th = torch.empty(n, dtype=torch.float64, device=dev)
        D = torch.empty_like(data[0][0])

        def ours():
            for S, T, M in data:
                sfft.sfft_fit(plan, S, T, M, None, th, want_info=False)
                sfft.sfft_subtract(plan, S, T, th, D)

        ours()
        ours_ms = _timed_once(ours, stream, 3)
        errs = []
        for (S, T, M), tl in zip(data, th_lib):
            sfft.sfft_fit(plan, S, T, M, None, th, want_info=True)
            errs.append(float(torch.linalg.norm(tl - th) / torch.linalg.norm(th)))
    print(json.dumps({"metric": "4088^2 difference images/s, library comparison build", "unit": UNIT,
                      "value": round(npairs / (ms / 1e3), 3), "ms_per_pair": round(ms / npairs, 2),
                      "workload": "%d headline pairs (4088^2, L=11, DK=2, DB=2, masked)" % npairs,
                      "library": "cuFFT 2-D FFTs (FP32) + full inverse per cross-spectrum, cuSOLVER Cholesky (FP64), "
                                 "FFT convolution for the difference image, through torch",
                      "libsfft_plain_ms_per_pair": round(ours_ms / npairs, 2),
                      "libsfft_over_library": round(ms / ours_ms, 2),
                      "library_coeff_rel_diff_vs_libsfft": errs}), flush=True)


def run_stress(args):
    """The precision-stress shape: a 4088^2 pair with fluxes log-uniform over 1e2..1e7 e-,
    L = 15, DK = 3, DB = 2 (2256 unknowns); fit + subtract in SPLIT precision (FP32 spectra,
    one compensated refinement) and in FP64 throughout, with their coefficient agreement.
    (Agreement with the FP64 CPU oracle is the parity test's job.)"""
    import torch
    from paper_2509_18544_gb300 import build as sfft_build
    from paper_2509_18544_gb300 import sfft, synth
    sfft_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Ls, dks, dbs = 15, 3, 2
    S, T, M = (torch.from_numpy(a).to(dev) for a in synth.roman_pair(NY, NX, seed=3000, flux_mode="dynamic"))
    out = {}
    for name, prec in (("split", sfft.PREC_SPLIT), ("fp64", sfft.PREC_FP64)):
        with sfft.sfft_plan(sfft.make_desc(NY, NX, Ls, dks, dbs, precision=prec), stream=stream) as plan:
            th = torch.empty(plan.n, dtype=torch.float64, device=dev)
            D = torch.empty_like(S)

            def step():
                sfft.sfft_fit(plan, S, T, M, None, th, want_info=False)
                sfft.sfft_subtract(plan, S, T, th, D)

            step()
            ms = _timed_once(step, stream, max(1, min(args.steps, 5)) if prec == sfft.PREC_SPLIT else 1)
            sfft.sfft_fit(plan, S, T, M, None, th, want_info=True)
            out[name] = (ms, th.clone())
    rel = float(torch.linalg.norm(out["split"][1] - out["fp64"][1]) / torch.linalg.norm(out["fp64"][1]))
    print(json.dumps({"metric": "precision-stress 4088^2 difference images/s (SPLIT)", "unit": UNIT,
                      "value": round(1e3 / out["split"][0], 3),
                      "workload": "stress4088: 4088^2 pair, fluxes 1e2..1e7 e-, L=15 DK=3 DB=2 (2256 unknowns)",
                      "split_ms": round(out["split"][0], 2), "fp64_ms": round(out["fp64"][0], 2),
                      "split_vs_fp64_gpu_coeff_rel": rel}), flush=True)


def run_learned256(args):
    """The warm-start network trained on `--train-samples` fits, driving PCG over a batch of
    256 2048^2 pairs (16 distinct seeded pairs, each used 16 times), against the same batch
    from cold starts and against sequential FP64-Cholesky fits."""
    import numpy as np
    import torch
    from paper_2509_18544_gb300 import build as sfft_build
    from paper_2509_18544_gb300 import learned, sfft, synth
    sfft_build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    z, npairs, ndistinct = 2048, 256, 16
    t0 = time.perf_counter()
    st, tg, _ = learned.make_training_set(args.train_samples, seed=1000, size=256)
    cnn, losses = learned.train(st, tg, epochs=args.train_epochs, batch=64, lr=1e-3, stream=stream)
    train_s = time.perf_counter() - t0
    del st, tg
    data = [tuple(torch.from_numpy(a).to(dev) for a in synth.roman_pair(z, z, seed=4000 + k)) for k in range(ndistinct)]
    n = L * L * (DK + 1) * (DK + 2) // 2 + (DB + 1) * (DB + 2) // 2
    stamps = torch.from_numpy(np.repeat(synth.psf_stamps(synth.roman_field())[None], npairs, 0)).to(dev)
    x0 = torch.zeros((npairs, n), dtype=torch.float64, device=dev)
    sfft.sfft_cnn_warm_start(cnn, stamps[:64], 64, n, x0[:64])

    def make(with_x0):
        th = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(npairs)]
        Ds = [torch.empty((z, z), dtype=torch.float32, device=dev) for _ in range(npairs)]
        ps = [sfft.make_pair(*data[k % ndistinct], th[k], Ds[k], z, z, x0=x0[k] if with_x0 else None)
              for k in range(npairs)]
        b = sfft.sfft_batch_create(sfft.make_desc(z, z, L, DK, DB, solver=sfft.SOLVE_PCG), ps, lanes=8,
                                   flags=sfft.BATCH_GRAPH | sfft.BATCH_AUTOTUNE, stream=stream)
        return b, th

    warm, th_w = make(True)
    cold, th_c = make(False)

    def warm_step():
        for s0 in range(0, npairs, 64):
            sfft.sfft_cnn_warm_start(cnn, stamps[s0:s0 + 64], 64, n, x0[s0:s0 + 64])
        sfft.sfft_batch_run(warm)

    for _ in range(args.warmup):
        warm_step()
        sfft.sfft_batch_run(cold)
    warm_ms = _timed_once(warm_step, stream, args.steps)
    cold_ms = _timed_once(lambda: sfft.sfft_batch_run(cold), stream, args.steps)
    iw, ic = sfft.sfft_batch_info(warm), sfft.sfft_batch_info(cold)
    # sequential FP64-Cholesky fits of the distinct pairs, scaled to the batch
    with sfft.sfft_plan(sfft.make_desc(z, z, L, DK, DB), stream=stream) as plan:
        thp = torch.empty(n, dtype=torch.float64, device=dev)
        Dp = torch.empty((z, z), dtype=torch.float32, device=dev)

        def plain_step():
            for S, T, M in data:
                sfft.sfft_fit(plan, S, T, M, None, thp, want_info=False)
                sfft.sfft_subtract(plan, S, T, thp, Dp)

        plain_step()
        plain_ms = _timed_once(plain_step, stream, args.steps) * npairs / ndistinct
        # the judge of the warm-started result: the FP64 Cholesky solution of pair 0
        sfft.sfft_fit(plan, *data[0], None, thp)
        ref = thp.clone()
    err = float(torch.linalg.norm(th_w[0] - ref) / torch.linalg.norm(ref))
    print(json.dumps({"metric": "2048^2 difference images/s, PCG batch with learned warm starts",
                      "value": round(npairs / (warm_ms / 1e3), 2), "unit": "difference images/s",
                      "workload": "learned256: 256 pairs of 2048^2 (16 distinct), L=11 DK=2 DB=2, 8 lanes, graph",
                      "warm_ms": round(warm_ms, 2), "cold_ms": round(cold_ms, 2), "plain_sequential_ms": round(plain_ms, 2),
                      "cold_value": round(npairs / (cold_ms / 1e3), 2), "plain_value": round(npairs / (plain_ms / 1e3), 2),
                      "mean_iterations_warm": sum(i.iterations for i in iw) / npairs,
                      "mean_iterations_cold": sum(i.iterations for i in ic) / npairs,
                      "mean_start_residual_warm": sum(i.start_residual for i in iw) / npairs,
                      "fallbacks_warm": sum(i.fallback for i in iw), "fallbacks_cold": sum(i.fallback for i in ic),
                      "warm_vs_cholesky_rel": err, "train_samples": args.train_samples, "train_s": round(train_s, 1),
                      "loss_first": losses[0], "loss_last": losses[-1]}), flush=True)
    warm.close()
    cold.close()
    cnn.close()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "sxt48":
        run_sxt48(args)
        return
    if args.workload == "learned256":
        run_learned256(args)
        return
    if args.workload == "library":
        run_library(args)
        return
    if args.workload == "stress4088":
        run_stress(args)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
