"""Learned warm start: training data from the method's own fits, training and inference.

Host orchestration only.  The fits, the network's forward and backward passes, the Adam
updates and the warm starts all run in libsfft's kernels through the C ABI
(``sfft_fit``, ``sfft_cnn_train``, ``sfft_cnn_warm_start``).

Training samples: for a seeded random pair of spatially varying PSF fields
(``synth.psf_field``), the input is the 18 x 32 x 32 stack of PSF stamps at the 3 x 3 cell
centres, and the target is the kernel part of the coefficients that ``sfft_fit`` returns
for a noise-free star-grid frame pair drawn with those fields.  The kernel is expressed in
the normalised coordinates xh, yh in [-1, 1], so a network trained on small frames applies
to frames of any size with the same PSF fields.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sfft, synth


def n_kernel(L: int, dk: int) -> int:
    return L * L * (dk + 1) * (dk + 2) // 2


def make_training_set(n: int, seed: int, size: int = 256, L: int = 11, dk: int = 2, db: int = 2,
                      device: str = "cuda", workers: int = 0, chunk: int = 128):
    """(stamps [n][18][32][32] float32, targets [n][L^2 nP(dk)] float32, full coefficients
    [n][n_unknowns] float64), all on the device.

    The frames and stamps are drawn on the host (``synth.training_sample``), in `workers`
    processes (0: one per host core, up to 16; started with "spawn", so no CUDA state is
    forked) a chunk at a time; each chunk is copied to the device in one transfer per array
    and fitted by queued sfft_fit calls while the workers draw the next chunks."""
    import multiprocessing as mp
    import os

    dev = torch.device(device)
    nk = n_kernel(L, dk)
    stamps = torch.empty((n, 18, synth.STAMP, synth.STAMP), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    nw = workers if workers > 0 else max(1, min(16, (os.cpu_count() or 2) - 1))
    jobs = [(seed + s0, min(chunk, n - s0), size) for s0 in range(0, n, chunk)]
    # the targets need no refinement: the plain FP32 mode is well inside the network's error
    with sfft.sfft_plan(sfft.make_desc(size, size, L, dk, db, precision=sfft.PREC_FP32, solver=sfft.SOLVE_PCG),
                        stream=stream) as plan:
        coeffs = torch.empty((n, plan.n), dtype=torch.float64, device=dev)
        S_d = torch.empty((chunk, size, size), dtype=torch.float32, device=dev)
        T_d = torch.empty_like(S_d)
        ctx = mp.get_context("spawn")
        with ctx.Pool(nw) as pool:
            s0 = 0
            for Sc, Tc, stc in pool.imap(synth.training_chunk, jobs):
                c = Sc.shape[0]
                # the previous chunk's fits read S_d, T_d: wait for them before the copies
                stream.synchronize()
                S_d[:c].copy_(torch.from_numpy(Sc))
                T_d[:c].copy_(torch.from_numpy(Tc))
                stamps[s0:s0 + c].copy_(torch.from_numpy(stc))
                for i in range(c):
                    sfft.sfft_fit(plan, S_d[i], T_d[i], None, None, coeffs[s0 + i], want_info=False)
                s0 += c
        sfft.sfft_sync_status(plan)
    targets = coeffs[:, :nk].to(torch.float32).contiguous()
    return stamps, targets, coeffs


def train(stamps, targets, epochs: int = 40, batch: int = 64, lr: float = 1e-3, seed: int = 1,
          init_seed: int = 7, stream=None):
    """A network trained on (stamps, targets); returns (sfft.Cnn, per-epoch losses).

    Initial parameters: seeded He-normal convolutions; the linear head starts at the mean
    training target (its bias) with weights scaled by 0.01, so training learns how the
    kernel departs from the average kernel rather than the kernel itself."""
    n, n_out = targets.shape
    cnn = sfft.sfft_cnn_create(n_out, max(batch, 64), stream=stream)
    p = synth.cnn_init(n_out, init_seed)
    p[-n_out:] = targets.mean(dim=0).cpu().numpy()
    p[-n_out - 128 * n_out:-n_out] *= 0.01
    sfft.sfft_cnn_set_params(cnn, torch.from_numpy(p).to(stamps.device))
    losses = sfft.sfft_cnn_train(cnn, stamps, targets, n, batch, epochs, lr, seed)
    return cnn, losses


def warm_starts(cnn, stamps, n_unknowns: int):
    """x0 [batch][n_unknowns] float64 on the device: the network's kernel coefficients and
    zeros for the background (the PCG solve projects the background itself)."""
    b = stamps.shape[0]
    x0 = torch.empty((b, n_unknowns), dtype=torch.float64, device=stamps.device)
    for s in range(0, b, cnn.max_batch):
        e = min(b, s + cnn.max_batch)
        sfft.sfft_cnn_warm_start(cnn, stamps[s:e], e - s, n_unknowns, x0[s:e])
    return x0
