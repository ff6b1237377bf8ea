"""Throughput of the FP32-batched path on the full-size synthetic workloads beside the 4 x 1024^2
peaks stack of bench.py's main line, one JSON line per workload:

  diffusion  500 x 1024 x 1024 uint16 (12-bit) time-lapse, erfc phase front in y, carrier 0.1 along
             x, derivative along y (column windows), N = 32, L = 8: the whole stack in one call.
  uneven     64 float32 frames of sizes {256..2048} x {256, 512, 1024}, (N, L) per frame from
             {24, 32, 48} x {6, 8, 12}, SNR 15 dB: one call (one persistent launch per distinct L).
  carriers   1024 x 1024 float32 peaks frames at carrier 0.08 / 0.1 / 0.15 cycles/px, 20 dB.

Each call is replayed from its CUDA graph with the L2 flushed before it and timed with CUDA events on
the launching stream (3 warm-ups, 5 timed calls, median). The frames are generated by the seeded
generators of synth.py in a spawned process pool. bench.py runs the diffusion and uneven workloads
through the same functions and adds the maps' agreement with the FP64 oracle on sampled pixels.

    python -m paper_1910_11872_gb300.config_bench [--diffusion-frames 500] [--workers 16]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics

import numpy as np

from . import rmusic, synth


def _diffusion(t: int) -> np.ndarray:
    return synth.diffusion_frame(t).image


def diffusion_stack(frames: int = 500, workers: int = 0) -> np.ndarray:
    """The diffusion time-lapse as one (frames, 1024, 1024) uint16 array, drawn in spawned processes."""
    workers = workers or min(16, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.stack(pool.map(_diffusion, range(frames)))


def time_call(dem, tensors, windows, flush, reps: int = 5, warmup: int = 3):
    """Median event-timed duration of one call (graph replay after the first, L2 flushed before each
    timed call). Returns (ms, out, status, shapes, stats of the last call)."""
    import torch

    out, st, shapes = dem.run(tensors, windows=windows)
    for _ in range(max(warmup - 1, 0)):
        dem.run(tensors, windows=windows, out=out, status=st)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dem.run(tensors, windows=windows, out=out, status=st, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms), out, st, shapes, dem.stats()


def run_diffusion(stack: np.ndarray, flush, reps: int = 5):
    """The whole diffusion stack in one call (derivative along y). Returns (result dict, maps
    (T, H, W) float32 on the device, statuses)."""
    import torch

    dem = rmusic.Demodulator(precision="batched", deriv_axis=1, use_graph=1, timing=1, autotune=1)
    try:
        x = torch.from_numpy(stack.view(np.int16)).cuda()
        ms, out, st, shapes, stats = time_call(dem, x, None, flush, reps)
        npx = x.numel()
        res = {"workload": f"diffusion {stack.shape[0]} x {stack.shape[1]}x{stack.shape[2]} uint16 12-bit, "
                           f"derivative along y, N=32, L=8, one call",
               "value": npx / ms / 1e3, "unit": "Mpixel/s", "ms_per_call": ms, "mpixels": npx / 1e6,
               "solver_ms": stats.solver_ms, "bandpass_ms": stats.bandpass_ms,
               "gpu_launches": stats.kernel_launches, "timing": f"graph replay, L2 flushed, median of {reps}"}
        del x
        return res, out.view(stack.shape), st.view(stack.shape)
    finally:
        dem.close()


def run_uneven(frames, flush, reps: int = 5):
    """The uneven batch in one call (per-frame windows). Returns (result dict, flat maps, statuses,
    shapes)."""
    import torch

    dem = rmusic.Demodulator(precision="batched", use_graph=1, timing=1, autotune=1)
    try:
        tens = [torch.from_numpy(f.image).cuda() for f in frames]
        windows = [(f.window_len, f.cov_order) for f in frames]
        ms, out, st, shapes, stats = time_call(dem, tens, windows, flush, reps)
        npx = sum(f.image.size for f in frames)
        res = {"workload": f"uneven batch: {len(frames)} float32 frames {{256..2048}}x{{256,512,1024}}, (N, L) per "
                           f"frame from {{24,32,48}}x{{6,8,12}}, 15 dB, one call",
               "value": npx / ms / 1e3, "unit": "Mpixel/s", "ms_per_call": ms, "mpixels": npx / 1e6,
               "solver_ms": stats.solver_ms, "bandpass_ms": stats.bandpass_ms,
               "gpu_launches": stats.kernel_launches, "timing": f"graph replay, L2 flushed, median of {reps}"}
        return res, out, st, shapes
    finally:
        dem.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--diffusion-frames", type=int, default=500)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    args = ap.parse_args()
    # the frames are generated before the first CUDA call, in spawned processes
    stack = diffusion_stack(args.diffusion_frames, args.workers)
    uneven = synth.uneven_batch()
    carriers = {f0: synth.peaks_frame(20.0, f0) for f0 in (0.08, 0.1, 0.15)}

    import torch

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res, out, st = run_diffusion(stack, flush)
    print(json.dumps(res), flush=True)
    del out, st
    res, out, st, _ = run_uneven(uneven, flush)
    print(json.dumps(res), flush=True)

    # carrier frequencies of the 1024^2 peaks workload
    for f0, fr in carriers.items():
        dem = rmusic.Demodulator(precision="batched", carrier_freq=f0, use_graph=1, timing=1, autotune=1)
        x = torch.from_numpy(fr.image).cuda()
        ms, out, st, shapes, stats = time_call(dem, x, None, flush)
        print(json.dumps({"workload": f"peaks 1024x1024 float32, carrier {f0}, 20 dB, N=32, L=8",
                          "mpixel_per_s": fr.image.size / ms / 1e3, "ms_per_call": ms,
                          "solver_ms": stats.solver_ms, "bandpass_ms": stats.bandpass_ms}), flush=True)
        dem.close()


if __name__ == "__main__":
    main()
