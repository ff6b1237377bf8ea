"""Serving measurement: camera streams with Poisson frame arrivals fed through the serving loop
(``include/rmusic_serve.h``); reports per-frame latency percentiles beside throughput.

Default workload: 16 streams, 2000 frames/s in total, each stream a fixed frame size drawn from
512^2 .. 2048^2 (uint16, 12-bit), a free-diffusion phase front with its own Dt schedule, HBM budget
64 GB, 10 s. Each stream cycles through a small pool of pre-generated frames (the generator is far
slower than the GPU). Frames whose stream has no free slot at arrival are counted as rejected
(back-pressure), not queued on the host.

    python -m paper_1910_11872_gb300.serve_bench [--streams 16] [--rate 2000] [--seconds 10]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import rmusic, serve, synth

SIZES = (512, 1024, 1536, 2048)


def _stream_frame(job):
    t, side, s = job
    return synth.diffusion_frame(t, H=side, W=side, seed_index=4 + 100 * s).image


def make_streams(n: int, pool: int, seed: int = 11876, workers: int = 0):
    """Per stream: (H, W, pinned uint16 frames (pool x H x W)). The frames are drawn in spawned
    processes (the same seeded frames as drawing them one by one)."""
    import multiprocessing as mp
    import os

    import torch

    rng = np.random.default_rng(seed)
    jobs, sides = [], []
    for s in range(n):
        side = int(rng.choice(SIZES))
        sides.append(side)
        for k in range(pool):
            jobs.append((int(rng.integers(0, 500)), side, s))
    workers = workers or min(16, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(workers) as p:
        imgs = p.map(_stream_frame, jobs)
    out = []
    for s in range(n):
        stack = torch.from_numpy(np.stack(imgs[s * pool:(s + 1) * pool]).view(np.int16)).pin_memory()
        out.append((sides[s], sides[s], stack))
    return out


def run(args) -> dict:
    import torch

    streams = make_streams(args.streams, args.pool)
    cfg = serve.make_config(max_streams=args.streams, ring_depth=args.ring_depth,
                            max_batch_frames=args.max_batch_frames, inflight_batches=args.inflight,
                            max_batch_pixels=args.max_batch_mpx << 20, hbm_budget_bytes=int(args.budget_gb * (1 << 30)))
    srv = serve.Server(device=args.device, cfg=cfg, window_len=32, cov_order=8, deriv_axis=1, carrier_freq=0.1)
    try:
        ids, outs, free = [], [], []
        for H, W, _ in streams:
            ids.append(srv.open_stream(H, W, rmusic.RMUSIC_DTYPE_U16))
            outs.append([torch.empty(H * W, dtype=torch.float32).pin_memory() for _ in range(args.ring_depth)])
            free.append(list(range(args.ring_depth)))
        # Poisson arrivals, rate / streams per stream
        rng = np.random.default_rng(7)
        lam = args.rate / args.streams
        events = []
        for s in range(args.streams):
            t = rng.exponential(1.0 / lam)
            while t < args.seconds:
                events.append((t, s))
                t += rng.exponential(1.0 / lam)
        events.sort()
        submitted = rejected = 0
        px_submitted = 0
        lat, done_px = [], 0
        counter = [0] * args.streams

        def drain(timeout_ms=0):
            nonlocal done_px
            for c in srv.poll(1024, timeout_ms):
                s, slot = divmod(int(c.tag), 1 << 16)
                free[s].append(slot)
                lat.append(c.t_done - c.t_submit)
                done_px += streams[s][0] * streams[s][1]

        t0 = time.perf_counter()
        for t, s in events:
            while True:
                now = time.perf_counter() - t0
                if now >= t:
                    break
                drain(0)
                if t - now > 2e-4:
                    time.sleep(min(t - now, 1e-3))
            drain(0)
            H, W, stack = streams[s]
            if not free[s]:
                rejected += 1
                continue
            slot = free[s].pop()
            frame = stack[counter[s] % stack.shape[0]]
            counter[s] += 1
            rc = srv.submit(ids[s], frame.data_ptr(), outs[s][slot].data_ptr(), None, s * (1 << 16) + slot)
            if rc == rmusic.RMUSIC_EAGAIN:
                free[s].append(slot)
                rejected += 1
                continue
            submitted += 1
            px_submitted += H * W
        while len(lat) < submitted:
            drain(100)
        wall = time.perf_counter() - t0
        st = srv.stats()
        lat_ms = np.array(lat) * 1e3
        return {
            "metric": "serving: per-frame latency and throughput of root-MUSIC phase-derivative maps",
            "streams": args.streams, "offered_frames_per_s": args.rate, "seconds": args.seconds,
            "frames_offered": len(events), "frames_done": len(lat), "frames_rejected": rejected,
            "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                           "max": float(lat_ms.max()), "mean": float(lat_ms.mean())},
            "throughput_mpx_s": done_px / wall / 1e6, "offered_mpx_s": sum(
                streams[s][0] * streams[s][1] for _, s in events) / args.seconds / 1e6,
            "frames_per_s": len(lat) / wall, "batches": int(st.batches),
            "mean_batch_frames": float(st.frames_done / max(st.batches, 1)),
            "device_bytes": int(st.device_bytes), "hbm_budget_bytes": int(cfg.hbm_budget_bytes),
            "config": {"ring_depth": args.ring_depth, "max_batch_frames": args.max_batch_frames,
                       "inflight_batches": args.inflight, "sizes": list(SIZES), "dtype": "u16 12-bit",
                       "N": 32, "L": 8, "deriv_axis": "y"},
        }
    finally:
        srv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=16)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--pool", type=int, default=2)
    ap.add_argument("--ring-depth", type=int, default=4)
    ap.add_argument("--max-batch-frames", type=int, default=32)
    ap.add_argument("--max-batch-mpx", type=int, default=32)
    ap.add_argument("--inflight", type=int, default=3)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--device", type=int, default=0)
    print(json.dumps(run(ap.parse_args())), flush=True)


if __name__ == "__main__":
    main()
