#!/usr/bin/env python3
"""Throughput of sliding-window root-MUSIC phase-derivative maps (arXiv:1910.11872) on GB300.

One step = the FP32-batched path over one batch of four 1024 x 1024 float32 fringe frames,
carrier 0.1 cycles/px, phase = peaks surface scaled to 0-10 rad, one frame per SNR of the sweep
40 / 20 / 10 / 5 dB; window N = 32, covariance order L = 8, forward-backward, derivative along x.

Printed: one JSON line (rank 0) with the device-timed value (inputs resident in HBM, L2 flushed
between steps), the end-to-end value through the host-buffer C entry point, the plain
thread-per-pixel path on the same GPU, the dominant kernel's roofline, the FP64 CPU oracle timed on
a bounded sample (and the element-wise error of the GPU maps against it), launch counts and the
SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs an independent replica (its own frames, no data exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1910_11872_gb300 import synth  # noqa: E402

METRIC = "Mpixel/s root-MUSIC phase-derivative, FP32-batched vs plain on same GB300"
SNRS = (40.0, 20.0, 10.0, 5.0)
H = W = 1024
F0 = 0.1
N_WIN, L_COV = 32, 8
WORKLOAD = (f"peaks phase 0-10 rad, {len(SNRS)} x {H}x{W} float32 frames per step (SNR 40/20/10/5 dB), "
            f"carrier {F0} cyc/px, N={N_WIN}, L={L_COV}, forward-backward, derivative along x")
# FP32 issue peak of the part: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz (maximum SM clock)
N_SM, FP32_LANES, MAX_SM_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = N_SM * FP32_LANES * 2 * MAX_SM_GHZ / 1e3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--plain-steps", type=int, default=10,
                    help="timed steps of the plain FP32 path (median reported)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-rows", type=int, default=512,
                    help="rows per frame in the oracle sample (about 10 s on 16 cores); an eighth of "
                         "them, of one frame, for the one-core figure")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forward-steps", type=int, default=5,
                    help="timed steps of the forward-only estimate on the main workload (0: skip)")
    ap.add_argument("--square-steps", type=int, default=5,
                    help="timed steps of the paper-geometry leg (square block, both derivatives and alpha)")
    ap.add_argument("--workloads", default=None,
                    help="comma-separated subset of the other workloads to run: gaussian, diffusion, uneven, "
                         "model_order, serving (default: all)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workloads (Gaussian-bump plain FP64, diffusion stack, uneven batch, serving)")
    ap.add_argument("--diffusion-frames", type=int, default=500)
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    return ap.parse_args()


def frames_for(rank: int):
    return [synth.peaks_frame(s, F0, H, W, stream=rank) for s in SNRS]


# The paper's own geometry and simulation setting (Sec. 3-4): a (2 Lp + 1)^2 block per pixel, Lp = 5,
# on a complex fringe at 0 dB; both derivatives and the local phase alpha per pixel.
SQ_LP, SQ_SNR, SQ_FRAMES = 5, 0.0, 4
SQ_WORKLOAD = (f"paper geometry: {SQ_FRAMES} x {H}x{W} complex64 fringes per step (peaks phase 0-10 rad, "
               f"SNR {SQ_SNR:g} dB), square block Lp={SQ_LP} (11x11), d/dx, d/dy and alpha per pixel")
# Table 2 of the paper (context only: other hardware, the full method including unwrapping)
PAPER_TABLE2_1024 = {"gpu": "Quadro M5000 (Maxwell, 16 SMs), FP32", "seconds_per_1024x1024_frame": 13.88,
                     "mpixel_per_s": 1024 * 1024 / 13.88 / 1e6}


def square_frames(rank: int):
    return [synth.complex_fringe_frame(SQ_SNR, H, W, 10.0, stream=100 * rank + i) for i in range(SQ_FRAMES)]


def aberth_flops(L: int, evals: float, updates: float) -> float:
    """Flops of the root stage (shared by both solvers) for one polynomial of half-size L, given the
    measured evaluations of Q and Q' and executed root updates: per evaluation Horner over 2L - 2
    steps (two complex multiply-adds, 16) and the residual test (4); per update Q/Q' (11), the
    2(L-1) - 1 reciprocal terms of the Aberth sum (10 each), the correction (21) and the mirror (8)."""
    NR, NI = 2 * L - 2, L - 1
    return evals * (16 * NR + 4) + updates * (11 + 10 * (2 * NI - 1) + 21 + 8)


def newton_flops(L: int) -> float:
    """One Newton step of the signal root (degree 2L - 2): Horner for Q and Q' (16 per step), the
    residual (4), the mirror and D = z - 1/conj(z) (8), Q D and Q' D - Q (14), one complex division
    (11), the update and the fold (6) and the tests (4)."""
    return 16 * (2 * L - 2) + 4 + 8 + 14 + 11 + 6 + 4


def schur_cohn_flops(L: int) -> float:
    """The Schur-Cohn count on Q(r z), n = 2L - 2: the scaled coefficients (3 per coefficient), then
    per level of degree d the two moduli (6), the reflection coefficient (9) and d complex
    multiply-subtracts (8 each), and the count."""
    n = 2 * L - 2
    return 3 * (n + 1) + sum(15 + 8 * d for d in range(1, n + 1)) + n


def rouche_flops(L: int) -> float:
    """The Rouche certificate of the selected root (degree n = 2L - 2): the rotation e^k and the
    rotated coefficients c_k e^k (2L - 3 complex products, 6 each), the division by the real
    quadratic (n - 1 steps: two multiply-adds and two subtractions, 6) with the weighted distance to
    the noise-free polynomial (difference, two magnitudes and the Horner step in rho, 5), the
    remainder and its bounds (20) and the table test (6)."""
    n = 2 * L - 2
    return 6 * (2 * L - 3) + 11 * (n - 1) + 26


def flops_per_pixel(L: int, N: int, sweeps: float, evals: float, updates: float, power_steps: float = 0.0,
                    eig_fallback: float = 0.0, newton: float = 0.0, root_fallback: float = 0.0,
                    polish: float = 2.0, pixels_per_lane: int = 16) -> float:
    """Algorithmic FP32 flops per pixel of the batched solver (FMA = 2, other arithmetic = 1),
    counted from the kernel's steps with the measured work per 32-pixel group (power steps,
    Jacobi sweeps and fallbacks, Newton steps, Aberth evaluations, updates and fallbacks):
      covariance  per rank-2 term: the folded snapshot (4 L adds) and X X^T + Y Y^T on the packed
                  triangle (L signs, 2 multiply-adds per entry); a lane of P pixels runs K terms for its
                  first pixel and 2 per further pixel, (K + 2 (P - 1)) / P per pixel; trace and scaling
      power it.   start column and Frobenius norm; per step S x (2 L^2), Rayleigh quotient, shift,
                  norm and the step size (10 L + 5)
      fallback    Jacobi: per rotation 14 + 6 (L - 2) + 4, L/2 rotations per step, L - 1 steps per
                  sweep, plus the off-diagonal norm L (L - 1); inverse iteration: L D L^T of
                  (mu I - S), two forward / diagonal / backward solves with norms
      polynomial  u = Q x (2 L), rho_k (8 flops per term), scaling and moduli
      roots       Newton steps (newton_flops), the Rouche certificate (rouche_flops; the Schur-Cohn
                  count that decides where it does not, measured in 0.2 % of the lanes of the bench
                  workload, is not counted); Aberth fallback: aberth_flops per executed evaluation and
                  update, starting points, selection
      polish      per measured step Horner on Q and Q' (16 per degree) and the deflated step (37);
                  angle (20); warps holding a split double root also form Q'' (not counted: rare on
                  noisy frames)
    """
    NS = L * (L + 1) // 2
    NR = 2 * L - 2
    NI = L - 1
    K, P = N - L + 1, pixels_per_lane
    cov = (K + 2 * (P - 1)) / P * (4 * L + L + 4 * NS) + L + NS + 1
    power = 2 * L + 3 * NS + 3 * L + 1 + power_steps * (2 * L * L + 10 * L + 5)
    rot = 14 + 6 * (L - 2) + 4
    jac = sweeps * ((L - 1) * (L // 2) * rot + L * (L - 1))
    ldl = sum(3 * j + 1 + (L - 1 - j) * (3 * j + 1) for j in range(L))
    inv = eig_fallback * (ldl + 2 * (2 * L * (L - 1) + 4 * L))
    coef = 2 * L + 3 * L + 4 * L * (L - 1) + 5 * (L - 1)
    roots = newton * newton_flops(L) + rouche_flops(L)
    aberth = aberth_flops(L, evals, updates) + root_fallback * (NI * 10 + 20 + 13 * NI)
    polish = polish * (16 * NR + 37) + 20
    return cov + power + jac + inv + coef + roots + aberth + polish


def square_flops_per_pixel(Lp: int, power_its: float, evals: float, updates: float, newton: float = 0.0,
                           root_fallback: float = 0.0, polish: float = 4.0, warm: float = 0.0) -> float:
    """Algorithmic FP32 flops per pixel of the square-block solver (block side M = 2 Lp + 1), from
    its steps with the measured power-iteration steps, Newton steps, Aberth evaluations, updates and
    fallbacks (the root figures add both polynomials):
      power it.   per step G^H u and G y (M^2 complex multiply-adds each, 8 flops), the norm (3 M),
                  normalisation and step size (8 M); the start vector (5 M); per measured warm start
                  (a row that starts from the row above's v1) G v (M^2 complex multiply-adds) and its
                  normalisation (5 M)
      polynomials per axis: |u|^2 (3 M), M (M - 1) / 2 lag products (8), scaling and moduli (8 per lag)
      roots       Newton steps (newton_flops) and per axis the Schur-Cohn certificate; Aberth fallback:
                  aberth_flops, starting points (10 per root + 20) and selection (13 per root)
      polish      per measured polish step (both axes together) Horner of degree 2M - 2 (16 per
                  degree) and the step (37); per axis the angle (20)
      alpha       four sincos (80), the recurrences (6 M), M^2 complex multiply-adds, M row terms
                  (16 M), angle and carrier phase (25)
    """
    M = 2 * Lp + 1
    NI, NR = M - 1, 2 * M - 2
    power = 5 * M + power_its * (16 * M * M + 11 * M) + warm * (8 * M * M + 5 * M)
    coefs = 2 * (3 * M + 4 * M * (M - 1) + 8 * (M - 1))
    roots = newton * newton_flops(M) + 2 * schur_cohn_flops(M)
    aberth = aberth_flops(M, evals, updates) + root_fallback * (10 * NI + 20 + 13 * NI)
    select = polish * (16 * NR + 37) + 2 * 20
    alpha = 80 + 6 * M + 8 * M * M + 16 * M + 25
    return power + coefs + roots + aberth + select + alpha


SOLVER_PROFILE = os.path.join(ROOT, "profiles", "batched_solver_L8_peaks4x1024.md")
SOLVER_SOURCES = ["batched_kernel.cuh", "roots_device.cuh", "rmusic_device.cuh", "rmusic_launch.h",
                  "batched_variants.h", "batched_l8.cu", "rouche_table.h"]
SQUARE_PROFILE = os.path.join(ROOT, "profiles", "square_solver_Lp5_complex4x1024.md")
SQUARE_SOURCES = ["square_kernel.cuh", "roots_device.cuh", "rmusic_device.cuh", "rmusic_launch.h",
                  "square_variants.h", "square_l5.cu", "rouche_table.h"]


def profiled_traffic(profile: str = SOLVER_PROFILE, sources=SOLVER_SOURCES):
    """DRAM bytes per solver launch from the committed ncu summary, or None when the solver's
    source has changed since those counters were taken (the summary records a hash of it)."""
    import hashlib
    import re

    if not os.path.exists(profile):
        return None
    text = open(profile).read()
    m_bytes = re.search(r"dram_bytes_per_launch = (\d+)", text)
    m_hash = re.search(r"source_sha256_16 = ([0-9a-f]{16})", text)
    if not m_bytes or not m_hash:
        return None
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_1910_11872_gb300", "csrc", f), "rb").read())
    return int(m_bytes.group(1)) if h.hexdigest()[:16] == m_hash.group(1) else None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)]
        return {"sm_mhz": statistics.median(busy or sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ----------------------------------------------------------------------------------------------
def oracle_sample(frames, rows_per_frame: int, nthreads: int = 0, fb: int = 1, seed: int = 11872):
    import oracle as O

    p = O.make_params(N_WIN, L_COV, fb, 0, 0, F0)
    rng = np.random.default_rng(seed)
    samples = []
    t0 = time.perf_counter()
    cores = 0
    npx = 0
    for fr in frames:
        rows = np.sort(rng.choice(H, rows_per_frame, replace=False))
        ys = np.repeat(rows, W).astype(np.int32)
        xs = np.tile(np.arange(W), rows_per_frame).astype(np.int32)
        vals, st, cores = O.demodulate_pixels(fr.image, p, ys, xs, nthreads)
        samples.append((ys, xs, vals, st))
        npx += ys.size
    dt = time.perf_counter() - t0
    return samples, npx, dt, cores


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O

    O.build()
    frames = frames_for(0)
    rows = max(1, args.cpu_rows // 4)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(frames[:1], 1)
    times, npx_step, cores = [], 0, 0
    for _ in range(args.steps):
        _, npx_step, dt, cores = oracle_sample(frames, rows)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = npx_step / (ms * 1e3)
    sample = f"{rows} random full rows of each of the {len(frames)} frames ({npx_step} px) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "oracle": "FP64 C, OpenMP over pixels"},
            "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
# GPU arms
# ----------------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1910_11872_gb300 import rmusic

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    frames = frames_for(rank)
    host = np.stack([f.image for f in frames]).astype(np.float32)
    x = torch.from_numpy(host).to(dev)
    npx = host.size
    out = torch.empty(npx, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # ---- FP32-batched path (persistent launch, CUDA graph) ------------------------------------
    # autotune: the first warm-up call times the solver's register-cap variants on these frames
    dem = rmusic.Demodulator(device=local, window_len=N_WIN, cov_order=L_COV, carrier_freq=F0,
                             precision="batched", use_graph=1, timing=1, autotune=1)
    for _ in range(args.warmup):
        dem.run(x, out=out, with_status=False)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    solver_ms, bandpass_ms, launches, sweeps, iters, updates, evals = [], [], 0, [], [], [], []
    psteps, eigfb, newton, rootfb, polish = [], [], [], [], []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        dem.run(x, out=out, with_status=False, stream=stream)
        ev[k][1].record(stream)
        st = dem.stats()  # waits for the call; reads the event-timed kernel durations
        solver_ms.append(st.solver_ms)
        bandpass_ms.append(st.bandpass_ms)
        launches += st.kernel_launches
        sweeps.append(st.mean_sweeps)
        iters.append(st.mean_root_iters)
        updates.append(st.mean_root_updates)
        evals.append(st.mean_root_evals)
        psteps.append(st.mean_power_steps)
        eigfb.append(st.eig_fallback_frac)
        newton.append(st.mean_newton_steps)
        rootfb.append(st.root_fallback_frac)
        polish.append(st.mean_polish_steps)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    step_ms_max = max_over_ranks(world, step_ms)
    value = npx * world / (step_ms_max * 1e3)
    # pixels whose window lies inside the frame: W - N + 1 positions per row (the others are
    # border pixels, NaN with status "border")
    npx_valid = len(frames) * H * (W - N_WIN + 1)
    result_gpu = out.view(len(frames), H, W).cpu().numpy()
    # every solver variant on the same frames (register caps and the warp-per-matrix schedule of
    # the eigenvalue sweeps), outside the timed region: the autotuner's choice, shown
    kept = st.solver_variant
    variants = []
    for v in range(4):
        rmusic.rmusic_set_solver_variant(dem.ctx, L_COV, v)
        dem.run(x, out=out, with_status=False, stream=stream)
        vms = []
        for _ in range(3):
            dem.run(x, out=out, with_status=False, stream=stream)
            sv = dem.stats()
            vms.append(sv.solver_ms)
        variants.append({"variant": v, "ctas_per_sm": sv.solver_ctas_per_sm,
                         "schedule": "warp per matrix" if v == 3 else "thread per matrix",
                         "solver_ms": statistics.mean(vms)})
    rmusic.rmusic_set_solver_variant(dem.ctx, L_COV, -1)
    # per-pixel outcomes of one step, outside the timed region (the timed steps skip the status map)
    sout, sst, _ = dem.run(x, with_status=True)
    torch.cuda.synchronize()
    st_np = sst.cpu().numpy()
    status_counts = {"ok": int((st_np == 0).sum()), "border": int((st_np == 1).sum()),
                     "degenerate": int((st_np == 2).sum()), "not_converged": int((st_np == 3).sum()),
                     "nan_values": int(torch.isnan(sout).sum().item())}
    del sout, sst

    # ---- plain path on the same GPU (thread per pixel, one launch per frame) -------------------
    plain = rmusic.Demodulator(device=local, window_len=N_WIN, cov_order=L_COV, carrier_freq=F0,
                               precision="plain_fp32", timing=1)
    for _ in range(3):  # warm-up
        plain.run(x, out=out, with_status=False)
    torch.cuda.synchronize()
    pms = []
    for _ in range(args.plain_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plain.run(x, out=out, with_status=False, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        pms.append(a.elapsed_time(b))
    plain_ms = max_over_ranks(world, statistics.median(pms))
    plain_value = npx * world / (plain_ms * 1e3)
    plain.close()

    # ---- end to end through the host-buffer entry points -----------------------------------------
    # Every step copies its frames from pinned host memory to the device and its maps back. The
    # asynchronous entry with two contexts on two streams (two calls in flight, each with its own
    # output buffer) is how a streaming caller uses the library: the copy engine moves one step's
    # frames while the other step's kernels run. The synchronous entry (one call at a time, frames
    # read in place by the band-pass) is reported beside it.
    hin = torch.from_numpy(host.reshape(-1)).pin_memory()
    houts = [torch.empty(npx, dtype=torch.float32).pin_memory() for _ in range(2)]
    descs, nbytes, nout = rmusic.frame_descs([(H, W)] * len(frames), rmusic.RMUSIC_DTYPE_F32, 4)
    e2e_dems = [rmusic.Demodulator(device=local, window_len=N_WIN, cov_order=L_COV, carrier_freq=F0,
                                   precision="batched", use_graph=1) for _ in range(2)]
    e2e_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]

    def e2e_async_step(k):
        i = k % 2
        e2e_streams[i].synchronize()  # this context's previous step is complete
        rmusic.rmusic_demodulate_frames_host_async(e2e_dems[i].ctx, hin.data_ptr(), nbytes, descs, len(frames),
                                                   houts[i].data_ptr(), None, e2e_streams[i].cuda_stream)

    for k in range(4):
        e2e_async_step(k)
    for st_ in e2e_streams:
        st_.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        e2e_async_step(k)
    for st_ in e2e_streams:
        st_.synchronize()
    e2e_ms = max_over_ranks(world, 1e3 * (time.perf_counter() - t0) / args.e2e_steps)
    e2e_launches = e2e_dems[0].stats().kernel_launches
    for d in e2e_dems:
        d.close()
    e2e_value = npx * world / (e2e_ms * 1e3)
    # the synchronous entry, one call at a time
    sdem = rmusic.Demodulator(device=local, window_len=N_WIN, cov_order=L_COV, carrier_freq=F0,
                              precision="batched", use_graph=1)
    for _ in range(2):
        rmusic.rmusic_demodulate_frames_host(sdem.ctx, hin.data_ptr(), nbytes, descs, len(frames),
                                             houts[0].data_ptr(), None, stream.cuda_stream)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        rmusic.rmusic_demodulate_frames_host(sdem.ctx, hin.data_ptr(), nbytes, descs, len(frames),
                                             houts[0].data_ptr(), None, stream.cuda_stream)
    e2e_sync_ms = max_over_ranks(world, 1e3 * (time.perf_counter() - t0) / args.e2e_steps)
    sdem.close()

    # ---- roofline of the dominant kernel (batched solver) ---------------------------------------
    fpp = flops_per_pixel(L_COV, N_WIN, statistics.mean(sweeps), statistics.mean(evals), statistics.mean(updates),
                          statistics.mean(psteps), statistics.mean(eigfb), statistics.mean(newton),
                          statistics.mean(rootfb), statistics.mean(polish))
    solver_avg = statistics.mean(solver_ms)
    achieved = fpp * npx / (solver_avg * 1e-3) / 1e12
    traffic = profiled_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "batched_kernel<8>", "flops_per_pixel": fpp, "launch_ms": solver_avg,
                "peak_note": "FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (unit counts and max clock)",
                "mean_power_steps": statistics.mean(psteps), "eig_fallback_frac": statistics.mean(eigfb),
                "mean_jacobi_sweeps": statistics.mean(sweeps), "mean_newton_steps": statistics.mean(newton),
                "mean_polish_steps": statistics.mean(polish),
                "root_fallback_frac": statistics.mean(rootfb), "mean_aberth_iters": statistics.mean(iters),
                "mean_aberth_updates": statistics.mean(updates), "mean_aberth_evals": statistics.mean(evals),
                "solver_ctas_per_sm": st.solver_ctas_per_sm, "solver_variant": kept,
                "solver_variants": variants,
                "bandpass_ms": statistics.mean(bandpass_ms)}

    fwd = (run_forward_leg(args, rank, world, dev, stream, flush, frames, x, step_ms_max)
           if args.forward_steps > 0 else None)
    sq = run_square_leg(args, rank, world, dev, stream, flush) if args.square_steps > 0 else None

    line = {"metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "valid_value": npx_valid * world / (step_ms_max * 1e3),
            "config": {"workload": WORKLOAD, "frames_per_step": len(frames), "pixels_per_step": npx,
                       "valid_pixels_per_step": npx_valid,
                       "l2": "flushed between steps (256 MiB write)", "cuda_graph": True,
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "Mpixel/s", "h2d_bytes_per_step": int(host.nbytes),
                    "d2h_bytes_per_step": int(npx * 4), "ms_per_step": e2e_ms, "kernels_per_step": e2e_launches,
                    "entry": "rmusic_demodulate_frames_host_async, two contexts double-buffered on two streams",
                    "sync": {"value": npx * world / (e2e_sync_ms * 1e3), "ms_per_step": e2e_sync_ms,
                             "entry": "rmusic_demodulate_frames_host, one call at a time"}},
            "gpu_launches": launches, "clocks": clk, "status_counts": status_counts,
            "plain": {"value": plain_value, "unit": "Mpixel/s", "ms_per_step": plain_ms,
                      "path": "plain FP32, thread per pixel, one launch per frame",
                      "timing": f"3 warm-ups, median of {args.plain_steps} event-timed steps, L2 flushed"},
            "speedup_vs_plain": value / plain_value}
    if fwd is not None:
        line["forward_estimate"] = fwd
    if sq is not None:
        line["paper_geometry"] = sq
    if not args.no_workloads:
        line["workloads"] = run_workloads(args, dev, stream, flush,
                                          cpu=rank == 0 and world == 1 and not args.no_cpu_baseline)

    # ---- CPU oracle on a bounded sample, and the GPU error against it -----------------------
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        samples, n_or, dt, cores = oracle_sample(frames, args.cpu_rows)
        # the same oracle on one core (the paper's sequential baseline), on a smaller sample
        rows1 = max(1, args.cpu_rows // 8)
        _, n1, dt1, _ = oracle_sample(frames[:1], rows1, nthreads=1)
        line["cpu_baseline"] = {"value": n_or / dt / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_rows} random full rows of each frame ({n_or} px), "
                                          f"{dt:.1f} s wall",
                                "per_core": n_or / dt / 1e6 / max(cores, 1),
                                "one_core": {"value": n1 / dt1 / 1e6, "unit": "Mpixel/s",
                                             "sample": f"{rows1} random full rows of the 40 dB frame ({n1} px), "
                                                       f"{dt1:.1f} s wall"},
                                "host": f"{platform.machine()}, {os.cpu_count()} logical CPUs"}
        acc = {}
        for snr, fr, g, (ys, xs, vals, st) in zip(SNRS, frames, result_gpu, samples):
            gv = g[ys, xs].astype(np.float64)
            ok = (st == 0) & np.isfinite(gv)
            d = np.abs(gv[ok] - vals[ok])
            inner = ok & (xs >= 32) & (xs < W - 32)
            rms_o = float(np.sqrt(np.mean((vals[inner] - fr.truth[ys[inner], xs[inner]]) ** 2)))
            rms_g = float(np.sqrt(np.mean((gv[inner] - fr.truth[ys[inner], xs[inner]]) ** 2)))
            acc[f"{int(snr)}dB"] = {"max_abs_rad_px": float(d.max()), "p999_rad_px": float(np.quantile(d, 0.999)),
                                    "rms_vs_truth_gpu": rms_g, "rms_vs_truth_oracle": rms_o,
                                    "rms_rel_diff": abs(rms_g - rms_o) / rms_o}
        line["accuracy_vs_fp64_oracle"] = acc
    dem.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_forward_leg(args, rank, world, dev, stream, flush, frames, x, fb_step_ms):
    """The same workload on the forward estimate R = R_f alone (forward_backward = 0; Sec. 3, Eq. 4-5),
    timed like the main leg (graph replay, L2 flushed between steps, CUDA events), with the error of
    its maps against the oracle's forward estimate on a bounded sample; reported beside the main line."""
    import torch

    from paper_1910_11872_gb300 import rmusic

    npx = x.numel()
    out = torch.empty(npx, dtype=torch.float32, device=dev)
    dem = rmusic.Demodulator(device=dev.index, window_len=N_WIN, cov_order=L_COV, carrier_freq=F0,
                             forward_backward=0, precision="batched", use_graph=1, timing=1, autotune=1)
    for _ in range(args.warmup):
        dem.run(x, out=out, with_status=False)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(dev.index)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.forward_steps)]
    solver_ms, psteps, eigfb, newton, rootfb, launches = [], [], [], [], [], 0
    for k in range(args.forward_steps):
        flush.zero_()
        ev[k][0].record(stream)
        dem.run(x, out=out, with_status=False, stream=stream)
        ev[k][1].record(stream)
        st = dem.stats()
        solver_ms.append(st.solver_ms)
        psteps.append(st.mean_power_steps)
        eigfb.append(st.eig_fallback_frac)
        newton.append(st.mean_newton_steps)
        rootfb.append(st.root_fallback_frac)
        launches += st.kernel_launches
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = max_over_ranks(world, statistics.mean(a.elapsed_time(b) for a, b in ev))
    res = {"workload": WORKLOAD.replace("forward-backward", "forward estimate only"),
           "value": npx * world / (step_ms * 1e3), "unit": "Mpixel/s", "ms_per_step": step_ms,
           "steps": args.forward_steps, "gpu_launches": launches, "clocks": clk,
           "kernel": f"batched_fwd_kernel<{L_COV}, {st.solver_ctas_per_sm}>",
           "solver_ms": statistics.mean(solver_ms), "mean_power_steps": statistics.mean(psteps),
           "eig_fallback_frac": statistics.mean(eigfb), "mean_newton_steps": statistics.mean(newton),
           "root_fallback_frac": statistics.mean(rootfb),
           "time_vs_forward_backward": step_ms / fb_step_ms,
           "timing": "graph replay, L2 flushed between steps, CUDA events on the launching stream"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sout, sst, _ = dem.run(x, with_status=True)
        torch.cuda.synchronize()
        g_all = sout.view(len(frames), H, W).cpu().numpy()
        s_all = sst.view(len(frames), H, W).cpu().numpy()
        rows = max(1, args.cpu_rows // 8)
        samples, n_or, dt, cores = oracle_sample(frames, rows, fb=0, seed=11873)
        acc = {}
        for snr, fr, g, s_, (ys, xs, vals, ost) in zip(SNRS, frames, g_all, s_all, samples):
            acc[f"{int(snr)}dB"] = _oracle_compare(g[ys, xs], s_[ys, xs], vals, ost, fr.truth[ys, xs])
        res["accuracy_vs_fp64_oracle"] = acc
        res["cpu_baseline"] = {"value": n_or / dt / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                               "sample": f"{rows} random full rows of each frame ({n_or} px), {dt:.1f} s wall"}
    dem.close()
    return res


def run_square_leg(args, rank, world, dev, stream, flush):
    """The paper's square-block geometry on its simulation setting, timed like the main leg
    (graph replay, L2 flushed between steps, CUDA events); reported beside the main line."""
    import torch

    from paper_1910_11872_gb300 import rmusic

    frames = square_frames(rank)
    host = np.stack([f.image for f in frames])
    x = torch.from_numpy(host).to(dev)
    npx = host.shape[0] * host.shape[1] * host.shape[2]
    out = torch.empty(3 * npx, dtype=torch.float32, device=dev)
    dem = rmusic.Demodulator(device=dev.index, geometry="square", half_width=SQ_LP, carrier_freq=0.0,
                             precision="batched", use_graph=1, timing=1, autotune=1)
    for _ in range(args.warmup):
        dem.run(x, out=out, with_status=False)
    torch.cuda.synchronize()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.square_steps)]
    solver_ms, its, evals, updates, launches, newton, rootfb, polish, warm = [], [], [], [], 0, [], [], [], []
    for k in range(args.square_steps):
        flush.zero_()
        ev[k][0].record(stream)
        dem.run(x, out=out, with_status=False, stream=stream)
        ev[k][1].record(stream)
        st = dem.stats()
        solver_ms.append(st.solver_ms)
        its.append(st.mean_sweeps)
        evals.append(st.mean_root_evals)
        updates.append(st.mean_root_updates)
        newton.append(st.mean_newton_steps)
        rootfb.append(st.root_fallback_frac)
        polish.append(st.mean_polish_steps)
        warm.append(st.mean_power_steps)  # square geometry: warm starts per 32-pixel group
        launches += st.kernel_launches
    torch.cuda.synchronize()
    step_ms = max_over_ranks(world, statistics.mean(a.elapsed_time(b) for a, b in ev))
    value = npx * world / (step_ms * 1e3)
    fpp = square_flops_per_pixel(SQ_LP, statistics.mean(its), statistics.mean(evals), statistics.mean(updates),
                                 statistics.mean(newton), statistics.mean(rootfb), statistics.mean(polish),
                                 statistics.mean(warm))
    solver_avg = statistics.mean(solver_ms)
    achieved = fpp * npx / (solver_avg * 1e-3) / 1e12
    res = {"workload": SQ_WORKLOAD, "value": value, "unit": "Mpixel/s", "ms_per_step": step_ms,
           "steps": args.square_steps, "gpu_launches": launches,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP32_PEAK_TFLOPS,
                        "traffic": profiled_traffic(SQUARE_PROFILE, SQUARE_SOURCES),
                        "kernel": f"square_kernel<{SQ_LP}, {st.solver_ctas_per_sm}>", "flops_per_pixel": fpp,
                        "launch_ms": solver_avg, "mean_power_iters": statistics.mean(its),
                        "mean_newton_steps": statistics.mean(newton), "root_fallback_frac": statistics.mean(rootfb),
                        "mean_polish_steps": statistics.mean(polish), "warm_start_frac": statistics.mean(warm),
                        "mean_aberth_evals": statistics.mean(evals), "mean_aberth_updates": statistics.mean(updates)},
           "paper_table2_context": PAPER_TABLE2_1024}

    # the paper's full method: the same call with phase assembly (the alpha maps unwrapped into a
    # fourth map by the reliability-sorting method, Sec. 3)
    out4 = torch.empty(4 * npx, dtype=torch.float32, device=dev)
    full = rmusic.Demodulator(device=dev.index, geometry="square", half_width=SQ_LP, carrier_freq=0.0,
                              precision="batched", use_graph=1, unwrap=1)
    for _ in range(args.warmup):
        full.run(x, out=out4, with_status=False)
    torch.cuda.synchronize()
    fms = []
    for _ in range(args.square_steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        full.run(x, out=out4, with_status=False, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        fms.append(a0.elapsed_time(a1))
    full_ms = max_over_ranks(world, statistics.mean(fms))
    res["with_phase_assembly"] = {"value": npx * world / (full_ms * 1e3), "unit": "Mpixel/s", "ms_per_step": full_ms,
                                  "unwrap_ms": full_ms - step_ms, "gpu_launches": full.stats().kernel_launches,
                                  "speedup_vs_paper_table2": (npx * world / (full_ms * 1e3))
                                  / PAPER_TABLE2_1024["mpixel_per_s"]}
    full.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O

        maps = out.view(len(frames), 3, H, W).cpu().numpy()
        rng = np.random.default_rng(5)
        worst = {"dx": 0.0, "dy": 0.0, "alpha": 0.0}
        for f, m in zip(frames, maps):
            ys, xs = rng.integers(0, H, 256), rng.integers(0, W, 256)
            odx, ody, oal, ost, _ = O.square_demodulate_pixels(f.image, O.make_params(carrier_freq=0.0), SQ_LP, ys, xs)
            ok = ost == 0
            for key, g, o in (("dx", m[0], odx), ("dy", m[1], ody), ("alpha", m[2], oal)):
                d = np.abs((g[ys, xs][ok] - o[ok] + np.pi) % (2 * np.pi) - np.pi)
                worst[key] = max(worst[key], float(d.max()))
        res["max_abs_vs_fp64_oracle"] = worst
        res["oracle_sample"] = f"256 random pixels of each frame ({256 * len(frames)} px)"
    dem.close()
    return res


# ----------------------------------------------------------------------------------------------
# The other workloads: Gaussian bump (plain FP64 vs the oracle), diffusion stack, uneven batch,
# serving. Each is timed on the GPU with its own clock record; the oracle is timed on a bounded
# sample of each and gives the GPU maps' error on that sample.
# ----------------------------------------------------------------------------------------------
def _oracle_compare(g, s, vals, st, truth=None):
    """Agreement of GPU values/statuses with the oracle's on the same pixels."""
    g = np.asarray(g, dtype=np.float64)
    both = (st == 0) & (s == 0)
    d = np.abs((g[both] - vals[both] + np.pi) % (2 * np.pi) - np.pi)
    res = {"pixels": int(st.size), "status_equal": bool(np.array_equal(s, st)),
           "status_differ": int((s != st).sum()), "max_abs_rad_px": float(d.max()) if d.size else 0.0,
           "p999_rad_px": float(np.quantile(d, 0.999)) if d.size else 0.0}
    if truth is not None and both.any():
        rms_o = float(np.sqrt(np.mean((vals[both] - truth[both]) ** 2)))
        rms_g = float(np.sqrt(np.mean((g[both] - truth[both]) ** 2)))
        res.update({"rms_vs_truth_gpu": rms_g, "rms_vs_truth_oracle": rms_o,
                    "rms_rel_diff": abs(rms_g - rms_o) / rms_o if rms_o > 0 else 0.0})
    return res


def run_workloads(args, dev, stream, flush, cpu: bool):
    import torch

    import oracle as O
    from paper_1910_11872_gb300 import config_bench, rmusic, serve_bench

    out = {}

    def want(name: str) -> bool:
        return args.workloads is None or name in args.workloads.split(",")

    if want("gaussian"):
        # ---- Gaussian bump 128 x 128: plain FP64 GPU path vs the FP64 oracle, whole frame --------
        fr = synth.small_gaussian_frame()
        x = torch.from_numpy(fr.image).to(dev)
        dem = rmusic.Demodulator(device=dev.index, precision="plain_fp64")
        clocks = ClockSampler(dev.index)
        clocks.start()
        for _ in range(3):
            g1, s1, _ = dem.run(x)
        ms = []
        for _ in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dem.run(x, out=g1, status=s1, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        clk = clocks.stop()
        dem.close()
        res = {"workload": "Gaussian bump 1 x 128x128 float32, noise 0.02, N=32, L=8, plain FP64 GPU path",
               "value": fr.image.size / statistics.median(ms) / 1e3, "unit": "Mpixel/s",
               "ms_per_call": statistics.median(ms), "timing": "3 warm-ups, median of 10 event-timed calls",
               "clocks": clk}
        if cpu:
            t0 = time.perf_counter()
            o, ost, cores = O.demodulate(fr.image, O.make_params(N_WIN, L_COV, 1, 0, 0, F0))
            dt = time.perf_counter() - t0
            res["vs_fp64_oracle"] = _oracle_compare(g1.cpu().numpy(), s1.cpu().numpy(), o.ravel(), ost.ravel())
            res["cpu_baseline"] = {"value": fr.image.size / dt / 1e6, "unit": "Mpixel/s", "cores": cores,
                                   "kind": "oracle", "sample": f"the whole frame ({fr.image.size} px), {dt:.2f} s wall"}
        out["gaussian_bump_plain_fp64"] = res
        del x, g1, s1

    if want("diffusion"):
        # ---- diffusion time-lapse: 500 x 1024^2 uint16 in one call, column windows ----------------
        stack = config_bench.diffusion_stack(args.diffusion_frames)
        clocks = ClockSampler(dev.index)
        clocks.start()
        res, dmaps, dst = config_bench.run_diffusion(stack, flush)
        res["clocks"] = clocks.stop()
        if cpu:
            rng = np.random.default_rng(11875)
            T = stack.shape[0]
            ts = sorted({0, T // 3, (2 * T) // 3, T - 1})
            comp, npx, dt, cores = [], 0, 0.0, 0
            p = O.make_params(N_WIN, L_COV, 1, 1, 0, F0)
            for t in ts:
                fr = synth.diffusion_frame(int(t), T=T)
                r0 = int(rng.integers(380, 580))
                rows = np.arange(r0, r0 + 64)  # 64 rows through the diffusion front, every column
                ys = np.repeat(rows, W).astype(np.int32)
                xs = np.tile(np.arange(W), rows.size).astype(np.int32)
                t0 = time.perf_counter()
                vals, st, cores = O.demodulate_pixels(fr.image, p, ys, xs)
                dt += time.perf_counter() - t0
                npx += ys.size
                g = dmaps[t].cpu().numpy()[ys, xs]
                s_ = dst[t].cpu().numpy()[ys, xs]
                comp.append((g, s_, vals, st, fr.truth[ys, xs]))
            cat = [np.concatenate([c[i] for c in comp]) for i in range(5)]
            res["vs_fp64_oracle"] = _oracle_compare(*cat)
            res["cpu_baseline"] = {"value": npx / dt / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                                   "sample": f"64 rows through the front, all columns, of frames {ts} ({npx} px), "
                                             f"{dt:.1f} s wall"}
        out["diffusion_stack"] = res
        del dmaps, dst, stack
        torch.cuda.empty_cache()

    if want("uneven"):
        # ---- uneven batch: 64 frames of uneven sizes and windows in one call ------------------------
        frames = synth.uneven_batch()
        clocks = ClockSampler(dev.index)
        clocks.start()
        res, umaps, ust, shapes = config_bench.run_uneven(frames, flush)
        res["clocks"] = clocks.stop()
        if cpu:
            rng = np.random.default_rng(11876)
            gm, sm = umaps.cpu().numpy(), ust.cpu().numpy()
            offs = np.cumsum([0] + [h * w for h, w in shapes])
            comp, npx, dt, cores = [], 0, 0.0, 0
            for i in sorted(rng.choice(len(frames), 8, replace=False)):
                fr = frames[i]
                Hf, Wf = fr.image.shape
                rows = np.sort(rng.choice(Hf, 16, replace=False))
                ys = np.repeat(rows, Wf).astype(np.int32)
                xs = np.tile(np.arange(Wf), rows.size).astype(np.int32)
                p = O.make_params(fr.window_len, fr.cov_order, 1, 0, 0, fr.carrier_freq)
                t0 = time.perf_counter()
                vals, st, cores = O.demodulate_pixels(fr.image, p, ys, xs)
                dt += time.perf_counter() - t0
                npx += ys.size
                g = gm[offs[i]:offs[i + 1]].reshape(Hf, Wf)[ys, xs]
                s_ = sm[offs[i]:offs[i + 1]].reshape(Hf, Wf)[ys, xs]
                comp.append((g, s_, vals, st, fr.truth[ys, xs]))
            cat = [np.concatenate([c[i] for c in comp]) for i in range(5)]
            res["vs_fp64_oracle"] = _oracle_compare(*cat)
            res["cpu_baseline"] = {"value": npx / dt / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                                   "sample": f"16 random full rows of each of 8 random frames ({npx} px), {dt:.1f} s wall"}
        out["uneven_batch"] = res
        del umaps, ust
        torch.cuda.empty_cache()

    if want("model_order"):
        # ---- model order p = 2 and 3 on raw real lines (Sec. 3 with p exponentials) -------------------
        res_p = {}
        for p, offset in ((2, 0.0), (3, 0.15)):
            frames_p = [synth.raw_fringe_frame(snr, offset, stream=k) for k, snr in enumerate(SNRS)]
            xp = torch.from_numpy(np.stack([f.image for f in frames_p])).to(dev)
            outp = torch.empty(xp.numel(), dtype=torch.float32, device=dev)
            kw = dict(device=dev.index, window_len=N_WIN, cov_order=L_COV, carrier_freq=F0, model_order=p, raw_input=1)
            demp = rmusic.Demodulator(precision="batched", use_graph=1, timing=1, **kw)
            clocks = ClockSampler(dev.index)
            clocks.start()
            for _ in range(3):
                demp.run(xp, out=outp, with_status=False)
            ms = []
            for _ in range(10):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                demp.run(xp, out=outp, with_status=False, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            st = demp.stats()
            clk = clocks.stop()
            gp, gps, _ = demp.run(xp)
            torch.cuda.synchronize()
            demp.close()
            plainp = rmusic.Demodulator(precision="plain_fp32", **kw)
            plainp.run(xp[:1])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plainp.run(xp[:1], stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            plain_ms = a.elapsed_time(b)
            plainp.close()
            npx_p = xp.numel()
            r = {"workload": f"{len(SNRS)} x {H}x{W} float32 raw real fringes (peaks phase 0-10 rad, SNR 40/20/10/5 dB"
                             f"{', local offset 0.15 sin(x/60)' if offset else ''}), carrier {F0}, N={N_WIN}, L={L_COV}, "
                             f"model order {p}, forward-backward",
                 "value": npx_p / statistics.median(ms) / 1e3, "unit": "Mpixel/s", "ms_per_call": statistics.median(ms),
                 "solver_ms": st.solver_ms, "mean_subspace_steps": st.mean_power_steps,
                 "jacobi_fallback_frac": st.eig_fallback_frac, "mean_aberth_iters": st.mean_root_iters,
                 "plain_fp32": {"value": H * W / plain_ms / 1e3, "unit": "Mpixel/s", "ms_one_frame": plain_ms},
                 "speedup_vs_plain": (npx_p / statistics.median(ms)) / (H * W / plain_ms),
                 "timing": "graph replay, L2 flushed, 3 warm-ups, median of 10 event-timed calls", "clocks": clk}
            if cpu:
                rng = np.random.default_rng(11877 + p)
                gm, sm = gp.view(len(frames_p), H, W).cpu().numpy(), gps.view(len(frames_p), H, W).cpu().numpy()
                comp, npx, dt, cores = [], 0, 0.0, 0
                prm = O.make_params(N_WIN, L_COV, 1, 0, 0, F0, model_order=p, raw_input=1)
                for fr, g_, s_ in zip(frames_p, gm, sm):
                    rows = np.sort(rng.choice(H, 8, replace=False))
                    ys = np.repeat(rows, W).astype(np.int32)
                    xs = np.tile(np.arange(W), rows.size).astype(np.int32)
                    t0 = time.perf_counter()
                    vals, ost, cores = O.demodulate_pixels(fr.image, prm, ys, xs)
                    dt += time.perf_counter() - t0
                    npx += ys.size
                    comp.append((g_[ys, xs], s_[ys, xs], vals, ost, fr.truth[ys, xs]))
                cat = [np.concatenate([c[i] for c in comp]) for i in range(5)]
                r["vs_fp64_oracle"] = _oracle_compare(*cat)
                r["cpu_baseline"] = {"value": npx / dt / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                                     "sample": f"8 random full rows of each frame ({npx} px), {dt:.1f} s wall"}
            res_p[f"p{p}"] = r
            del xp, outp, gp, gps
        out["model_order"] = res_p

    if want("serving"):
        # ---- serving: 16 camera streams, Poisson arrivals at 2000 frames/s ---------------------------
        sargs = argparse.Namespace(streams=16, rate=2000.0, seconds=args.serve_seconds, pool=2, ring_depth=4,
                                   max_batch_frames=32, max_batch_mpx=32, inflight=3, budget_gb=64.0, device=dev.index)
        clocks = ClockSampler(dev.index)
        clocks.start()
        res = serve_bench.run(sargs)
        res["clocks"] = clocks.stop()
        res["shed_frac"] = res["frames_rejected"] / max(res["frames_offered"], 1)
        out["serving"] = res

    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
