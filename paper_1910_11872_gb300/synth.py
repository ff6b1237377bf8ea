"""Seeded synthetic fringe stacks shaped like the paper's workloads.

This module only draws inputs: carrier fringes I = a + b cos(2 pi f0 x + phi) with a phase map
phi, additive Gaussian noise and optional 12-bit quantisation, plus the closed-form derivative of
each phase map (the ground truth the accuracy checks compare against). It holds none of the
demodulation arithmetic; both the CUDA path's tests and the oracle's tests take their inputs
from here.

The phase models follow the paper's setting: a time-lapse stack of carrier fringes (Sec. 2) and
free diffusion, whose concentration profile is an erfc of y / (2 sqrt(D t)) (Appendix, Eq. 16).
The paper's own simulation phase map and its experimental frames are not available; these are
stand-ins with the stated shapes, sizes and noise levels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 11872


def rng_for(index: int) -> np.random.Generator:
    """PCG64 generator for workload ``index`` (0-based), seeded 11872 + index."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


def sigma_for_snr(b: float, snr_db: float) -> float:
    """Noise std for SNR(dB) = 10 log10((b^2/2) / sigma^2), the AC power of the real fringe."""
    if not np.isfinite(snr_db):
        return 0.0
    return math.sqrt((b * b / 2.0) / (10.0 ** (snr_db / 10.0)))


def fringe(phi: np.ndarray, f0: float, a: float = 0.5, b: float = 0.4, carrier_axis: int = 0,
           gy: float = 0.0) -> np.ndarray:
    """I = a + b cos(2 pi f0 t + 2 pi gy s + phi), t along ``carrier_axis`` (float64)."""
    H, W = phi.shape
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    t, s = (x, y) if carrier_axis == 0 else (y, x)
    return a + b * np.cos(2.0 * np.pi * f0 * t + 2.0 * np.pi * gy * s + phi)


def add_noise(img: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    if sigma <= 0:
        return img
    return img + rng.normal(0.0, sigma, size=img.shape)


def quantize12(img: np.ndarray) -> np.ndarray:
    """12-bit camera code round(4095 * clip(I, 0, 1)) stored as uint16."""
    return np.round(4095.0 * np.clip(img, 0.0, 1.0)).astype(np.uint16)


# ------------------------------------------------------------------------------------------
# Phase maps and their closed-form derivatives
# ------------------------------------------------------------------------------------------
def gaussian_bump(H: int, W: int, amp: float = 3.0, cx: float = 64.0, cy: float = 64.0,
                  s: float = 20.0):
    """phi = amp exp(-((x-cx)^2 + (y-cy)^2) / (2 s^2)); returns (phi, dphi/dx, dphi/dy)."""
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    g = amp * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * s * s))
    return g, -(x - cx) / (s * s) * g, -(y - cy) / (s * s) * g


def peaks(H: int, W: int, lo: float = 0.0, hi: float = 10.0):
    """MATLAB-style peaks surface on X, Y in [-3, 3], min-max scaled to [lo, hi] rad.

    Returns (phi, dphi/dx, dphi/dy) per pixel."""
    X = np.linspace(-3.0, 3.0, W)[None, :]
    Y = np.linspace(-3.0, 3.0, H)[:, None]
    e1 = np.exp(-X ** 2 - (Y + 1) ** 2)
    e2 = np.exp(-X ** 2 - Y ** 2)
    e3 = np.exp(-(X + 1) ** 2 - Y ** 2)
    p = 3 * (1 - X) ** 2 * e1 - 10 * (X / 5 - X ** 3 - Y ** 5) * e2 - e3 / 3.0
    dpx = (3 * e1 * (-2 * (1 - X) - 2 * X * (1 - X) ** 2)
           - 10 * e2 * ((0.2 - 3 * X ** 2) - 2 * X * (X / 5 - X ** 3 - Y ** 5))
           + (2.0 / 3.0) * (X + 1) * e3)
    dpy = (3 * (1 - X) ** 2 * e1 * (-2 * (Y + 1))
           - 10 * e2 * (-5 * Y ** 4 - 2 * Y * (X / 5 - X ** 3 - Y ** 5))
           + (2.0 / 3.0) * Y * e3)
    pmin, pmax = p.min(), p.max()
    k = (hi - lo) / (pmax - pmin)
    phi = lo + k * (p - pmin)
    return phi, k * dpx * (6.0 / (W - 1)), k * dpy * (6.0 / (H - 1))


def erfc_front(H: int, W: int, amp: float, Dt: float, y0: float):
    """Free-diffusion phase phi = amp erfc((y - y0) / (2 sqrt(Dt))) (Appendix, Eq. 16).

    Returns (phi, dphi/dx = 0, dphi/dy = -amp exp(-u^2) / sqrt(pi Dt))."""
    from scipy.special import erfc

    y = np.arange(H, dtype=np.float64)[:, None] * np.ones((1, W))
    u = (y - y0) / (2.0 * math.sqrt(Dt))
    phi = amp * erfc(u)
    dy = -amp * np.exp(-u * u) / math.sqrt(math.pi * Dt)
    return phi, np.zeros_like(phi), dy


def gaussian_sum(rng: np.random.Generator, H: int, W: int, n: int = 5, hi: float = 12.0,
                 max_grad: float = 0.25):
    """Sum of n random Gaussians, min-max scaled to [0, hi] rad, shrunk if max|grad| > max_grad."""
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    m = min(H, W)
    phi = np.zeros((H, W))
    gx = np.zeros((H, W))
    gy = np.zeros((H, W))
    for _ in range(n):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        s = rng.uniform(m / 8.0, m / 4.0)
        a = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 1.0)
        g = a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
        phi += g
        gx += -(x - cx) / (s * s) * g
        gy += -(y - cy) / (s * s) * g
    lo, hi_ = phi.min(), phi.max()
    k = hi / (hi_ - lo) if hi_ > lo else 0.0
    gmax = k * max(np.abs(gx).max(), np.abs(gy).max())
    if gmax > max_grad:
        k *= max_grad / gmax
    return k * (phi - lo), k * gx, k * gy


# ------------------------------------------------------------------------------------------
# Workloads
# ------------------------------------------------------------------------------------------
@dataclass
class Frame:
    """One synthetic frame and the parameters it is meant to be demodulated with."""

    image: np.ndarray                    # float32, uint16 (12-bit) or complex64, H x W
    carrier_freq: float
    deriv_axis: int = 0
    carrier_axis: int = 0
    window_len: int = 32
    cov_order: int = 8
    truth: np.ndarray | None = None      # closed-form derivative along deriv_axis (rad/px)
    meta: dict = field(default_factory=dict)


def small_gaussian_frame(sigma: float = 0.02, H: int = 128, W: int = 128, seed_index: int = 0) -> Frame:
    """128 x 128 float32, I = 0.5 + 0.4 cos(2 pi 0.1 x + phi), phi a 3-rad Gaussian bump of
    std 20 px at (64, 64), Gaussian noise sigma = 0.02; N = 32, L = 8, derivative along x."""
    rng = rng_for(seed_index)
    phi, dx, _ = gaussian_bump(H, W, 3.0, W / 2.0, H / 2.0, 20.0)
    img = add_noise(fringe(phi, 0.1), sigma, rng).astype(np.float32)
    return Frame(img, 0.1, truth=dx, meta={"workload": f"gaussian-bump {H}x{W} sigma={sigma}"})


def periodic_linear_frame(H: int = 16, W: int = 128, f: float = 16 / 128, f0: float = 0.1,
                          gy: float = 0.0, deriv_axis: int = 0, phase0: float = 0.3) -> Frame:
    """Noise-free fringe with a whole number of carrier periods per line (W f integer) and an
    optional linear phase ramp 2 pi gy y: its analytic signal is one exact complex exponential."""
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = 0.5 + 0.4 * np.cos(2 * np.pi * f * x + 2 * np.pi * gy * y + phase0)
    truth = np.full((H, W), 2 * np.pi * (f - f0) if deriv_axis == 0 else 2 * np.pi * gy)
    return Frame(img.astype(np.float32), f0, deriv_axis=deriv_axis, truth=truth,
                 meta={"workload": f"periodic-linear {H}x{W} f={f} gy={gy}"})


def peaks_frame(snr_db: float, f0: float = 0.1, H: int = 1024, W: int = 1024,
                seed_index: int = 1, stream: int = 0) -> Frame:
    """Single frame, float32, carrier f0, phi = peaks scaled to 0-10 rad, SNR in dB (inf = clean)."""
    rng = np.random.Generator(np.random.PCG64([SEED_BASE + seed_index, stream]))
    phi, dx, _ = peaks(H, W)
    img = add_noise(fringe(phi, f0), sigma_for_snr(0.4, snr_db), rng).astype(np.float32)
    return Frame(img, f0, truth=dx, meta={"workload": f"peaks {H}x{W} f0={f0} snr={snr_db}dB"})


def raw_fringe_frame(snr_db: float, offset_amp: float = 0.0, f0: float = 0.1, H: int = 1024, W: int = 1024,
                     seed_index: int = 6, stream: int = 0) -> Frame:
    """Real fringe for model order p > 1 on raw lines: 0.5 + offset_amp sin(x / 60) + 0.4 cos(2 pi f0 x
    + phi), phi = peaks scaled to 0-10 rad (the local offset varies along the line: the third
    exponential, at zero frequency, of p = 3), noise at snr_db. float32; truth is dphi/dx."""
    rng = np.random.Generator(np.random.PCG64([SEED_BASE + seed_index, stream]))
    phi, dx, _ = peaks(H, W)
    x = np.arange(W, dtype=np.float64)[None, :]
    img = add_noise(fringe(phi, f0) + offset_amp * np.sin(x / 60.0), sigma_for_snr(0.4, snr_db), rng)
    return Frame(img.astype(np.float32), f0, truth=dx,
                 meta={"workload": f"raw fringe {H}x{W} f0={f0} offset={offset_amp} snr={snr_db}dB"})


def diffusion_frame(t: int, T: int = 500, H: int = 1024, W: int = 1024, seed_index: int = 2,
                    amp: float = 8.0, dt0: float = 400.0, dt1: float = 40000.0,
                    sigma: float = 0.01) -> Frame:
    """Frame t of the diffusion time-lapse: uint16 12-bit, carrier 0.1 along x,
    phi(y, t) = amp erfc((y - H/2) / (2 sqrt(Dt))), Dt linear from dt0 to dt1 over T frames,
    noise 1 % of full scale. The derivative is taken along y (column windows)."""
    rng = np.random.Generator(np.random.PCG64([SEED_BASE + seed_index, t]))
    Dt = dt0 + (dt1 - dt0) * (t / max(T - 1, 1))
    phi, _, dy = erfc_front(H, W, amp, Dt, H / 2.0)
    img = quantize12(add_noise(fringe(phi, 0.1), sigma, rng))
    return Frame(img, 0.1, deriv_axis=1, truth=dy,
                 meta={"workload": f"diffusion t={t}/{T} {H}x{W} Dt={Dt:.1f}"})


def complex_fringe_frame(snr_db: float = 0.0, H: int = 512, W: int = 512, hi: float = 10.0, f0: float = 0.0,
                         seed_index: int = 5, stream: int = 0) -> Frame:
    """Complex fringe A exp(j(2 pi f0 x + phi)) + circular complex Gaussian noise, as the paper
    simulates it (Sec. 4: a 512 x 512 complex fringe at 0 dB), complex64. A = 1 and
    SNR(dB) = 10 log10(A^2 / E|noise|^2); phi = peaks scaled to 0 .. hi rad (the paper's own map is
    not given). truth is dphi/dx; meta holds dphi/dy and phi."""
    rng = np.random.Generator(np.random.PCG64([SEED_BASE + seed_index, stream]))
    phi, dx, dy = peaks(H, W, 0.0, hi)
    x = np.arange(W, dtype=np.float64)[None, :]
    g = np.exp(1j * (2.0 * math.pi * f0 * x + phi))
    if math.isfinite(snr_db):
        s = math.sqrt(0.5 * 10.0 ** (-snr_db / 10.0))
        g = g + s * (rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W)))
    return Frame(g.astype(np.complex64), f0, truth=dx,
                 meta={"workload": f"complex peaks {H}x{W} 0-{hi} rad snr={snr_db}dB", "truth_dy": dy, "phi": phi})


UNEVEN_HEIGHTS = (256, 512, 768, 1024, 2048)
UNEVEN_WIDTHS = (256, 512, 1024)
UNEVEN_WINDOWS = ((24, 6), (24, 8), (24, 12), (32, 6), (32, 8), (32, 12), (48, 6), (48, 8), (48, 12))


def uneven_batch(n: int = 64, seed_index: int = 3, snr_db: float = 15.0, f0: float = 0.1,
                 scale: float = 1.0) -> list[Frame]:
    """Frames of sizes drawn from {256..2048} x {256, 512, 1024} (optionally scaled down),
    phi a sum of 5 random Gaussians (0-12 rad), SNR 15 dB, (N, L) drawn from
    {24, 32, 48} x {6, 8, 12} with L <= N / 2."""
    rng = rng_for(seed_index)
    out = []
    for i in range(n):
        H = int(rng.choice(UNEVEN_HEIGHTS) * scale)
        W = int(rng.choice(UNEVEN_WIDTHS) * scale)
        N, L = UNEVEN_WINDOWS[int(rng.integers(len(UNEVEN_WINDOWS)))]
        phi, dx, _ = gaussian_sum(rng, H, W)
        img = add_noise(fringe(phi, f0), sigma_for_snr(0.4, snr_db), rng).astype(np.float32)
        out.append(Frame(img, f0, window_len=N, cov_order=L, truth=dx,
                         meta={"workload": f"uneven {H}x{W} N={N} L={L}"}))
    return out
