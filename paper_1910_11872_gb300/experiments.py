"""Accuracy experiments of the paper on synthetic stand-ins, run through the library's GPU path
(Sec. 4: the phase error of the method against the noise level, Fig. 4, and against the window
half-width L, Table 1).

The paper's simulated phase map is not given. The stand-in is a complex fringe exp(j phi) + noise
with phi the peaks surface scaled to 0 .. hi rad on a 512 x 512 frame (the paper's size); the
steepness hi sets the curvature that the local linear-phase model must absorb, which is what moves
the best window size (a small window is noise-limited, a large one model-limited). These errors are
reported on the pixels every window size leaves valid (8 pixels from each edge):
  * alpha_rmse   RMS of the wrapped difference between the local phase alpha (Eq. 15) and phi,
                 after removing the mean offset (the phase is defined up to a constant);
  * phase_rmse   RMS difference between the unwrapped phase map (phase assembly, Sec. 3) and phi
                 after removing the mean offset; unwrapping slips count in full here, as in the
                 paper's Table 1 (its L = 1 entry is 5.4 rad);
  * dx_rmse, dy_rmse  RMS error of the two derivative maps against the closed-form gradient.

    python -m paper_1910_11872_gb300.experiments [--size 512] [--hi 150] [--snr 0]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import rmusic, synth

MARGIN = 8  # the largest supported half-width: pixels valid for every window size


def _wrap(a):
    return (np.asarray(a) + np.pi) % (2 * np.pi) - np.pi


def wrapped_rmse(est, truth) -> float:
    d = _wrap(np.asarray(est, np.float64) - truth)
    c = np.angle(np.mean(np.exp(1j * d)))
    return float(np.sqrt(np.mean(_wrap(d - c) ** 2)))


def offset_rmse(est, truth) -> float:
    d = np.asarray(est, np.float64) - truth
    return float(np.sqrt(np.mean((d - d.mean()) ** 2)))


def square_maps(image: np.ndarray, Lp: int, device: int = 0):
    """(dx, dy, alpha, unwrapped phase) of one complex frame through the GPU square path."""
    import torch

    dem = rmusic.Demodulator(device=device, geometry="square", half_width=Lp, carrier_freq=0.0, unwrap=1)
    try:
        out, _, _ = dem.run(torch.from_numpy(np.ascontiguousarray(image)).cuda(device), with_status=False)
        torch.cuda.synchronize(device)
    finally:
        dem.close()
    return out.cpu().numpy().reshape(4, *image.shape)


def errors(maps, fr) -> dict:
    H, W = fr.image.shape
    m = np.zeros((H, W), dtype=bool)
    m[MARGIN:H - MARGIN, MARGIN:W - MARGIN] = True
    phi = fr.meta["phi"]
    return {"alpha_rmse": wrapped_rmse(maps[2][m], phi[m]), "phase_rmse": offset_rmse(maps[3][m], phi[m]),
            "dx_rmse": float(np.sqrt(np.mean((maps[0][m] - fr.truth[m]) ** 2))),
            "dy_rmse": float(np.sqrt(np.mean((maps[1][m] - fr.meta["truth_dy"][m]) ** 2)))}


def rmse_vs_half_width(half_widths=range(1, 9), snr_db: float = 0.0, size: int = 512, hi: float = 150.0,
                       stream: int = 0) -> list[dict]:
    fr = synth.complex_fringe_frame(snr_db, size, size, hi, stream=stream)
    return [{"Lp": Lp, "snr_db": snr_db, **errors(square_maps(fr.image, Lp), fr)} for Lp in half_widths]


def rmse_vs_snr(snrs=(-5.0, 0.0, 5.0, 10.0, 15.0, 20.0), Lp: int = 4, size: int = 512, hi: float = 150.0,
                stream: int = 0) -> list[dict]:
    out = []
    for snr in snrs:
        fr = synth.complex_fringe_frame(snr, size, size, hi, stream=stream)
        out.append({"Lp": Lp, "snr_db": snr, **errors(square_maps(fr.image, Lp), fr)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--hi", type=float, default=150.0, help="phase range of the peaks stand-in (rad)")
    ap.add_argument("--snr", type=float, default=0.0, help="SNR of the half-width sweep (dB)")
    ap.add_argument("--lp", type=int, default=4, help="half-width of the SNR sweep")
    args = ap.parse_args()
    for r in rmse_vs_half_width(snr_db=args.snr, size=args.size, hi=args.hi):
        print(json.dumps({"experiment": "rmse_vs_half_width", "hi": args.hi, **r}))
    for r in rmse_vs_snr(Lp=args.lp, size=args.size, hi=args.hi):
        print(json.dumps({"experiment": "rmse_vs_snr", "hi": args.hi, **r}))


if __name__ == "__main__":
    main()
