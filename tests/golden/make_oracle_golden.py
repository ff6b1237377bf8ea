"""Writes oracle_gaussian_bump_128_samples.txt: the FP64 oracle's derivative at 160 seeded pixels of
the 128 x 128 Gaussian-bump fringe (I = 0.5 + 0.4 cos(2 pi 0.1 x + phi), phi a 3-rad Gaussian of
std 20 px, noise sigma 0.02; window N = 32, covariance order L = 8, forward-backward, derivative
along x). Calls only the oracle and the seeded input generator.

    python tests/golden/make_oracle_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1910_11872_gb300 import synth  # noqa: E402

PATH = os.path.join(HERE, "oracle_gaussian_bump_128_samples.txt")


def sample_pixels():
    rng = np.random.default_rng(20191026)
    return rng.integers(0, 128, 160).astype(np.int32), rng.integers(0, 128, 160).astype(np.int32)


def compute():
    fr = synth.small_gaussian_frame()
    ys, xs = sample_pixels()
    vals, st, _ = O.demodulate_pixels(fr.image, O.make_params(32, 8, 1, 0, 0, 0.1), ys, xs)
    return ys, xs, vals, st


def main():
    ys, xs, vals, st = compute()
    with open(PATH, "w") as f:
        f.write("# FP64 oracle, 128 x 128 Gaussian-bump fringe (noise sigma 0.02), N = 32, L = 8,\n")
        f.write("# forward-backward, derivative along x, carrier 0.1 removed; written by make_oracle_golden.py\n")
        f.write("# y x status derivative_rad_per_px (nan where status != 0)\n")
        for y, x, s, v in zip(ys, xs, st, vals):
            f.write(f"{int(y)} {int(x)} {int(s)} {float(v)!r}\n")
    print(PATH)


if __name__ == "__main__":
    main()
