"""Pins for the oracle's 2-D band-pass variant (Sec. 2: the analytic signal from band-pass filtering;
the 2-D Fourier methods the paper cites): the carrier's one-sided band times a low-pass
|k / len| < B_c across the carrier lines, applied as a second pass. Checked against numpy's 2-D FFT
with the same rectangular mask, a closed form, and the method's exactness on a noise-free fringe."""
import numpy as np
import pytest

import oracle as O

TWO_PI = 2 * np.pi


def _mask(H, W, f0, B, Bc):
    ky = np.arange(H)[:, None]
    kx = np.arange(W)[None, :]
    kys = np.where(2 * ky < H, ky, ky - H)
    return (kx >= 1) & (2 * kx < W) & (np.abs(kx / W - f0) < B) & (np.abs(kys) < Bc * H)


@pytest.mark.parametrize("carrier_axis", [0, 1])
def test_band2d_matches_fft2_rectangle(carrier_axis):
    rng = np.random.default_rng(carrier_axis)
    H, W, f0, B, Bc = 36, 60, 0.12, 0.06, 0.11
    img = rng.normal(size=(H, W))
    ref = np.fft.ifft2(np.where(_mask(H, W, f0, B, Bc), np.fft.fft2(img), 0))
    if carrier_axis == 1:
        img, ref = img.T.copy(), ref.T
    g = O.cross_band(O.analytic_frame(img, f0, B, carrier_axis=carrier_axis), Bc, carrier_axis)
    assert np.abs(g - ref).max() < 1e-12


def test_band2d_plane_waves_inside_and_outside():
    """exp(2 pi j (kx x / W + ky y / H)) passes unchanged when |ky| / H < Bc and vanishes otherwise."""
    H, W = 32, 48
    y, x = np.mgrid[0:H, 0:W]
    for ky, keep in ((0, True), (3, True), (-3, True), (4, False), (10, False)):
        g = np.exp(TWO_PI * 1j * (6 * x / W + ky * y / H))
        out = O.cross_band(g, 0.12, 0)  # 0.12 * 32 = 3.84: |ky| <= 3 kept
        assert np.abs(out - (g if keep else 0)).max() < 1e-12, (ky, keep)


def test_band2d_keeps_noise_free_linear_phase_exact():
    """A periodic noise-free fringe with a y tilt inside the cross band demodulates exactly (P1)."""
    H, W, f, f0 = 32, 128, 16 / 128, 0.1
    y, x = np.mgrid[0:H, 0:W]
    wy = TWO_PI * 2 / H
    img = 0.5 + 0.4 * np.cos(TWO_PI * f * x + wy * y)
    out, st, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, f0, band_cross=0.1))
    v = st == 0
    assert v.sum() > 0 and np.abs(out[v] - TWO_PI * (f - f0)).max() < 1e-9
    dx, dy, al, sst, _ = O.square_demodulate(img, O.make_params(carrier_freq=f0, band_cross=0.1), 3)
    v = sst == 0
    assert np.abs(dy[v] - wy).max() < 1e-9


def test_band2d_sampled_equals_full():
    rng = np.random.default_rng(5)
    img = (0.5 + 0.4 * np.cos(TWO_PI * 0.1 * np.arange(96)[None, :] + rng.normal(0, 0.3, (24, 96)))).astype(np.float32)
    p = O.make_params(24, 6, 1, 0, 0, 0.1, band_cross=0.15)
    full, fst, _ = O.demodulate(img, p)
    ys, xs = rng.integers(0, 24, 40), rng.integers(0, 96, 40)
    smp, sst, _ = O.demodulate_pixels(img, p, ys, xs)
    np.testing.assert_array_equal(smp, full[ys, xs])
    np.testing.assert_array_equal(sst, fst[ys, xs])
