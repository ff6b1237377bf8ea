"""GPU parity of the 2-D band-pass variant (the carrier band times a low-pass across the carrier
lines, rmusic_params.band_cross) against the FP64 oracle. The plain FP64 path runs the cross pass
in double precision and must reproduce the oracle to float32 output resolution; the FP32 paths are
held to the usual bars (1e-4 noise-free, RMS within 1 % under noise)."""
import numpy as np
import pytest

import oracle as O
from paper_1910_11872_gb300 import rmusic, synth

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _torch():
    import torch

    assert torch.cuda.is_available(), "these tests need a CUDA device"
    return torch


def run(frames, **params):
    torch = _torch()
    dem = rmusic.Demodulator(**params)
    try:
        out, st, shapes = dem.run([torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames])
        torch.cuda.synchronize()
        launches = dem.stats().kernel_launches
    finally:
        dem.close()
    out, st = out.cpu().numpy(), st.cpu().numpy()
    maps = 3 if params.get("geometry") == "square" else 1
    res, o = [], 0
    for H, W in shapes:
        n = H * W
        res.append(([out[o + i * n:o + (i + 1) * n].reshape(H, W) for i in range(maps)], st[o:o + n].reshape(H, W)))
        o += maps * n
    return res, launches


def _noisy(H, W, snr, carrier_axis=0, seed=0):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    phi = 2.0 * np.sin(x / 37.0) + 1.5 * np.cos(y / 23.0)
    arg = TWO_PI * 0.1 * (x if carrier_axis == 0 else y) + phi
    return (0.5 + 0.4 * np.cos(arg) + synth.sigma_for_snr(0.4, snr) * rng.normal(size=(H, W))).astype(np.float32)


@pytest.mark.parametrize("deriv_axis,carrier_axis", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_plain_fp64_with_cross_band_matches_oracle(deriv_axis, carrier_axis):
    """Both workspace layouts (cross lines adjacent in memory or contiguous along themselves), ragged
    sizes (lines not a multiple of 32, lengths not a multiple of 64)."""
    img = _noisy(70, 100, 20.0, carrier_axis)
    Bc = 0.12
    ((g,), st), = run([img], window_len=24, cov_order=6, forward_backward=1, deriv_axis=deriv_axis,
                      carrier_axis=carrier_axis, carrier_freq=0.1, precision="plain_fp64", band_cross=Bc)[0]
    o, ost, _ = O.demodulate(img, O.make_params(24, 6, 1, deriv_axis, carrier_axis, 0.1, band_cross=Bc))
    assert np.array_equal(st, ost)
    v = ost == 0
    o32 = o[v].astype(np.float32)
    tol = np.maximum(np.spacing(np.abs(o32)), np.float32(1e-9))
    assert (np.abs(g[v] - o32) <= tol).all(), np.abs(g[v] - o32).max()


def test_batched_with_cross_band():
    H, W, f, f0 = 48, 256, 32 / 256, 0.1
    y, x = np.mgrid[0:H, 0:W]
    clean = (0.5 + 0.4 * np.cos(TWO_PI * f * x + TWO_PI * 2 / H * y)).astype(np.float32)
    noisy = _noisy(96, 256, 10.0)
    (((gc,), sc), ((gn,), sn)), launches = run([clean, noisy], carrier_freq=f0, band_cross=0.1)
    assert launches == 3  # band-pass, cross pass, solver
    v = sc == 0
    assert np.abs(gc[v] - TWO_PI * (f - f0)).max() <= 1e-4
    o, ost, _ = O.demodulate(noisy, O.make_params(32, 8, 1, 0, 0, f0, band_cross=0.1))
    both = (sn == 0) & (ost == 0)
    assert np.abs(gn[both] - o[both]).max() <= 1e-4


def test_square_with_cross_band():
    img = _noisy(64, 96, 15.0, 0, seed=2)
    ((dx, dy, al), st), = run([img], geometry="square", half_width=4, carrier_freq=0.1, band_cross=0.15)[0]
    odx, ody, oal, ost, _ = O.square_demodulate(img, O.make_params(carrier_freq=0.1, band_cross=0.15), 4)
    assert np.array_equal(st, ost)
    v = ost == 0
    for g, o in ((dx, odx), (dy, ody), (al, oal)):
        assert np.abs((g[v] - o[v] + np.pi) % TWO_PI - np.pi).max() <= 1e-4
