"""GPU parity of model order p > 1 on raw real fringes (no band-pass; the line minus its mean) in
the plain paths, against the FP64 oracle: the FP64 path to float32 output resolution, the FP32 path
within 1e-4 on noise-free inputs and within 1 % RMS under noise."""
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


def run(img, **params):
    torch = _torch()
    dem = rmusic.Demodulator(**params)
    try:
        out, st, _ = dem.run(torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda())
        torch.cuda.synchronize()
    finally:
        dem.close()
    return out.cpu().numpy().reshape(img.shape), st.cpu().numpy().reshape(img.shape)


def _fringe(H, W, snr, offset_step=0.0, seed=0):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    phi = 1.5 * np.sin(x / 41.0) + 0.02 * y
    img = 0.5 + offset_step * (x < W // 2) + 0.4 * np.cos(TWO_PI * 0.1 * x + phi)
    if np.isfinite(snr):
        img = img + synth.sigma_for_snr(0.4, snr) * rng.normal(size=(H, W))
    return img.astype(np.float32), phi


@pytest.mark.parametrize("p,step", [(2, 0.0), (3, 0.25)])
def test_plain_fp64_model_order_matches_oracle(p, step):
    img, _ = _fringe(24, 160, 20.0, step)
    g, st = run(img, window_len=32, cov_order=8, model_order=p, raw_input=1, carrier_freq=0.1,
                precision="plain_fp64")
    o, ost, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, 0.1, model_order=p, raw_input=1))
    assert np.array_equal(st, ost)
    v = ost == 0
    o32 = o[v].astype(np.float32)
    tol = np.maximum(np.spacing(np.abs(o32)), np.float32(1e-9))
    assert (np.abs(g[v] - o32) <= tol).all(), np.abs(g[v] - o32).max()


def test_plain_fp32_model_order_two():
    H, W, f, f0 = 8, 256, 32 / 256, 0.1
    y, x = np.mgrid[0:H, 0:W]
    clean = (0.5 + 0.4 * np.cos(TWO_PI * f * x + 0.2 * y)).astype(np.float32)
    g, st = run(clean, window_len=32, cov_order=8, model_order=2, raw_input=1, carrier_freq=f0,
                precision="plain_fp32")
    # a noise-free cosine gives two double roots on the circle, where FP32 Aberth may stop at its
    # iteration cap (status 3, best estimate stored): those values must be right as well
    v = (st == 0) | (st == 3)
    assert v.sum() == H * (W - 31), np.bincount(st.ravel(), minlength=4)
    assert np.abs(g[v] - TWO_PI * (f - f0)).max() <= 1e-4, np.bincount(st.ravel(), minlength=4)
    img, phi = _fringe(32, 256, 15.0, seed=3)
    g, st = run(img, window_len=32, cov_order=8, model_order=2, raw_input=1, carrier_freq=0.1,
                precision="plain_fp32")
    o, ost, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, 0.1, model_order=2, raw_input=1))
    truth = np.gradient(phi, axis=1)
    m = (st == 0) & (ost == 0)
    m[:, :48] = False
    m[:, -48:] = False
    eg = np.sqrt(np.mean((g[m] - truth[m]) ** 2))
    eo = np.sqrt(np.mean((o[m] - truth[m]) ** 2))
    assert abs(eg - eo) <= 0.01 * eo, (eg, eo)
