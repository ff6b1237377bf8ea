"""The FP32-batched path on the paper's own forward estimate (forward_backward = 0: R = R_f of Sec. 3,
Eq. 4-5, without the forward-backward average), against the FP64 oracle with fb = 0, through the C ABI.

The bar is the batched path's: identical status maps and max |GPU - oracle| <= 1e-4 rad/px on every
pixel both call ok (noise-free and noisy; near ties excused only as tests/parity.py allows), RMS error
against the closed-form derivative within 1 % of the oracle's under noise; certified and exhaustive
roots agree; frames mixed in one call give the maps they give alone, bit for bit.
"""
import numpy as np
import pytest

import oracle as O
import parity
from paper_1910_11872_gb300 import rmusic, synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _run(frames, windows=None, **params):
    import torch

    dem = rmusic.Demodulator(forward_backward=0, **params)
    try:
        tens = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]
        out, st, shapes = dem.run(tens, windows=windows)
        torch.cuda.synchronize()
        stats = dem.stats()
    finally:
        dem.close()
    out, st = out.cpu().numpy(), st.cpu().numpy()
    res, o = [], 0
    for H, W in shapes:
        res.append((out[o:o + H * W].reshape(H, W), st[o:o + H * W].reshape(H, W)))
        o += H * W
    return res, stats


@pytest.mark.parametrize("N,L", [(32, 8), (24, 6), (16, 4), (48, 12), (21, 7), (12, 3), (8, 2), (40, 10)])
def test_forward_noise_free_and_noisy_match_the_oracle(N, L):
    for snr in (np.inf, 20.0, 5.0):
        fr = synth.peaks_frame(snr, 0.1, H=24, W=320)
        ((g, gs),), _ = _run([fr.image], window_len=N, cov_order=L)
        o, os_, _ = O.demodulate(fr.image, O.make_params(N, L, 0, 0, 0, 0.1))
        parity.check(g, gs, o, os_, TOL, parity.Window(fr.image, N, L, 0, 0, 0, 0.1), what=f"fb=0 N={N} L={L} {snr} dB")
        if np.isfinite(snr):
            v = (os_ == 0) & (gs == 0)
            inner = np.zeros_like(v)
            inner[:, N:-N] = True
            parity.rms_check(g, o, fr.truth, v & inner, what=f"fb=0 N={N} L={L} {snr} dB")


def test_forward_column_windows_uint16_diffusion():
    frames = [synth.diffusion_frame(t, T=50, H=160, W=96) for t in (0, 49)]
    res, _ = _run([f.image for f in frames], deriv_axis=1)
    for fr, (g, gs) in zip(frames, res):
        o, os_, _ = O.demodulate(fr.image, O.make_params(32, 8, 0, 1, 0, 0.1))
        parity.check(g, gs, o, os_, TOL, parity.Window(fr.image, 32, 8, 0, 1, 0, 0.1), what="fb=0 diffusion")


@pytest.mark.parametrize("N,L", [(32, 8), (24, 5)])
def test_forward_certified_and_exhaustive_select_the_same_root(N, L):
    fr = synth.peaks_frame(10.0, 0.1, H=32, W=256)
    ((g, gs),), st = _run([fr.image], window_len=N, cov_order=L)
    ((ge, ges),), se = _run([fr.image], window_len=N, cov_order=L, exhaustive=1)
    assert np.array_equal(gs, ges)
    v = gs == 0
    assert np.abs(g[v] - ge[v]).max() <= 2e-5
    assert se.eig_fallback_frac == 1.0 and se.root_fallback_frac == 1.0
    assert st.root_fallback_frac <= 0.05 and 1.0 <= st.mean_power_steps <= 8.0


def test_forward_uneven_mix_equals_alone():
    rng = np.random.default_rng(9)
    shapes = [(40, 96), (17, 300), (33, 129), (8, 512)]
    windows = [(32, 8), (24, 5), (32, 8), (48, 11)]
    frames = []
    for H, W in shapes:
        phi, _, _ = synth.gaussian_sum(rng, H, W)
        frames.append(synth.add_noise(synth.fringe(phi, 0.1), 0.03, rng).astype(np.float32))
    mix, _ = _run(frames, windows=windows)
    for f, w, (g, gs) in zip(frames, windows, mix):
        (ga, gsa), = _run([f], window_len=w[0], cov_order=w[1])[0]
        assert np.array_equal(gs, gsa)
        assert np.array_equal(g, ga, equal_nan=True)
        o, os_, _ = O.demodulate(f, O.make_params(w[0], w[1], 0, 0, 0, 0.1))
        parity.check(g, gs, o, os_, TOL, parity.Window(f, w[0], w[1], 0, 0, 0, 0.1), what=f"fb=0 mix {f.shape} {w}")


def test_forward_is_not_the_forward_backward_estimate():
    """Where the two estimates differ (a fringe whose amplitude ramps from 0.02 to 0.47 along the
    window: R_f is far from centro-Hermitian where the amplitude is small), the path follows the
    forward estimate's oracle, not the forward-backward one's."""
    H, W = 8, 256
    x = np.arange(W)[None, :]
    rng = np.random.default_rng(1)
    phi, _, _ = synth.gaussian_sum(rng, H, W)
    img = 0.5 + (0.02 + 0.45 * (x / W) ** 3) * np.cos(2 * np.pi * 0.1 * x + phi)
    img = (img + 0.01 * rng.normal(size=img.shape)).astype(np.float32)
    ((g, gs),), _ = _run([img])
    o0, s0, _ = O.demodulate(img, O.make_params(32, 8, 0, 0, 0, 0.1))
    o1, s1, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, 0.1))
    v = (s0 == 0) & (s1 == 0) & (gs == 0)
    differ = v & (np.abs(o0 - o1) > 1e-2)
    assert differ.sum() >= 5
    d0 = np.abs(g[differ] - o0[differ])
    d1 = np.abs(g[differ] - o1[differ])
    assert np.all(d0 < d1) and np.median(d0) < 1e-3, (np.median(d0), np.median(d1))
