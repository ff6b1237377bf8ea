"""The two band-pass schedules against the oracle.

Row lines of 256, 512 or 1024 samples whose windows run along the carrier go through the warp-FFT
kernel (a warp takes 32 / R lines of 32 R samples, a CTA four warps); other lines through the
per-line kernel. These cases cover the warp-FFT kernel's partial line groups (line counts that are
not multiples of a warp's or a CTA's group), a padded row pitch, 12-bit uint16 input, frames of both
schedules in one call, and the same frame through both schedules (transposed, so that the per-line
kernel takes it), each against the FP64 oracle: noise-free within 1e-4 rad/px, noisy with the
oracle's RMS error against the closed form within 1 %.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_11872_gb300 import rmusic, synth

pytestmark = pytest.mark.gpu


def _run(frames, windows=None, **params):
    import torch

    dem = rmusic.Demodulator(**params)
    try:
        tens = []
        for f in frames:
            a = np.ascontiguousarray(f)
            tens.append(torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda())
        out, st, shapes = dem.run(tens, windows=windows)
        torch.cuda.synchronize()
    finally:
        dem.close()
    out, st = out.cpu().numpy(), st.cpu().numpy()
    res, o = [], 0
    for H, W in shapes:
        res.append((out[o:o + H * W].reshape(H, W), st[o:o + H * W].reshape(H, W)))
        o += H * W
    return res


def _check(img, g, gs, f0=0.1, deriv_axis=0, carrier_axis=0, truth=None, quantized=False):
    o, os_ = O.demodulate(img, O.make_params(32, 8, 1, deriv_axis, carrier_axis, f0))[:2]
    assert np.array_equal(gs, os_)
    v = os_ == 0
    if quantized:
        # 12-bit codes: elementwise agreement at the FP32 level except near ties of the estimator
        d = np.abs(g[v].astype(np.float64) - o[v])
        assert np.quantile(d, 0.999) <= 1e-4 and d.max() <= 1e-3
    elif truth is None:
        assert np.abs(g[v].astype(np.float64) - o[v]).max() <= 1e-4
    else:
        rms_o = np.sqrt(np.mean((o[v] - truth[v]) ** 2))
        rms_g = np.sqrt(np.mean((g[v].astype(np.float64) - truth[v]) ** 2))
        assert abs(rms_g - rms_o) <= 0.01 * rms_o


@pytest.mark.parametrize("W", [256, 512, 1024])
@pytest.mark.parametrize("H", [2, 3, 5, 17])
def test_warp_fft_partial_line_groups_noise_free(H, W):
    fr = synth.peaks_frame(np.inf, 0.1, H=H, W=W)
    (g, gs), = _run([fr.image])
    _check(fr.image, g, gs)


@pytest.mark.parametrize("W", [256, 512, 1024])
def test_warp_fft_single_line_exact_frequency(W):
    """One line (a warp group with one valid line): a periodic fringe at 0.125 cycles/px gives
    2 pi (0.125 - 0.1) rad/px at every valid pixel, as the oracle."""
    fr = synth.periodic_linear_frame(H=1, W=W, f=0.125, f0=0.1)
    (g, gs), = _run([fr.image])
    _check(fr.image, g, gs)
    v = gs == 0
    assert v.sum() == W - 31 and np.abs(g[v] - fr.truth[v]).max() <= 1e-4


@pytest.mark.parametrize("W", [256, 1024])
def test_warp_fft_noisy_uint16_and_float(W):
    fr = synth.peaks_frame(10.0, 0.1, H=37, W=W)
    (g, gs), = _run([fr.image])
    _check(fr.image, g, gs, truth=fr.truth)
    q = synth.quantize12(fr.image)
    (g16, gs16), = _run([q])
    _check(q, g16, gs16, truth=fr.truth)


def test_warp_fft_padded_pitch_equals_dense():
    import torch

    fr = synth.peaks_frame(20.0, 0.1, H=9, W=512)
    padded = np.zeros((9, 640), dtype=np.float32)
    padded[:, :512] = fr.image
    buf = torch.from_numpy(np.concatenate([np.zeros(8, np.float32), padded.ravel()])).cuda()
    out = torch.empty(9 * 512, device="cuda")
    st = torch.empty(9 * 512, dtype=torch.uint8, device="cuda")
    dem = rmusic.Demodulator()
    try:
        d = rmusic.rmusic_frame_desc(8 * 4, 9, 512, 640, rmusic.RMUSIC_DTYPE_F32, 0, 0, 0)
        rmusic.rmusic_demodulate_frames(dem.ctx, buf.data_ptr(), [d], 1, out.data_ptr(), st.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        dem.close()
    (g, gs), = _run([fr.image])
    assert np.array_equal(out.cpu().numpy().reshape(9, 512), g, equal_nan=True)
    assert np.array_equal(st.cpu().numpy().reshape(9, 512), gs)


def test_both_schedules_in_one_call_and_transposed_frame():
    """A 1024-wide frame (warp FFT), a 300-wide frame (per-line DFT) and a 2048-wide frame
    (per-line FFT) in one call; and the 1024-wide frame transposed with the carrier along y (its
    carrier lines are then columns, which the per-line kernel takes) gives the transposed map."""
    f1 = synth.peaks_frame(np.inf, 0.1, H=12, W=1024)
    f2 = synth.peaks_frame(np.inf, 0.1, H=10, W=300)
    f3 = synth.peaks_frame(np.inf, 0.1, H=6, W=2048)
    res = _run([f1.image, f2.image, f3.image])
    for fr, (g, gs) in zip((f1, f2, f3), res):
        _check(fr.image, g, gs)
    (gt, gst), = _run([np.ascontiguousarray(f1.image.T)], deriv_axis=1, carrier_axis=1)
    v = res[0][1] == 0
    assert np.array_equal(gst.T, res[0][1])
    assert np.abs(gt.T[v] - res[0][0][v]).max() <= 2e-5


@pytest.mark.parametrize("W", [256, 512, 1024])
def test_warp_fft_with_column_windows(W):
    """Carrier lines are rows (warp FFT), windows run down the columns: the band-pass writes the
    analytic signal column-major. Partial line groups (H = 45) and 12-bit input."""
    fr = synth.peaks_frame(np.inf, 0.1, H=45, W=W)
    q = synth.quantize12(fr.image)
    for img, quantized in ((fr.image, False), (q, True)):
        (g, gs), = _run([img], deriv_axis=1)
        _check(img, g, gs, deriv_axis=1, quantized=quantized)
