"""GPU parity of the square-block path (the paper's own geometry: a (2Lp+1) x (2Lp+1) block per
pixel giving d/dx, d/dy and the local phase alpha; Sec. 3, Eq. 4-15, Algorithm 1) against the FP64
oracle, through the C ABI.

Tolerances:
  * noise-free inputs: |gpu - oracle| <= 1e-4 (rad/pixel for the derivatives, rad for alpha) on
    every valid pixel, and the same against the closed form;
  * under noise: the RMS error against the closed-form phase derivatives and phase is within 1 %
    of the oracle's; element-wise differences are reported and bounded loosely (a near tie between
    two roots' distances to the circle can be decided differently in FP32 and FP64).
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_11872_gb300 import rmusic, synth

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _wrap(a):
    return (np.asarray(a) + np.pi) % TWO_PI - np.pi


def _torch():
    import torch

    assert torch.cuda.is_available(), "these tests need a CUDA device"
    return torch


def _to_dev(img):
    torch = _torch()
    img = np.ascontiguousarray(img)
    if img.dtype == np.uint16:
        return torch.from_numpy(img.view(np.int16)).cuda()
    if img.dtype == np.complex64:
        return torch.from_numpy(img).cuda()
    return torch.from_numpy(img.astype(np.float32)).cuda()


def run_square(frames, Lp, f0=0.0, carrier_axis=0, with_stats=False, **kw):
    """Demodulate 2-D numpy frames in ONE call; returns [(dx, dy, alpha, status), ...]."""
    torch = _torch()
    dem = rmusic.Demodulator(geometry="square", half_width=Lp, carrier_freq=f0, carrier_axis=carrier_axis,
                             precision="batched", **kw)
    try:
        out, st, shapes = dem.run([_to_dev(f) for f in frames])
        torch.cuda.synchronize()
        out, st = out.cpu().numpy(), st.cpu().numpy()
        res, o = [], 0
        for H, W in shapes:
            n = H * W
            res.append((out[o:o + n].reshape(H, W), out[o + n:o + 2 * n].reshape(H, W),
                        out[o + 2 * n:o + 3 * n].reshape(H, W), st[o:o + n].reshape(H, W)))
            o += 3 * n
        if with_stats:
            return res, dem.stats()
        return res
    finally:
        dem.close()


def oracle_square(img, Lp, f0=0.0, carrier_axis=0):
    dx, dy, al, st, _ = O.square_demodulate(img, O.make_params(carrier_axis=carrier_axis, carrier_freq=f0), Lp)
    return dx, dy, al, st


def _plane(H, W, wx, wy, a0, f0=0.0):
    y, x = np.mgrid[0:H, 0:W]
    return np.exp(1j * (a0 + (wx + TWO_PI * f0) * x + wy * y)).astype(np.complex64), a0 + wx * x + wy * y


# ------------------------------------------------------------------------------------------------
# noise-free: closed form and oracle within 1e-4
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("Lp", [1, 2, 3, 4, 5, 6, 7, 8])
def test_square_plane_wave_noise_free(Lp):
    H, W = 37, 70  # ragged against the 32 x 4 tiles
    img, phase = _plane(H, W, 0.61, -0.37, 0.9)
    (dx, dy, al, st), = run_square([img], Lp)
    valid = st == 0
    assert valid.sum() == (H - 2 * Lp) * (W - 2 * Lp)
    assert np.abs(dx[valid] - 0.61).max() <= 1e-4
    assert np.abs(dy[valid] + 0.37).max() <= 1e-4
    assert np.abs(_wrap(al[valid] - phase[valid])).max() <= 1e-4
    odx, ody, oal, ost = oracle_square(img, Lp)
    assert np.array_equal(st, ost)
    assert np.abs(dx[valid] - odx[valid]).max() <= 1e-4
    assert np.abs(dy[valid] - ody[valid]).max() <= 1e-4
    assert np.abs(_wrap(al[valid] - oal[valid])).max() <= 1e-4
    border = st == 1
    assert np.isnan(dx[border]).all() and np.isnan(dy[border]).all() and np.isnan(al[border]).all()


@pytest.mark.parametrize("wx,wy", [(2.9, 0.1), (-2.8, -2.9), (0.0, 0.0), (1.5, -1.5)])
def test_square_plane_wave_angles(wx, wy):
    img, phase = _plane(24, 64, wx, wy, -2.0)
    (dx, dy, al, st), = run_square([img], 3)
    v = st == 0
    assert np.abs(_wrap(dx[v] - wx)).max() <= 1e-4 and np.abs(_wrap(dy[v] - wy)).max() <= 1e-4
    assert np.abs(_wrap(al[v] - phase[v])).max() <= 1e-4


@pytest.mark.parametrize("carrier_axis", [0, 1])
def test_square_real_fringe_with_carrier(carrier_axis):
    """Real fringe through the band-pass; the carrier is removed from the derivative along it and
    from alpha (closed form as in the oracle's pin)."""
    H, W, f, f0, wy, th = 48, 128, 16 / 128, 0.1, 0.3, 0.4
    y, x = np.mgrid[0:H, 0:W]
    img = (0.5 + 0.4 * np.cos(TWO_PI * f * x + wy * y + th)).astype(np.float32)
    exp_dx, exp_dy = TWO_PI * (f - f0), wy
    exp_al = TWO_PI * (f - f0) * x + wy * y + th
    if carrier_axis == 1:
        img, exp_al = np.ascontiguousarray(img.T), exp_al.T
        exp_dx, exp_dy = exp_dy, exp_dx
    (dx, dy, al, st), = run_square([img], 3, f0=f0, carrier_axis=carrier_axis)
    v = st == 0
    assert v.sum() == (img.shape[0] - 6) * (img.shape[1] - 6)
    assert np.abs(dx[v] - exp_dx).max() <= 1e-4
    assert np.abs(dy[v] - exp_dy).max() <= 1e-4
    assert np.abs(_wrap(al[v] - exp_al[v])).max() <= 1e-4


# ------------------------------------------------------------------------------------------------
# under noise: RMS error within 1 % of the oracle's; element-wise differences reported
# ------------------------------------------------------------------------------------------------
def _rms(a):
    return float(np.sqrt(np.mean(np.square(a))))


@pytest.mark.parametrize("snr,Lp", [(20.0, 3), (10.0, 5), (0.0, 5), (0.0, 7), (5.0, 2)])
def test_square_noisy_complex_fringe_vs_oracle(snr, Lp):
    fr = synth.complex_fringe_frame(snr, H=96, W=160, hi=6.0)
    img = fr.image
    (dx, dy, al, st), = run_square([img], Lp)
    odx, ody, oal, ost = oracle_square(img, Lp)
    assert np.array_equal(st == 1, ost == 1)
    both = (st == 0) & (ost == 0)
    assert both.sum() >= 0.999 * (ost == 0).sum()
    ddx = np.abs(dx[both] - odx[both])
    ddy = np.abs(dy[both] - ody[both])
    dal = np.abs(_wrap(al[both] - oal[both]))
    # a near tie between two roots may be decided differently: at most 0.2 % of the pixels differ
    # by more than 1e-3, and the rest agree to the FP32 resolution of the estimator
    for d in (ddx, ddy, dal):
        assert np.mean(d > 1e-3) <= 2e-3, (snr, Lp, np.percentile(d, [50, 99, 99.9]), d.max())
        assert np.percentile(d, 99) <= 2e-4, (snr, Lp, np.percentile(d, [50, 99, 99.9]), d.max())
    # accuracy against the closed form, interior pixels
    m = np.zeros_like(both)
    m[2 * Lp:-2 * Lp, 2 * Lp:-2 * Lp] = True
    m &= both
    for g, o, t in ((dx, odx, fr.truth), (dy, ody, fr.meta["truth_dy"])):
        eg, eo = _rms(g[m] - t[m]), _rms(o[m] - t[m])
        assert abs(eg - eo) <= 0.01 * eo, (snr, Lp, eg, eo)
    eg = _rms(_wrap(al[m] - fr.meta["phi"][m]))
    eo = _rms(_wrap(oal[m] - fr.meta["phi"][m]))
    assert abs(eg - eo) <= 0.01 * eo, (snr, Lp, eg, eo)


def test_square_full_size_real_frame_sampled():
    """1024 x 1024 real peaks fringe (f0 = 0.1, 20 dB), Lp = 5, against the oracle on sampled pixels."""
    fr = synth.peaks_frame(20.0, 0.1, 1024, 1024)
    (dx, dy, al, st), = run_square([fr.image], 5, f0=0.1)
    rng = np.random.default_rng(11)
    ys = rng.integers(0, 1024, 1500)
    xs = rng.integers(0, 1024, 1500)
    ys[:4] = [0, 5, 1023, 517]
    xs[:4] = [0, 5, 1023, 1018]
    odx, ody, oal, ost, _ = O.square_demodulate_pixels(fr.image, O.make_params(carrier_freq=0.1), 5, ys, xs)
    assert np.array_equal(st[ys, xs] == 1, ost == 1)
    v = (ost == 0) & (st[ys, xs] == 0)
    assert v.sum() >= 0.999 * (ost == 0).sum()
    for g, o in ((dx[ys, xs], odx), (dy[ys, xs], ody)):
        d = np.abs(g[v] - o[v])
        assert np.percentile(d, 99) <= 1e-4 and np.mean(d > 1e-3) <= 2e-3, (np.percentile(d, [50, 99]), d.max())
    d = np.abs(_wrap(al[ys, xs][v] - oal[v]))
    assert np.percentile(d, 99) <= 1e-4 and np.mean(d > 1e-3) <= 2e-3, (np.percentile(d, [50, 99]), d.max())


# ------------------------------------------------------------------------------------------------
# batching, edges, formats
# ------------------------------------------------------------------------------------------------
def test_square_alone_equals_batched_bitwise():
    frames = [synth.complex_fringe_frame(10.0, H=h, W=w, hi=5.0, stream=i).image
              for i, (h, w) in enumerate([(40, 70), (9, 9), (64, 33), (5, 200), (100, 128)])]
    mixed = run_square(frames, 4)
    for f, m in zip(frames, mixed):
        (alone,) = run_square([f], 4)
        for a, b in zip(alone, m):
            assert np.array_equal(a, b, equal_nan=True)


def test_square_edge_shapes_and_zero_frame():
    tiny = np.ones((5, 8), np.complex64)          # smaller than the 9 x 9 block: all border
    one = np.ones((1, 1), np.complex64)
    zero = np.zeros((20, 40), np.complex64)       # valid blocks of zeros: degenerate
    res = run_square([tiny, one, zero], 4)
    for dx, dy, al, st in res[:2]:
        assert (st == 1).all() and np.isnan(dx).all() and np.isnan(al).all()
    dx, dy, al, st = res[2]
    inner = np.zeros_like(st, dtype=bool)
    inner[4:-4, 4:-4] = True
    assert (st[inner] == 2).all() and (st[~inner] == 1).all()
    assert np.isnan(dx).all() and np.isnan(dy).all() and np.isnan(al).all()


def test_square_uint16_frame_matches_float():
    fr = synth.diffusion_frame(100, H=64, W=256)
    img16 = fr.image
    res16 = run_square([img16], 3, f0=0.1)[0]
    res32 = run_square([img16.astype(np.float32)], 3, f0=0.1)[0]
    v = res32[3] == 0
    assert np.array_equal(res16[3], res32[3])
    for a, b in zip(res16[:2], res32[:2]):
        assert np.abs(a[v] - b[v]).max() <= 1e-4
    assert np.abs(_wrap(res16[2][v] - res32[2][v])).max() <= 1e-4


def test_square_graph_replay_and_host_entry():
    torch = _torch()
    frames = [synth.complex_fringe_frame(10.0, H=64, W=96, stream=i).image for i in range(3)]
    dem = rmusic.Demodulator(geometry="square", half_width=3, carrier_freq=0.0, use_graph=1)
    try:
        tens = torch.stack([_to_dev(f) for f in frames])  # one contiguous input: same pointer each call
        o, st, _ = dem.run(tens)
        o1 = o.clone()
        o2, s2, _ = dem.run(tens, out=o, status=st)  # same buffers: the captured graph is replayed
        torch.cuda.synchronize()
        assert dem.stats().graph_replayed == 1
        assert torch.equal(torch.nan_to_num(o1, 7.0), torch.nan_to_num(o2, 7.0))
        # host buffers: same maps
        flat = np.concatenate([f.reshape(-1) for f in frames])
        descs, nbytes, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_C64, 8, maps=3)
        h_out = np.empty(nout, np.float32)
        h_st = np.empty(nout, np.uint8)
        rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, len(frames),
                                             h_out.ctypes.data, h_st.ctypes.data, None)
        assert np.array_equal(h_out, o1.cpu().numpy(), equal_nan=True)
    finally:
        dem.close()


def test_square_variants_identical():
    """Both register-cap variants compute the same maps bit for bit: rmusic_autotune runs every
    variant on the call's frames, so its output is the last variant's; plain calls use variant 0."""
    torch = _torch()
    frames = [synth.complex_fringe_frame(5.0, H=80, W=128, stream=i).image for i in range(2)]
    outs = []
    for v in range(2):
        dem = rmusic.Demodulator(geometry="square", half_width=5, carrier_freq=0.0)
        try:
            tens = [_to_dev(f) for f in frames]
            descs, _, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_C64, 8, maps=3)
            flat = torch.cat([t.reshape(-1) for t in tens])
            out = torch.empty(nout, dtype=torch.float32, device="cuda")
            if v == 0:
                rmusic.rmusic_demodulate_frames(dem.ctx, flat.data_ptr(), descs, 2, out.data_ptr(), None, None)
            else:
                rmusic.rmusic_autotune(dem.ctx, flat.data_ptr(), descs, 2, out.data_ptr(), None, None)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        finally:
            dem.close()
    assert np.array_equal(outs[0], outs[1], equal_nan=True)


def test_square_stats_and_launches():
    frames = [synth.complex_fringe_frame(0.0, H=64, W=64).image]
    res, st = run_square(frames, 5, with_stats=True, timing=1)
    assert st.kernel_launches == 1  # a complex frame is the analytic signal: the solver reads it in place
    assert 1.0 <= st.mean_sweeps <= 100.0
    # the signal root of both polynomials by Newton's method; the Aberth fallback only where the
    # certificate fails in some lane (at most both polynomials of every work item)
    assert 2.0 <= st.mean_newton_steps <= 32.0 and 0.0 <= st.root_fallback_frac <= 2.0
    assert st.mean_polish_steps == 4.0, st.mean_polish_steps  # two steps for each polynomial
    assert st.solver_ms > 0


def test_square_complex_frames_in_place_pitched():
    """Complex64 frames are read in place: frames at byte offsets inside a wider, padded buffer (row
    pitch above the width) give the same maps bit for bit as the same frames packed."""
    torch = _torch()
    frames = [synth.complex_fringe_frame(5.0, H=h, W=w, stream=i).image for i, (h, w) in
              enumerate([(40, 72), (33, 50)])]
    packed = run_square(frames, 4)
    pitch = 80
    rows = sum(f.shape[0] for f in frames) + 3
    buf = np.full((rows, pitch), np.complex64(7 + 7j))  # padding that must never be read
    descs = (rmusic.rmusic_frame_desc * 2)()
    r0, oo = 1, 0
    for i, f in enumerate(frames):
        H, W = f.shape
        buf[r0:r0 + H, 2:2 + W] = f
        descs[i] = rmusic.rmusic_frame_desc((r0 * pitch + 2) * 8, H, W, pitch, rmusic.RMUSIC_DTYPE_C64, oo, 0, 0)
        r0 += H + 1
        oo += 3 * H * W
    dem = rmusic.Demodulator(geometry="square", half_width=4, carrier_freq=0.0, precision="batched")
    try:
        d_in = torch.from_numpy(buf).cuda()
        out = torch.empty(oo, dtype=torch.float32, device="cuda")
        st = torch.empty(oo, dtype=torch.uint8, device="cuda")
        rmusic.rmusic_demodulate_frames(dem.ctx, d_in.data_ptr(), descs, 2, out.data_ptr(), st.data_ptr(), None)
        torch.cuda.synchronize()
        assert dem.stats().kernel_launches == 1
        o, s8 = out.cpu().numpy(), st.cpu().numpy()
    finally:
        dem.close()
    off = 0
    for (dx, dy, al, stp), f in zip(packed, frames):
        n = f.size
        H, W = f.shape
        assert np.array_equal(o[off:off + n].reshape(H, W), dx, equal_nan=True)
        assert np.array_equal(o[off + n:off + 2 * n].reshape(H, W), dy, equal_nan=True)
        assert np.array_equal(o[off + 2 * n:off + 3 * n].reshape(H, W), al, equal_nan=True)
        assert np.array_equal(s8[off:off + n].reshape(H, W), stp)
        off += 3 * n
