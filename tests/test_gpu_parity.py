"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle on the same seeded
inputs, element by element.

Tolerances (rad/pixel):
  * plain FP64 path: |gpu - oracle| <= 1e-9 on every valid pixel, identical status maps;
  * FP32-batched path, noise-free and noisy inputs alike: identical status maps and
    |gpu - oracle| <= 1e-4 on every pixel both call ok, except pixels the oracle's own roots show to
    be near ties at FP32 resolution (tests/parity.py; counted, at most 1e-4 of the pixels);
  * FP32 paths under noise, in addition: the RMS error against the closed-form derivative is within
    1 % of the oracle's RMS error (interior pixels).
"""
import numpy as np
import pytest

import oracle as O
import parity
from paper_1910_11872_gb300 import rmusic, synth

TOL = 1e-4  # rad/pixel: the FP32-batched path against the FP64 oracle, with or without noise

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def _torch():
    import torch

    assert torch.cuda.is_available(), "these tests need a CUDA device"
    return torch


def _to_dev(img):
    torch = _torch()
    if img.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(img).view(np.int16)).cuda()
    return torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()


def run_gpu(frames, windows=None, **params):
    """Demodulate a list of 2-D numpy frames in ONE call; returns [(deriv, status), ...]."""
    torch = _torch()
    dem = rmusic.Demodulator(**params)
    try:
        tens = [_to_dev(f) for f in frames]
        out, st, shapes = dem.run(tens, windows=windows)
        torch.cuda.synchronize()
        out = out.cpu().numpy()
        st = st.cpu().numpy()
        res, o = [], 0
        for H, W in shapes:
            res.append((out[o:o + H * W].reshape(H, W), st[o:o + H * W].reshape(H, W)))
            o += H * W
        dem.last_stats = dem.stats()
        return res
    finally:
        dem.close()


def oracle_run(img, N=32, L=8, fb=1, deriv_axis=0, carrier_axis=0, f0=0.1):
    out, st, _ = O.demodulate(img, O.make_params(N, L, fb, deriv_axis, carrier_axis, f0))
    return out, st


# ------------------------------------------------------------------------------------------------
# plain FP64 path == oracle to 1e-9
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N,L,fb", [(32, 8, 1), (32, 8, 0), (12, 3, 1), (24, 6, 0), (48, 12, 1), (9, 2, 1)])
def test_plain_fp64_matches_oracle(N, L, fb):
    fr = synth.small_gaussian_frame()
    (g, gs), = run_gpu([fr.image], window_len=N, cov_order=L, forward_backward=fb, precision="plain_fp64")
    o, os_ = oracle_run(fr.image, N, L, fb)
    assert np.array_equal(gs, os_)
    v = os_ == 0
    assert v.sum() == 128 * (128 - N + 1)
    # the map is float32: the FP64 result must round to the oracle's value within one float32 ulp
    # (or 1e-9 rad/pixel where the ulp is smaller)
    o32 = o[v].astype(np.float32)
    tol = np.maximum(np.spacing(np.abs(o32)), np.float32(1e-9))
    d = np.abs(g[v] - o32)
    bad = d > tol
    assert not bad.any(), (f"{bad.sum()} pixels differ; max {d.max():.3e}; gpu {g[v][bad][:4]} "
                           f"oracle {o[v][bad][:4]}")
    assert np.all(np.isnan(g[~v]))


def test_plain_fp64_periodic_is_exact():
    fr = synth.periodic_linear_frame(H=8, W=128)
    (g, gs), = run_gpu([fr.image], precision="plain_fp64")
    o, os_ = oracle_run(fr.image)
    v = os_ == 0
    assert np.array_equal(gs, os_)
    assert np.abs(g[v].astype(np.float64) - o[v]).max() < 1e-7  # float32 output rounding
    assert np.abs(g[v] - np.float32(TWO_PI * (16 / 128 - 0.1))).max() < 1e-7


# ------------------------------------------------------------------------------------------------
# FP32 batched path
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("f0", [0.08, 0.1, 0.15])
def test_batched_noise_free_within_1e4(f0):
    fr = synth.peaks_frame(np.inf, f0, H=48, W=384)
    (g, gs), = run_gpu([fr.image], carrier_freq=f0)
    o, os_ = oracle_run(fr.image, f0=f0)
    assert np.array_equal(gs, os_)
    v = os_ == 0
    err = np.abs(g[v].astype(np.float64) - o[v])
    assert err.max() <= TOL, f"max {err.max():.3e} p99.9 {np.quantile(err, 0.999):.3e}"


@pytest.mark.parametrize("snr", [40, 20, 10, 5])
def test_batched_noisy_rms_within_one_percent(snr):
    fr = synth.peaks_frame(snr, 0.1, H=64, W=384)
    (g, gs), = run_gpu([fr.image])
    o, os_ = oracle_run(fr.image)
    parity.check(g, gs, o, os_, TOL, parity.Window(fr.image, 32, 8, 1, 0, 0, 0.1), what=f"{snr} dB")
    inner = np.zeros_like(os_, dtype=bool)
    inner[:, 32:-32] = True
    v = inner & (os_ == 0) & (gs == 0)
    parity.rms_check(g, o, fr.truth, v, what=f"{snr} dB")


@pytest.mark.parametrize("N,L", [(8, 2), (16, 4), (24, 6), (48, 12), (40, 10), (33, 8)])
def test_batched_windows(N, L):
    fr = synth.peaks_frame(np.inf, 0.1, H=24, W=256)
    (g, gs), = run_gpu([fr.image], window_len=N, cov_order=L)
    o, os_ = oracle_run(fr.image, N, L)
    assert np.array_equal(gs, os_)
    v = os_ == 0
    assert np.abs(g[v].astype(np.float64) - o[v]).max() <= TOL
    fr = synth.peaks_frame(10, 0.1, H=24, W=256)
    (g, gs), = run_gpu([fr.image], window_len=N, cov_order=L)
    o, os_ = oracle_run(fr.image, N, L)
    parity.check(g, gs, o, os_, TOL, parity.Window(fr.image, N, L, 1, 0, 0, 0.1), what=f"N={N} L={L} 10 dB")
    v = (os_ == 0) & (gs == 0)
    inner = np.zeros_like(v)
    inner[:, 32:-32] = True
    parity.rms_check(g, o, fr.truth, v & inner, what=f"N={N} L={L}")


def test_batched_deriv_y_uint16_diffusion():
    """Diffusion frames (uint16, 12-bit), carrier along x, windows along y."""
    frames = [synth.diffusion_frame(t, T=50, H=160, W=96) for t in (0, 25, 49)]
    res = run_gpu([f.image for f in frames], deriv_axis=1)
    for fr, (g, gs) in zip(frames, res):
        o, os_ = oracle_run(fr.image, deriv_axis=1)
        parity.check(g, gs, o, os_, TOL, parity.Window(fr.image, 32, 8, 1, 1, 0, 0.1), what="diffusion")
        v = (os_ == 0) & (gs == 0)
        inner = np.zeros_like(v)
        inner[:, 16:-16] = True
        parity.rms_check(g, o, fr.truth, v & inner, what="diffusion")


def test_batched_carrier_along_y():
    fr = synth.peaks_frame(np.inf, 0.1, H=48, W=256)
    img = np.ascontiguousarray(fr.image.T)
    (g, gs), = run_gpu([img], deriv_axis=1, carrier_axis=1)
    o, os_ = oracle_run(img, deriv_axis=1, carrier_axis=1)
    assert np.array_equal(gs, os_)
    v = os_ == 0
    assert np.abs(g[v].astype(np.float64) - o[v]).max() <= TOL


def test_uneven_batch_alone_equals_mix():
    """Frames of different sizes and windows in one launch give bit-identical maps to
    single-frame calls (the per-pixel arithmetic does not depend on the schedule)."""
    rng = np.random.default_rng(4)
    shapes = [(40, 96), (17, 300), (64, 64), (33, 129), (8, 512), (50, 77)]
    windows = [(32, 8), (24, 6), (48, 12), (32, 8), (16, 4), (24, 6)]
    frames = []
    for H, W in shapes:
        phi, _, _ = synth.gaussian_sum(rng, H, W)
        frames.append(synth.add_noise(synth.fringe(phi, 0.1), 0.03, rng).astype(np.float32))
    mix = run_gpu(frames, windows=windows)
    for f, w, (g, gs) in zip(frames, windows, mix):
        (ga, gsa), = run_gpu([f], window_len=w[0], cov_order=w[1])
        assert np.array_equal(gs, gsa)
        assert np.array_equal(np.isnan(g), np.isnan(ga))
        assert np.array_equal(g[~np.isnan(g)], ga[~np.isnan(ga)])
        o, os_ = oracle_run(f, w[0], w[1])
        parity.check(g, gs, o, os_, TOL, parity.Window(f, w[0], w[1], 1, 0, 0, 0.1), what=f"{f.shape} {w}")


@pytest.mark.parametrize("H,W", [(1, 64), (3, 31), (5, 33), (2, 1), (4, 20), (7, 97)])
def test_edge_shapes(H, W):
    rng = np.random.default_rng(H * 1000 + W)
    img = (0.5 + 0.4 * np.cos(TWO_PI * 0.1 * np.arange(W))[None, :] + 0.02 * rng.normal(size=(H, W))).astype(np.float32)
    for prec in ("batched", "plain_fp64"):
        (g, gs), = run_gpu([img], window_len=16, cov_order=4, precision=prec)
        o, os_ = oracle_run(img, 16, 4)
        tol = 1e-9 + 1e-7 if prec == "plain_fp64" else TOL  # 1e-7: the float32 map's rounding
        parity.check(g, gs, o, os_, tol, parity.Window(img, 16, 4, 1, 0, 0, 0.1), what=f"{H}x{W} {prec}")


def test_zero_frame_is_degenerate():
    img = np.zeros((4, 96), dtype=np.float32)
    for prec in ("batched", "plain_fp64", "plain_fp32"):
        (g, gs), = run_gpu([img], precision=prec)
        assert np.all(np.isnan(g))
        assert set(np.unique(gs)) <= {1, 2}
        assert (gs == 2).sum() == 4 * (96 - 32 + 1)


def test_pitch_and_offsets():
    """A frame read with a row pitch larger than its width equals the dense frame."""
    torch = _torch()
    fr = synth.peaks_frame(20, 0.1, H=16, W=200)
    padded = np.zeros((16, 256), dtype=np.float32)
    padded[:, :200] = fr.image
    dem = rmusic.Demodulator()
    try:
        buf = torch.from_numpy(np.concatenate([np.zeros(16, np.float32), padded.ravel()])).cuda()
        out = torch.empty(16 * 200, device="cuda")
        st = torch.empty(16 * 200, dtype=torch.uint8, device="cuda")
        d = rmusic.rmusic_frame_desc(16 * 4, 16, 200, 256, rmusic.RMUSIC_DTYPE_F32, 0, 0, 0)
        rmusic.rmusic_demodulate_frames(dem.ctx, buf.data_ptr(), [d], 1, out.data_ptr(), st.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        (g, gs), = run_gpu([fr.image])
        assert np.array_equal(out.cpu().numpy().reshape(16, 200), g, equal_nan=True)
    finally:
        dem.close()


def test_graph_replay_identical():
    torch = _torch()
    fr = synth.peaks_frame(20, 0.1, H=32, W=256)
    dem = rmusic.Demodulator(use_graph=1)
    try:
        x = _to_dev(fr.image)
        out = torch.empty(32 * 256, device="cuda")
        st = torch.empty(32 * 256, dtype=torch.uint8, device="cuda")
        dem.run(x, out=out, status=st)
        torch.cuda.synchronize()
        a = out.clone()
        assert dem.stats().graph_replayed == 0
        out.fill_(0)
        dem.run(x, out=out, status=st)
        torch.cuda.synchronize()
        assert dem.stats().graph_replayed == 1
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(out, nan=7.0))
        (g, gs), = run_gpu([fr.image])
        assert np.array_equal(out.cpu().numpy().reshape(32, 256), g, equal_nan=True)
    finally:
        dem.close()


def test_host_entry_matches_device_entry():
    import ctypes

    frames = [synth.peaks_frame(15, 0.1, H=20, W=160).image, synth.peaks_frame(np.inf, 0.1, H=12, W=96).image]
    flat = np.concatenate([f.ravel() for f in frames]).astype(np.float32)
    descs, nbytes, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_F32, 4)
    dem = rmusic.Demodulator()
    try:
        out = np.empty(nout, np.float32)
        st = np.empty(nout, np.uint8)
        rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, 2, out.ctypes.data,
                                             st.ctypes.data, None)
    finally:
        dem.close()
    dev = run_gpu(frames)
    o = 0
    for f, (g, gs) in zip(frames, dev):
        n = f.size
        assert np.array_equal(out[o:o + n].reshape(f.shape), g, equal_nan=True)
        assert np.array_equal(st[o:o + n].reshape(f.shape), gs)
        o += n


def test_hbm_budget_splits_batches_and_rejects_oversize():
    frames = [synth.peaks_frame(20, 0.1, H=32, W=128, stream=i).image for i in range(5)]
    ref = run_gpu(frames)
    one = 32 * 128 * 8
    torch = _torch()
    dem = rmusic.Demodulator(hbm_budget_bytes=one + 64 * 1024)
    try:
        out, st, shapes = dem.run([_to_dev(f) for f in frames])
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, np.concatenate([g.ravel() for g, _ in ref]), equal_nan=True)
    finally:
        dem.close()
    dem = rmusic.Demodulator(hbm_budget_bytes=4096)
    try:
        with pytest.raises(rmusic.RmusicError) as e:
            dem.run([_to_dev(frames[0])])
        assert e.value.code == rmusic.RMUSIC_ENOMEM
    finally:
        dem.close()


def test_reserve_allocates_once_and_respects_the_budget():
    """rmusic_reserve sizes the workspace for calls of up to (max_pixels, max_frames) in advance:
    later calls within the limits leave the workspace as it is (no allocation, hence no device
    synchronisation), their maps equal an unreserved context's, and a reservation over the budget
    is refused with ENOMEM and changes nothing."""
    frames = [synth.peaks_frame(20, 0.1, H=32 + 16 * i, W=128, stream=i).image for i in range(4)]
    ref = run_gpu(frames)
    total = sum(f.size for f in frames)
    torch = _torch()
    # room for the analytic signal of all four frames, the frame tables and the counters, not for
    # twice the pixels
    dem = rmusic.Demodulator(hbm_budget_bytes=8 * total + (64 << 10))
    try:
        dem.reserve(total, 8)
        held = dem.stats().workspace_bytes
        assert held >= 8 * total
        for k in range(1, 5):  # growing calls: 1, 2, 3, then all 4 frames
            out, st, _ = dem.run([_to_dev(f) for f in frames[:k]])
            torch.cuda.synchronize()
            assert dem.stats().workspace_bytes == held, k
        assert np.array_equal(out.cpu().numpy(), np.concatenate([g.ravel() for g, _ in ref]), equal_nan=True)
        with pytest.raises(rmusic.RmusicError) as e:
            dem.reserve(2 * total, 8)
        assert e.value.code == rmusic.RMUSIC_ENOMEM
        assert dem.stats().workspace_bytes == held
        with pytest.raises(rmusic.RmusicError) as e:
            rmusic.rmusic_reserve(dem.ctx, 16, -1)
        assert e.value.code == rmusic.RMUSIC_EINVAL
    finally:
        dem.close()


def test_invalid_descriptors_rejected():
    torch = _torch()
    dem = rmusic.Demodulator()
    try:
        buf = torch.zeros(1024, device="cuda")
        out = torch.empty(1024, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        for d, code in [
            (rmusic.rmusic_frame_desc(0, 0, 16, 0, 0, 0, 0, 0), rmusic.RMUSIC_EINVAL),
            (rmusic.rmusic_frame_desc(0, 4, 16, 8, 0, 0, 0, 0), rmusic.RMUSIC_EINVAL),
            (rmusic.rmusic_frame_desc(2, 4, 16, 0, 0, 0, 0, 0), rmusic.RMUSIC_EINVAL),
            (rmusic.rmusic_frame_desc(0, 4, 16, 0, 7, 0, 0, 0), rmusic.RMUSIC_EINVAL),
            (rmusic.rmusic_frame_desc(0, 4, 16, 0, 0, 0, 8, 12), rmusic.RMUSIC_EINVAL),
            (rmusic.rmusic_frame_desc(0, 4, 16, 0, 0, 0, 32, 7), rmusic.RMUSIC_EUNSUPPORTED),
            # 2^30 rows of two 512-pixel work items: 2^31 items, past the solvers' 32-bit item index
            # (rejected while the descriptors are checked, before anything is queued)
            (rmusic.rmusic_frame_desc(0, 1 << 30, 1024, 0, 0, 0, 0, 0), rmusic.RMUSIC_EUNSUPPORTED),
        ]:
            with pytest.raises(rmusic.RmusicError) as e:
                rmusic.rmusic_demodulate_frames(dem.ctx, buf.data_ptr(), [d], 1, out.data_ptr(), None, s)
            assert e.value.code == code
    finally:
        dem.close()


def test_full_size_frame_sampled_against_oracle():
    """1024 x 1024 frame in the bench's configuration (batched FP32, N = 32, L = 8): oracle values at
    sampled pixels, computed one by one."""
    rng = np.random.default_rng(0)
    for snr in (np.inf, 20):
        fr = synth.peaks_frame(snr, 0.1)
        (g, gs), = run_gpu([fr.image])
        ys = np.concatenate([rng.integers(0, 1024, 600), np.full(40, 1023), np.zeros(40, int)])
        xs = np.concatenate([rng.integers(0, 1024, 600), rng.integers(0, 1024, 80)])
        xs[:20] = np.arange(20) + 10  # around the left border
        o, os_, _ = O.demodulate_pixels(fr.image, O.make_params(32, 8, 1, 0, 0, 0.1), ys, xs)
        parity.check(g[ys, xs], gs[ys, xs], o, os_, TOL, parity.Window(fr.image, 32, 8, 1, 0, 0, 0.1), ys, xs,
                     what=f"1024^2 at {snr} dB")


def test_plain_fp32_and_polish64_accuracy():
    fr = synth.peaks_frame(np.inf, 0.1, H=24, W=256)
    o, os_ = oracle_run(fr.image)
    # the plain FP32 path has no higher-precision polish: near-double roots keep FP32 noise, and
    # its Aberth may stop at the iteration cap there (status 3, best estimate stored, checked too)
    for kw, tol in ((dict(precision="plain_fp32"), 5e-3), (dict(polish_fp64=1), 1e-4)):
        (g, gs), = run_gpu([fr.image], **kw)
        v = (os_ == 0) & ((gs == 0) | (gs == 3))
        assert v.sum() >= 0.99 * (os_ == 0).sum()
        d = np.abs(g[v].astype(np.float64) - o[v])
        assert d.max() <= tol, f"{kw}: max {d.max():.3e} p99.9 {np.quantile(d, 0.999):.3e}"


def test_launch_counts():
    fr = synth.peaks_frame(20, 0.1, H=16, W=128)
    dem = rmusic.Demodulator()
    try:
        dem.run(_to_dev(fr.image))
        assert dem.stats().kernel_launches == 2  # band-pass + one persistent solver launch
    finally:
        dem.close()
    dem = rmusic.Demodulator(precision="plain_fp32")
    try:
        dem.run([_to_dev(fr.image), _to_dev(fr.image)])
        assert dem.stats().kernel_launches == 3  # band-pass + one launch per frame
    finally:
        dem.close()


def _sampled_oracle(fr, N, L, deriv_axis, rows, cols):
    ys = np.repeat(np.asarray(rows), len(cols)).astype(np.int32)
    xs = np.tile(np.asarray(cols), len(rows)).astype(np.int32)
    p = O.make_params(N, L, 1, deriv_axis, 0, fr.carrier_freq)
    vals, st, _ = O.demodulate_pixels(fr.image, p, ys, xs)
    return ys, xs, vals, st


def test_diffusion_stack_full_frames_one_launch_sampled():
    """Diffusion time-lapse at full frame size (1024 x 1024 uint16, 12-bit), 32 frames spread over the
    500-frame schedule in one launch, windows along y; oracle at sampled pixels of four frames."""
    ts = np.linspace(0, 499, 32).astype(int)
    frames = [synth.diffusion_frame(int(t)) for t in ts]
    res = run_gpu([f.image for f in frames], deriv_axis=1)
    rng = np.random.default_rng(3)
    for i in (0, 11, 22, 31):
        fr, (g, gs) = frames[i], res[i]
        r0 = int(rng.integers(400, 560))
        rows = np.arange(r0, r0 + 24)                   # near the diffusion front
        cols = np.sort(rng.choice(1024, 40, replace=False))
        ys, xs, vals, st = _sampled_oracle(fr, 32, 8, 1, rows, cols)
        parity.check(g[ys, xs], gs[ys, xs], vals, st, TOL, parity.Window(fr.image, 32, 8, 1, 1, 0, 0.1), ys, xs,
                     what=f"diffusion frame {ts[i]}")
        v = (st == 0) & (gs[ys, xs] == 0)
        # accuracy against the closed-form derivative equals the oracle's
        parity.rms_check(g[ys, xs], vals, fr.truth[ys, xs], v, what=f"diffusion frame {ts[i]}")


def test_uneven_batch_full_sizes_one_launch_sampled():
    """64 frames with sizes drawn from {256..2048} x {256, 512, 1024} and (N, L) from
    {24, 32, 48} x {6, 8, 12}, SNR 15 dB, in one call; oracle at sampled pixels of every frame."""
    frames = synth.uneven_batch(64)
    windows = [(f.window_len, f.cov_order) for f in frames]
    res = run_gpu([f.image for f in frames], windows=windows)
    rng = np.random.default_rng(5)
    worst = 0.0
    gv, ov, tv = [], [], []
    for fr, (g, gs) in zip(frames, res):
        H, W = fr.image.shape
        rows = [int(rng.integers(0, H))]
        cols = np.sort(rng.choice(W, min(W, 24), replace=False))
        ys, xs, vals, st = _sampled_oracle(fr, fr.window_len, fr.cov_order, 0, rows, cols)
        rep = parity.check(g[ys, xs], gs[ys, xs], vals, st, TOL,
                           parity.Window(fr.image, fr.window_len, fr.cov_order, 1, 0, 0, fr.carrier_freq), ys, xs,
                           what=f"{H}x{W} N={fr.window_len} L={fr.cov_order}")
        worst = max(worst, rep["max"])
        v = (st == 0) & (gs[ys, xs] == 0)
        gv.append(g[ys, xs][v])
        ov.append(vals[v])
        tv.append(fr.truth[ys, xs][v])
    assert worst <= TOL, worst
    # accuracy against the closed-form derivative over every sampled pixel equals the oracle's
    g_all, o_all, t_all = np.concatenate(gv), np.concatenate(ov), np.concatenate(tv)
    parity.rms_check(g_all, o_all, t_all, np.ones(g_all.size, bool), what="uneven batch")


def test_autotune_variants_identical_and_cached(tmp_path, monkeypatch):
    """rmusic_autotune keeps one register-cap variant per covariance order and records it in the cache
    file named by RMUSIC_TUNE_CACHE; the tuned call's maps equal, bit for bit, those of a context
    pinned to the recorded variants (each variant is deterministic), and agree with the untuned
    default's to FP32 rounding with identical statuses."""
    import json

    torch = _torch()
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("RMUSIC_TUNE_CACHE", str(cache))
    frames = [synth.peaks_frame(10, 0.1, H=64, W=512).image, synth.peaks_frame(np.inf, 0.1, H=32, W=256).image]
    windows = [(32, 8), (24, 6)]
    descs, nbytes, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_F32, 4, windows)
    x = torch.from_numpy(np.concatenate([f.ravel() for f in frames])).cuda()
    s = torch.cuda.current_stream().cuda_stream

    def call(pin=None, tune=False):
        dem = rmusic.Demodulator()
        try:
            for L, v in (pin or {}).items():
                rmusic.rmusic_set_solver_variant(dem.ctx, L, v)
            out = torch.empty(nout, device="cuda")
            st = torch.empty(nout, dtype=torch.uint8, device="cuda")
            fn = rmusic.rmusic_autotune if tune else rmusic.rmusic_demodulate_frames
            fn(dem.ctx, x.data_ptr(), descs, 2, out.data_ptr(), st.data_ptr(), s)
            torch.cuda.synchronize()
            return out.cpu().numpy(), st.cpu().numpy()
        finally:
            dem.close()

    default = {8: 0, 6: 1}  # the untuned variants (batched_variants.h)
    ref, ref_st = call(pin=default)
    tuned, tuned_st = call(tune=True)
    again, again_st = call()  # the tuned choice, taken from this process's tuning
    lines = [json.loads(l) for l in cache.read_text().strip().splitlines()]
    chosen = {int(d["L"]): int(d["variant"]) for d in lines}
    assert set(chosen) == {6, 8}
    pinned, pinned_st = call(pin=chosen)
    assert np.array_equal(tuned, pinned, equal_nan=True) and np.array_equal(tuned_st, pinned_st)
    assert np.array_equal(again, pinned, equal_nan=True) and np.array_equal(again_st, pinned_st)
    assert np.array_equal(tuned_st, ref_st)
    ok = ref_st == 0
    assert np.abs(tuned[ok] - ref[ok]).max() <= 3e-5


@pytest.mark.parametrize("L", [4, 6, 8])
def test_solver_variants_and_warp_per_matrix_schedule(L):
    """Variants 0-2 (register caps) run the same source; the compiler's instruction selection (which
    multiply-adds it fuses) may differ between them, so their maps agree to the FP32 rounding of the
    estimator, which small L (a flat pseudospectrum minimum) magnifies to ~1e-5 rad/px in the angle.
    Variant 3 runs the eigenvalue sweeps with one warp per matrix followed by inverse iteration, the
    others the power iteration, which stops at a 1e-6 step: the two eigenvectors agree to ~1e-6, with
    the same magnification. Statuses are identical throughout."""
    torch = _torch()
    frames = [synth.peaks_frame(10, 0.1, H=40, W=256).image, synth.peaks_frame(np.inf, 0.1, H=24, W=256).image]
    x = torch.from_numpy(np.concatenate([f.ravel() for f in frames])).cuda()
    descs, _, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_F32, 4)
    maps = []
    dem = rmusic.Demodulator(cov_order=L)
    try:
        for v in range(4):
            rmusic.rmusic_set_solver_variant(dem.ctx, L, v)
            out = torch.empty(nout, device="cuda")
            st = torch.empty(nout, dtype=torch.uint8, device="cuda")
            rmusic.rmusic_demodulate_frames(dem.ctx, x.data_ptr(), descs, 2, out.data_ptr(), st.data_ptr(), None)
            torch.cuda.synchronize()
            assert dem.stats().solver_variant == v
            maps.append((out.cpu().numpy(), st.cpu().numpy()))
        with pytest.raises(rmusic.RmusicError):
            rmusic.rmusic_set_solver_variant(dem.ctx, L, 4)
    finally:
        dem.close()
    for v in (0, 2):
        assert np.array_equal(maps[v][1], maps[1][1])
        ok = maps[1][1] == 0
        assert np.array_equal(np.isnan(maps[v][0]), np.isnan(maps[1][0]))
        assert np.abs(maps[v][0][ok] - maps[1][0][ok]).max() <= 3e-5
    g, gs = maps[3]
    assert np.array_equal(gs, maps[1][1])
    ok = gs == 0
    assert np.abs(g[ok] - maps[1][0][ok]).max() <= 3e-5
    o, os_ = oracle_run(frames[1], 32, L, 1)
    off = frames[0].size
    v = (os_.ravel() == 0) & (gs[off:] == 0)
    assert np.abs(g[off:][v] - o.ravel()[v]).max() <= 1e-4


def test_host_entry_pinned_buffers_in_place_equal_device_entry():
    """Pinned host buffers are read and written by the kernels in place (no staging copies); the
    maps and statuses equal the device entry's, and so do those of a staged (pageable) call."""
    torch = _torch()
    frames = [synth.peaks_frame(10, 0.1, H=33, W=1024).image, synth.peaks_frame(np.inf, 0.1, H=20, W=300).image]
    flat = np.concatenate([f.ravel() for f in frames]).astype(np.float32)
    descs, nbytes, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_F32, 4)
    hin = torch.from_numpy(flat).pin_memory()
    hout = torch.full((nout,), 7.0).pin_memory()
    hst = torch.full((nout,), 9, dtype=torch.uint8).pin_memory()
    dem = rmusic.Demodulator(use_graph=1)
    try:
        for _ in range(2):  # the second call replays the captured graph with the host pointers
            rmusic.rmusic_demodulate_frames_host(dem.ctx, hin.data_ptr(), nbytes, descs, 2, hout.data_ptr(),
                                                 hst.data_ptr(), None)
        pout = np.empty(nout, np.float32)
        pst = np.empty(nout, np.uint8)
        rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, 2, pout.ctypes.data,
                                             pst.ctypes.data, None)
    finally:
        dem.close()
    dev = run_gpu(frames)
    o = 0
    for f, (g, gs) in zip(frames, dev):
        n = f.size
        assert np.array_equal(hout.numpy()[o:o + n].reshape(f.shape), g, equal_nan=True)
        assert np.array_equal(hst.numpy()[o:o + n].reshape(f.shape), gs)
        assert np.array_equal(pout[o:o + n].reshape(f.shape), g, equal_nan=True)
        assert np.array_equal(pst[o:o + n].reshape(f.shape), gs)
        o += n


def test_host_entry_statistics_and_graph_owned_timing_events():
    """The host entry's statistics describe its call: the pixel count, one band-pass and one solver
    launch, the iteration means of the device entry (work items sit at the same absolute
    positions), positive stage timers, also when the call replays a captured graph. With a budget
    that splits a call into groups, each group's graph records its own timing events: calls that
    capture new graphs while replaying older ones in the same call keep positive timers no larger
    than the wall time of the call."""
    import time

    torch = _torch()
    shapes = [(40, 256), (24, 512), (64, 128), (16, 1024), (33, 300)]
    frames = [synth.peaks_frame(12, 0.1, H=h, W=w, stream=i).image for i, (h, w) in enumerate(shapes)]
    flat = np.concatenate([f.ravel() for f in frames]).astype(np.float32)
    descs, nbytes, nout = rmusic.frame_descs(shapes, rmusic.RMUSIC_DTYPE_F32, 4)
    hin = torch.from_numpy(flat).pin_memory()
    hout = torch.full((nout,), 7.0).pin_memory()
    dev = run_gpu(frames)
    ddem = rmusic.Demodulator(timing=1)
    try:
        ddem.run([_to_dev(f) for f in frames])
        torch.cuda.synchronize()
        dst = ddem.stats()
    finally:
        ddem.close()
    for graph in (0, 1):
        dem = rmusic.Demodulator(use_graph=graph, timing=1)
        try:
            for _ in range(2):
                rmusic.rmusic_demodulate_frames_host(dem.ctx, hin.data_ptr(), nbytes, descs, len(frames),
                                                     hout.data_ptr(), None, None)
                st = dem.stats()
                assert st.pixels == sum(h * w for h, w in shapes)
                assert st.kernel_launches == 2
                assert st.bandpass_ms > 0 and st.solver_ms > 0
                assert st.mean_power_steps == dst.mean_power_steps
                assert st.mean_newton_steps == dst.mean_newton_steps
            assert st.graph_replayed == graph
            o = 0
            for f, (g, gs) in zip(frames, dev):
                assert np.array_equal(hout.numpy()[o:o + f.size].reshape(f.shape), g, equal_nan=True)
                o += f.size
        finally:
            dem.close()
    # budget for about two frames' analytic signal: calls split into groups, one graph per group
    dem = rmusic.Demodulator(use_graph=1, timing=1, hbm_budget_bytes=8 * 2 * 64 * 128 + (64 << 10))
    try:
        dframes = [_to_dev(f) for f in frames[:3]]
        for order in ([0, 1, 2], [2, 1, 0], [0, 1, 2], [1, 2, 0]):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dem.run([dframes[i] for i in order])
            torch.cuda.synchronize()
            wall_ms = 1e3 * (time.perf_counter() - t0)
            st = dem.stats()
            assert 0 < st.bandpass_ms < wall_ms and 0 < st.solver_ms < wall_ms, (order, st.bandpass_ms,
                                                                                st.solver_ms, wall_ms)
    finally:
        dem.close()


def test_host_entry_async_double_buffered_equals_sync():
    """The asynchronous host entry queues the call and returns; once its stream is synchronised the
    maps equal the synchronous entry's (pinned buffers, maps written in place; pageable buffers,
    staged). Two contexts on two streams, alternated with two calls in flight, give every step its
    own correct maps."""
    torch = _torch()
    shapes = [(40, 256), (24, 512)]
    steps = [[synth.peaks_frame(snr, 0.1, H=h, W=w, stream=k).image for h, w in shapes]
             for k, snr in enumerate((30.0, 10.0, np.inf, 5.0, 20.0))]
    descs, nbytes, nout = rmusic.frame_descs(shapes, rmusic.RMUSIC_DTYPE_F32, 4)
    ref = []
    dem = rmusic.Demodulator()
    try:
        for fr in steps:
            flat = np.concatenate([f.ravel() for f in fr]).astype(np.float32)
            out = np.empty(nout, np.float32)
            rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, 2, out.ctypes.data, None, None)
            ref.append(out)
    finally:
        dem.close()
    hins = [torch.from_numpy(np.concatenate([f.ravel() for f in fr]).astype(np.float32)).pin_memory() for fr in steps]
    houts = [torch.full((nout,), 7.0).pin_memory() for _ in steps]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    dems = [rmusic.Demodulator(use_graph=1), rmusic.Demodulator(use_graph=1)]
    try:
        for k in range(len(steps)):
            i = k % 2
            streams[i].synchronize()  # this context's previous call is complete
            rmusic.rmusic_demodulate_frames_host_async(dems[i].ctx, hins[k].data_ptr(), nbytes, descs, 2,
                                                       houts[k].data_ptr(), None, streams[i].cuda_stream)
        for st in streams:
            st.synchronize()
        for k in range(len(steps)):
            assert np.array_equal(houts[k].numpy(), ref[k], equal_nan=True), k
        # pageable buffers
        flat = np.concatenate([f.ravel() for f in steps[1]]).astype(np.float32)
        pout = np.empty(nout, np.float32)
        rmusic.rmusic_demodulate_frames_host_async(dems[0].ctx, flat.ctypes.data, nbytes, descs, 2, pout.ctypes.data,
                                                   None, streams[0].cuda_stream)
        streams[0].synchronize()
        assert np.array_equal(pout, ref[1], equal_nan=True)
    finally:
        for d in dems:
            d.close()
