"""GPU parity of model order p > 1 on raw real fringes (no band-pass; the line minus its mean)
against the FP64 oracle: the plain FP64 path to float32 output resolution, the plain FP32 path
within 1e-4 on noise-free inputs and within 1 % RMS under noise, and the FP32-batched model-order
solver with status maps equal to the oracle's, max |GPU - oracle| <= 1e-4 rad/px under noise (a
selected root with a near-double neighbour, beyond FP32's resolution, excused and bounded) and RMS
within 1 %."""
import numpy as np
import pytest

import oracle as O
import parity
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


# ---- the FP32-batched model-order solver (batched_p_kernel.cuh) ------------------------------------
def _fringe_rows(H, W, snr, offset, f=0.1, seed=0):
    """Raw real fringe a + b cos(2 pi f x + phi) along rows, phi smooth; with a local offset step."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    phi = 1.2 * np.sin(x / 37.0 + 0.3 * y / H) + 0.015 * y
    img = 0.5 + offset * (x > W // 3) + 0.4 * np.cos(TWO_PI * f * x + phi)
    if np.isfinite(snr):
        img = img + synth.sigma_for_snr(0.4, snr) * rng.normal(size=(H, W))
    truth = 1.2 * np.cos(x / 37.0 + 0.3 * y / H) / 37.0
    return img.astype(np.float32), truth


def _oracle_roots_p(w, L, p, fb, omega_ref):
    """The oracle's selected root of one window and all roots of its polynomial (model order p)."""
    r = O.window_derivative_p(w, L, p, fb, omega_ref)
    R = O.covariance(w, L, fb)
    ev, V, _ = O.eig_hermitian(R)
    C = np.eye(L, dtype=complex)
    for j in np.argsort(ev)[::-1][:p]:
        C -= np.outer(V[:, j], V[:, j].conj()) / np.vdot(V[:, j], V[:, j]).real
    q = np.array([np.trace(C, offset=k) for k in range(-(L - 1), L)])
    return r["zsel"], np.roots(q[::-1])


def _check_p(g, gs, o, os_, img, N, L, fb, p, what, tol=1e-4, max_excused=1e-3):
    """Statuses equal (two bounded exceptions below); |GPU - oracle| <= tol where both are ok, except where the oracle's selected root
    has another root (not its own mirror) within 4e-3: FP32 resolves such a pair only to about
    eps / separation, and the GPU's value must then lie within the pair's separation of the oracle's.
    Such pixels may be at most max_excused of those compared."""
    d = np.abs((g.astype(np.float64) - o + np.pi) % TWO_PI - np.pi)
    x_ = img.astype(np.float64) - img.mean(axis=1, keepdims=True)
    wref = TWO_PI * 0.1
    # status disagreements: only "not converged" on the GPU (an FP32 iteration cap; the value is
    # stored and must still agree) or "degenerate" where the oracle's own eigen-gap is below 1e-5 l1
    assert np.array_equal(gs == 1, os_ == 1), f"{what}: border maps differ"
    diff = np.argwhere(gs != os_)
    for y, x in diff:
        if gs[y, x] == 3 and os_[y, x] == 0:
            assert d[y, x] <= tol, f"{what}: pixel {(y, x)} not converged and off by {d[y, x]:.3e}"
        else:
            assert gs[y, x] == 2 and os_[y, x] == 0, f"{what}: pixel {(y, x)} status {gs[y, x]} vs {os_[y, x]}"
            w = x_[y, x - N // 2: x - N // 2 + N].astype(complex)
            ev = np.sort(np.linalg.eigvalsh(O.covariance(w, L, fb)))[::-1]
            assert ev[p - 1] - ev[p] <= 1e-5 * ev[0], f"{what}: pixel {(y, x)} degenerate, oracle gap {ev[p - 1] - ev[p]:.3e}"
    both = (gs == 0) & (os_ == 0)
    bad = np.argwhere(both & (d > tol))
    for y, x in bad:
        w = x_[y, x - N // 2: x - N // 2 + N].astype(complex)
        z, roots = _oracle_roots_p(w, L, p, fb, wref)
        others = roots[(np.abs(roots - z) > 1e-12) & (np.abs(roots - 1 / np.conj(z)) > 1e-9)]
        sep = np.abs(others - z).min()
        assert sep < 4e-3 and d[y, x] <= sep, f"{what}: pixel {(y, x)} off by {d[y, x]:.3e}, separation {sep:.3e}"
    assert len(bad) + len(diff) <= max_excused * both.sum(), f"{what}: {len(bad)} + {len(diff)} excused of {both.sum()}"
    return len(bad) + len(diff)


# Shapes from L = p + 3 up. With a noise subspace of one or two dimensions (L = p + 1, p + 2) Q's
# roots crowd into near-double pairs about the circle, which float32 coefficients resolve only to a
# few 1e-4 rad (measured on the GPU: up to 3.2e-4 at p = 3, L = 5 and at p = 2, L = 3); those
# shapes are outside this bar.
@pytest.mark.parametrize("p,fb,N,L,offset", [(2, 1, 32, 8, 0.0), (2, 0, 32, 8, 0.0), (3, 1, 32, 8, 0.25),
                                             (3, 0, 24, 6, 0.25), (2, 1, 21, 7, 0.0), (2, 1, 48, 12, 0.0),
                                             (3, 1, 20, 6, 0.3), (2, 0, 16, 5, 0.0)])
def test_batched_model_order_matches_oracle(p, fb, N, L, offset, tol=1e-4):
    """Status maps equal to the oracle's and max |GPU - oracle| <= tol rad/px on every pixel both
    call ok (near-double roots aside, see _check_p), at 20 and 10 dB; RMS error against the
    closed-form derivative within 1 % of the oracle's."""
    for snr, seed in ((20.0, 1), (10.0, 2)):
        img, truth = _fringe_rows(16, 320, snr, offset, seed=seed)
        g, st = run(img, window_len=N, cov_order=L, model_order=p, raw_input=1, carrier_freq=0.1,
                    forward_backward=fb, precision="batched")
        o, ost, _ = O.demodulate(img, O.make_params(N, L, fb, 0, 0, 0.1, model_order=p, raw_input=1))
        _check_p(g, st, o, ost, img, N, L, fb, p, what=f"p={p} fb={fb} N={N} L={L} {snr} dB", tol=tol)
        m = (st == 0) & (ost == 0)
        m[:, :N] = False
        m[:, -N:] = False
        parity.rms_check(g, o, truth, m, what=f"p={p} fb={fb} N={N} L={L} {snr} dB")


def test_batched_model_order_noise_free_closed_form():
    """A noise-free cosine puts p double roots on the circle; the selected one's angle is the local
    frequency minus the carrier (pixels the root finder's sweep cap ends carry status 3 and the best
    estimate, which must be right as well)."""
    H, W, f, f0 = 8, 256, 32 / 256, 0.1
    y, x = np.mgrid[0:H, 0:W]
    clean = (0.5 + 0.4 * np.cos(TWO_PI * f * x + 0.2 * y)).astype(np.float32)
    for fb in (1, 0):
        g, st = run(clean, window_len=32, cov_order=8, model_order=2, raw_input=1, carrier_freq=f0,
                    forward_backward=fb, precision="batched")
        v = (st == 0) | (st == 3)
        assert v.sum() == H * (W - 31), np.bincount(st.ravel(), minlength=4)
        assert np.abs(g[v] - TWO_PI * (f - f0)).max() <= 1e-4, np.bincount(st.ravel(), minlength=4)


def test_batched_model_order_mix_equals_alone_and_rejections():
    """Frames of different sizes and windows in one call give the maps they give alone, bit for bit;
    complex frames (the solver takes R as real symmetric) and inputs that are not raw are refused."""
    torch = _torch()
    rng = np.random.default_rng(4)
    shapes = [(9, 200), (17, 96), (4, 512)]
    windows = [(32, 8), (24, 6), (32, 8)]
    frames = []
    for H, W in shapes:
        img, _ = _fringe_rows(H, W, 15.0, 0.2, seed=int(rng.integers(100)))
        frames.append(img)
    dem = rmusic.Demodulator(model_order=3, raw_input=1, carrier_freq=0.1, precision="batched")
    try:
        tens = [torch.from_numpy(f).cuda() for f in frames]
        out, st, shp = dem.run(tens, windows=windows)
        torch.cuda.synchronize()
        out, st = out.cpu().numpy(), st.cpu().numpy()
    finally:
        dem.close()
    o = 0
    for f, w, (H, W) in zip(frames, windows, shp):
        ga, sa = run(f, window_len=w[0], cov_order=w[1], model_order=3, raw_input=1, carrier_freq=0.1,
                     precision="batched")
        assert np.array_equal(st[o:o + H * W].reshape(H, W), sa)
        assert np.array_equal(out[o:o + H * W].reshape(H, W), ga, equal_nan=True)
        o += H * W
    with pytest.raises(rmusic.RmusicError):
        rmusic.Demodulator(model_order=2, raw_input=0, carrier_freq=0.1, precision="batched")
    dem = rmusic.Demodulator(model_order=2, raw_input=1, carrier_freq=0.1, precision="batched")
    try:
        with pytest.raises(rmusic.RmusicError):
            dem.run(torch.zeros(4, 64, dtype=torch.complex64, device="cuda"))
    finally:
        dem.close()


def test_batched_model_order_columns_uint16_and_fp64_step():
    """Column windows (carrier and windows along y), 12-bit uint16 frames, and the optional FP64
    step (on Q itself): statuses equal to the oracle's and max |GPU - oracle| <= 1e-4 rad/px."""
    rng = np.random.default_rng(21)
    y, x = np.mgrid[0:320, 0:24]
    phi = 1.2 * np.sin(y / 37.0 + 0.3 * x / 24) + 0.015 * x
    real = 0.5 + 0.2 * (y > 100) + 0.4 * np.cos(TWO_PI * 0.1 * y + phi) + synth.sigma_for_snr(0.4, 20.0) * rng.normal(size=y.shape)
    u16 = np.clip(np.round(real * 3000.0), 0, 4095).astype(np.uint16)
    for p in (2, 3):
        for polish in (0, 1):
            g, st = run_u16_cols(u16, p, polish)
            o, ost, _ = O.demodulate(u16, O.make_params(32, 8, 1, 1, 1, 0.1, model_order=p, raw_input=1))
            _check_p_cols(g, st, o, ost, what=f"columns uint16 p={p} fp64={polish}")


def run_u16_cols(u16, p, polish):
    torch = _torch()
    dem = rmusic.Demodulator(window_len=32, cov_order=8, model_order=p, raw_input=1, carrier_freq=0.1,
                             carrier_axis=1, deriv_axis=1, polish_fp64=polish, precision="batched")
    try:
        t16 = torch.from_numpy(u16.astype(np.int16)).cuda()
        out, st, _ = dem.run(t16)
        torch.cuda.synchronize()
    finally:
        dem.close()
    return out.cpu().numpy().reshape(u16.shape), st.cpu().numpy().reshape(u16.shape)


def _check_p_cols(g, gs, o, os_, what, tol=1e-4):
    assert np.array_equal(gs, os_), f"{what}: status maps differ at {int((gs != os_).sum())} pixels"
    both = (gs == 0) & (os_ == 0)
    d = np.abs((g.astype(np.float64) - o + np.pi) % TWO_PI - np.pi)
    assert both.sum() > 0 and d[both].max() <= tol, f"{what}: max {d[both].max():.3e}"


@pytest.mark.parametrize("fb,N,L", [(1, 32, 8), (0, 24, 6), (1, 48, 12)])
def test_batched_model_order_two_certified_equals_exhaustive(fb, N, L):
    """p = 2: the certified Newton root (the conjugate pair proven the two inner roots nearest the
    circle by a Schur-Cohn count) selects what the full root finder selects, to FP32 resolution, and
    decides nearly every lane."""
    torch = _torch()
    img, _ = _fringe_rows(16, 320, 15.0, 0.0, seed=5)
    res = {}
    for ex in (0, 1):
        dem = rmusic.Demodulator(window_len=N, cov_order=L, model_order=2, raw_input=1, carrier_freq=0.1,
                                 forward_backward=fb, precision="batched", exhaustive=ex)
        try:
            out, st, _ = dem.run(torch.from_numpy(img).cuda())
            torch.cuda.synchronize()
            res[ex] = (out.cpu().numpy(), st.cpu().numpy(), dem.stats())
        finally:
            dem.close()
    (g0, s0, st0), (g1, s1, st1) = res[0], res[1]
    assert np.array_equal(s0, s1)
    v = s0 == 0
    assert np.abs((g0[v].astype(np.float64) - g1[v] + np.pi) % TWO_PI - np.pi).max() <= 2e-5
    assert st1.root_fallback_frac == 1.0 and st0.root_fallback_frac <= 0.1 and st0.mean_newton_steps >= 1.0
