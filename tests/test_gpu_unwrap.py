"""GPU parity of phase assembly (Sec. 3: the local phases are unwrapped with the reliability-sorting
method the paper cites) against the oracle's sequential implementation of that method.

Both sides read the same float32 wrapped maps (drawn here, not produced by the GPU) and take the
reliabilities and 2 pi jumps in float32, so the integer jump maps must agree exactly once every
region is anchored at its first pixel (row-major), which is how the library reports them.
"""
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


def _wrapf(a):
    return ((np.asarray(a, dtype=np.float64) + np.pi) % TWO_PI - np.pi).astype(np.float32)


def _anchored_k(k, valid):
    """k of every 4-connected region of valid pixels minus k at the region's first pixel."""
    from scipy import ndimage

    lab, n = ndimage.label(valid, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    out = np.zeros_like(k, dtype=np.int64)
    flat_lab = lab.ravel()
    first = {}
    for idx in np.flatnonzero(flat_lab):
        first.setdefault(flat_lab[idx], idx)
    kf = k.ravel().astype(np.int64)
    for r, idx in first.items():
        m = flat_lab == r
        out.ravel()[m] = kf[m] - kf[idx]
    return out


def gpu_unwrap(maps, in_place=False, launched_rounds=-1):
    torch = _torch()
    dem = rmusic.Demodulator(geometry="square", half_width=1)
    try:
        flat = torch.from_numpy(np.concatenate([m.ravel() for m in maps]).astype(np.float32)).cuda()
        descs, _, n = rmusic.frame_descs([m.shape for m in maps], rmusic.RMUSIC_DTYPE_F32, 4)
        out = flat if in_place else torch.empty_like(flat)
        if launched_rounds == -1:
            rmusic.rmusic_unwrap_phase(dem.ctx, flat.data_ptr(), descs, len(maps), out.data_ptr(), None)
        else:
            rmusic.rmusic_unwrap_phase_sched(dem.ctx, flat.data_ptr(), descs, len(maps), out.data_ptr(),
                                             launched_rounds, None)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        res, off = [], 0
        for m in maps:
            res.append(o[off:off + m.size].reshape(m.shape))
            off += m.size
        st = dem.stats()
        assert st.wait_timeouts == 0  # no grid-wide wait of the cooperative rounds gave up
        return res, st.kernel_launches
    finally:
        dem.close()


def _check_exact(w, u_gpu):
    valid = ~np.isnan(w)
    assert np.array_equal(np.isnan(u_gpu), ~valid)
    kg = np.round((u_gpu.astype(np.float64) - w) / TWO_PI)
    kg[~valid] = 0
    assert np.abs((u_gpu[valid] - w[valid]) - TWO_PI * kg[valid]).max() < 1e-3
    _, ko, _ = O.unwrap(w)
    assert np.array_equal(_anchored_k(kg.astype(np.int64), valid), _anchored_k(ko, valid))
    # the library anchors every region at its first pixel
    assert np.array_equal(kg.astype(np.int64), _anchored_k(kg.astype(np.int64), valid))


@pytest.mark.parametrize("seed", range(3))
def test_unwrap_noisy_maps_match_oracle_exactly(seed):
    """Noisy maps with residues: the result depends on the edge order, so this checks the whole
    method (reliabilities, order, jumps), not just integration."""
    rng = np.random.default_rng(100 + seed)
    H, W = 70 + 13 * seed, 97
    y, x = np.mgrid[0:H, 0:W]
    w = _wrapf(0.07 * (x - 40) ** 2 / 9 + 0.3 * y + rng.normal(0, 0.9, (H, W)))
    (u,), launches = gpu_unwrap([w])
    assert launches > 10
    _check_exact(w, u)


def test_unwrap_batch_uneven_with_holes_and_in_place():
    rng = np.random.default_rng(7)
    maps = []
    for H, W in [(33, 40), (1, 50), (64, 17), (5, 5), (90, 120)]:
        y, x = np.mgrid[0:H, 0:W]
        m = _wrapf(0.4 * x - 0.25 * y + rng.normal(0, 0.6, (H, W)))
        if H > 30:
            m[:, W // 2] = np.nan           # splits the frame into two regions
            m[rng.random((H, W)) < 0.03] = np.nan
        maps.append(m)
    maps[3][:] = np.nan                     # a frame without values
    res, _ = gpu_unwrap(maps)
    res2, _ = gpu_unwrap(maps, in_place=True)
    for w, u, u2 in zip(maps, res, res2):
        assert np.array_equal(u, u2, equal_nan=True)
        if np.isnan(w).all():
            assert np.isnan(u).all()
            continue
        _check_exact(w, u)


def test_unwrap_smooth_large_frame_recovers_phase():
    H, W = 1024, 1536
    y, x = np.mgrid[0:H, 0:W]
    phi = 40.0 * np.exp(-((x - 700.0) ** 2 + (y - 500.0) ** 2) / (2 * 300.0 ** 2)) + 0.01 * x
    w = _wrapf(phi)
    (u,), _ = gpu_unwrap([w])
    d = (u.astype(np.float64) - phi) / TWO_PI
    assert np.abs(d - np.round(d[0, 0])).max() < 1e-4
    assert np.round(d[0, 0]) == np.round((w[0, 0] - phi[0, 0]) / TWO_PI)  # first pixel keeps its value


def test_unwrap_full_size_noisy_matches_oracle():
    rng = np.random.default_rng(3)
    H = W = 1024
    y, x = np.mgrid[0:H, 0:W]
    w = _wrapf(10 * np.sin(x / 150.0) * np.cos(y / 200.0) + rng.normal(0, 0.7, (H, W)))
    (u,), _ = gpu_unwrap([w])
    _check_exact(w, u)


def test_square_path_with_unwrap_map():
    """The fourth map of the square geometry (unwrap = 1) is the unwrapped alpha map: on a 20 dB
    complex fringe it reproduces the phase up to one 2 pi multiple and equals the oracle's
    unwrapping of its own alpha map (the unwrapping is unique there)."""
    torch = _torch()
    fr = synth.complex_fringe_frame(20.0, H=200, W=240, hi=30.0)
    Lp = 4
    dem = rmusic.Demodulator(geometry="square", half_width=Lp, carrier_freq=0.0, unwrap=1)
    try:
        out, st, _ = dem.run(torch.from_numpy(fr.image).cuda())
        torch.cuda.synchronize()
    finally:
        dem.close()
    maps = out.cpu().numpy().reshape(4, 200, 240)
    alpha, phase = maps[2], maps[3]
    valid = ~np.isnan(alpha)
    assert np.array_equal(np.isnan(phase), ~valid)
    k = np.round((phase.astype(np.float64) - alpha) / TWO_PI)
    assert np.abs(phase[valid] - alpha[valid] - TWO_PI * k[valid]).max() < 1e-3
    d = phase[valid].astype(np.float64) - fr.meta["phi"][valid]
    assert np.abs(d - np.median(d)).max() < 0.5  # no 2 pi slips anywhere
    _, _, oal, ost, _ = O.square_demodulate(fr.image, O.make_params(carrier_freq=0.0), Lp)
    _, ko, _ = O.unwrap(oal.astype(np.float32))
    assert np.array_equal(k[valid].astype(np.int64), _anchored_k(ko, ~np.isnan(oal))[valid])


@pytest.mark.parametrize("launched", [0, 1, 3, 64])
def test_unwrap_schedules_agree(launched):
    """Every split of the global rounds between separate launches and the cooperative kernel gives
    the default's maps bit for bit (0: every round cooperative; 64: every round launched), on
    noisy maps with residues of uneven sizes in one call, and the oracle's values."""
    rng = np.random.default_rng(300)
    maps = []
    for H, W in ((96, 130), (41, 77), (128, 64)):
        y, x = np.mgrid[0:H, 0:W]
        w = _wrapf(0.05 * (x - 30) ** 2 / 7 + 0.4 * y + rng.normal(0, 1.0, (H, W)))
        w[rng.random((H, W)) < 0.03] = np.nan
        maps.append(w)
    ref, n_ref = gpu_unwrap(maps)
    got, n_got = gpu_unwrap(maps, launched_rounds=launched)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b, equal_nan=True)
    for w, u in zip(maps, got):
        _check_exact(w, u)
    if launched == 0:
        assert n_got == 6  # prepare, reliabilities, tiles, the cooperative rounds, anchors, output
