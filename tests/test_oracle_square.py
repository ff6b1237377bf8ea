"""Pins for the oracle's square-block geometry (the paper's own: a (2Lp+1) x (2Lp+1) block whose
columns are the snapshots of the y analysis and whose conjugated rows are those of the x analysis;
Sec. 3, Eq. 4-15, Algorithm 1). Each test checks the oracle against something other than itself:
the closed form of a noise-free plane wave, the library SVD the paper uses, an independent
evaluation of Eq. 12-13 through the pseudospectrum on the unit circle, the least-squares property
of Eq. 15's alpha, and exact symmetries of the estimator.
"""
import numpy as np
import pytest

import oracle as O

TWO_PI = 2 * np.pi


def _wrap(a):
    return (np.asarray(a) + np.pi) % TWO_PI - np.pi


def _plane_block(Lp, wx, wy, a0, amp=1.0):
    y, x = np.mgrid[-Lp:Lp + 1, -Lp:Lp + 1]
    return amp * np.exp(1j * (a0 + wx * x + wy * y))


def _noisy_block(Lp, seed, sigma=0.6):
    rng = np.random.default_rng(seed)
    M = 2 * Lp + 1
    G = _plane_block(Lp, rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(-3, 3))
    return G + sigma * (rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M)))


# ----------------------------------------------------------------------------------------------
# Closed form: a noise-free plane wave A exp(j(alpha + wx x + wy y)) (Eq. 2-8) makes both
# auto-correlation matrices rank one; the estimator returns (wx, wy, alpha) exactly.
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("Lp", [1, 2, 3, 5, 7, 8])
def test_square_plane_wave_exact(Lp):
    for wx, wy, a0 in [(0.7, -0.4, 1.1), (-2.5, 0.3, -3.0), (0.05, 2.9, 0.0), (-1.2, -2.2, 2.5)]:
        r = O.square_window(_plane_block(Lp, wx, wy, a0, amp=0.37))
        assert r["status"] == O.STATUS_OK
        assert abs(r["wx"] - wx) < 1e-9 and abs(r["wy"] - wy) < 1e-9
        assert abs(_wrap(r["alpha"] - a0)) < 1e-9
        # z_y = exp(j wy) and z_x = exp(-j wx) (the paper's sign convention for x, Eq. 13-15)
        assert abs(r["zy"] - np.exp(1j * wy)) < 1e-7 and abs(r["zx"] - np.exp(-1j * wx)) < 1e-7


@pytest.mark.parametrize("carrier_axis", [0, 1])
def test_square_real_fringe_with_carrier_exact(carrier_axis):
    """Real fringe 0.5 + 0.4 cos(2 pi f X + wy Y + theta), periodic along the carrier axis so the
    band-pass is exact: derivative along the carrier 2 pi (f - f0), across it wy, alpha the fringe
    phase with the carrier's 2 pi f0 X removed."""
    H, W, f, f0, wy, th = 48, 128, 16 / 128, 0.1, 0.3, 0.4
    y, x = np.mgrid[0:H, 0:W]
    phase = TWO_PI * f * x + wy * y + th
    img = 0.5 + 0.4 * np.cos(phase)
    exp_dx, exp_dy = TWO_PI * (f - f0), wy
    exp_alpha = _wrap(TWO_PI * (f - f0) * x + wy * y + th)
    if carrier_axis == 1:
        img, exp_alpha = img.T.copy(), exp_alpha.T
        exp_dx, exp_dy = exp_dy, exp_dx
    p = O.make_params(carrier_axis=carrier_axis, carrier_freq=f0)
    Lp = 3
    dx, dy, al, st, _ = O.square_demodulate(img, p, Lp)
    valid = st == O.STATUS_OK
    assert valid.sum() == (img.shape[0] - 2 * Lp) * (img.shape[1] - 2 * Lp)
    assert np.abs(dx[valid] - exp_dx).max() < 1e-9
    assert np.abs(dy[valid] - exp_dy).max() < 1e-9
    assert np.abs(_wrap(al[valid] - exp_alpha[valid])).max() < 1e-9


def test_square_border_pixels():
    """A pixel whose block leaves the frame is a border pixel (Sec. 4): NaN in every map."""
    rng = np.random.default_rng(5)
    img = rng.normal(size=(20, 26)).astype(np.float32) + 1
    Lp = 2
    dx, dy, al, st, _ = O.square_demodulate(img, O.make_params(carrier_freq=0.15), Lp)
    inner = np.zeros_like(st, dtype=bool)
    inner[Lp:-Lp, Lp:-Lp] = True
    assert (st[~inner] == O.STATUS_BORDER).all()
    assert np.isnan(dx[~inner]).all() and np.isnan(dy[~inner]).all() and np.isnan(al[~inner]).all()
    assert (st[inner] == O.STATUS_OK).all() and np.isfinite(al[inner]).all()


# ----------------------------------------------------------------------------------------------
# The paper takes the eigenvectors from the SVD of Gamma_w (Sec. 3): u1 and v1 must be its first
# left and right singular vectors (this fixes which operand of each product is conjugated).
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("Lp", [1, 3, 5])
def test_square_eigenvectors_are_singular_vectors(Lp):
    for seed in range(4):
        G = _noisy_block(Lp, 100 + seed)
        r = O.square_window(G)
        U, S, Vh = np.linalg.svd(G)
        assert abs(abs(np.vdot(U[:, 0], r["u1"])) - 1) < 1e-10
        assert abs(abs(np.vdot(Vh[0].conj(), r["v1"])) - 1) < 1e-10


# ----------------------------------------------------------------------------------------------
# Eq. 12-13 evaluated independently: on the unit circle the polynomial is the quadratic form
# a(z)^H (I - w w^H) a(z), a(z) = [1, z, ..., z^(M-1)]; sampling it at K >= 2M-1 points and
# taking the inverse DFT gives its Laurent coefficients, whose roots (numpy's companion matrix,
# the paper's method) are enumerated by brute force for the selection rule.
# ----------------------------------------------------------------------------------------------
def _angle_by_enumeration(w, sign):
    M = w.size
    K = 4 * M
    th = TWO_PI * np.arange(K) / K
    A = np.exp(1j * np.outer(np.arange(M), th))          # columns a(e^{j th})
    P = np.sum(np.abs(A) ** 2, axis=0) - np.abs(w.conj() @ A) ** 2
    c = np.fft.fft(P) / K                               # c[k mod K] multiplies z^k
    lag = np.arange(-(M - 1), M)
    coef = np.array([c[k % K] for k in lag])             # coefficient of z^k
    roots = np.roots(coef[::-1])                         # highest power first
    cand = roots[np.abs(roots) <= 1 + 1e-9]
    z = cand[np.argmin(np.abs(np.abs(cand) - 1))]
    return sign * np.angle(z)


@pytest.mark.parametrize("Lp", [1, 2, 4])
def test_square_angles_by_enumeration(Lp):
    for seed in range(6):
        G = _noisy_block(Lp, 200 + seed, sigma=0.8)
        r = O.square_window(G)
        assert r["status"] == O.STATUS_OK
        U, S, Vh = np.linalg.svd(G)
        wy = _angle_by_enumeration(U[:, 0], +1)
        wx = _angle_by_enumeration(Vh[0].conj(), -1)
        assert abs(_wrap(r["wy"] - wy)) < 1e-8
        assert abs(_wrap(r["wx"] - wx)) < 1e-8


# ----------------------------------------------------------------------------------------------
# Eq. 15 row 3: alpha is the least-squares phase of the block given the two angles: over
# amplitude and phase, it minimises sum |G - A exp(j(alpha + wx x + wy y))|^2.
# ----------------------------------------------------------------------------------------------
def test_square_alpha_is_least_squares_phase():
    Lp = 4
    y, x = np.mgrid[-Lp:Lp + 1, -Lp:Lp + 1]
    for seed in range(5):
        G = _noisy_block(Lp, 300 + seed, sigma=0.5)
        r = O.square_window(G)
        base = np.exp(1j * (r["wx"] * x + r["wy"] * y))

        def cost(a):
            e = np.exp(1j * a) * base
            amp = max(np.real(np.vdot(e, G)) / e.size, 0.0)   # best A >= 0 for this phase
            return np.sum(np.abs(G - amp * e) ** 2)

        c0 = cost(r["alpha"])
        for d in (1e-4, 1e-2, 0.3, 2.0):
            assert c0 <= cost(r["alpha"] + d) + 1e-12
            assert c0 <= cost(r["alpha"] - d) + 1e-12


# ----------------------------------------------------------------------------------------------
# Symmetries of the estimator.
# ----------------------------------------------------------------------------------------------
def test_square_transpose_swaps_axes():
    """Transposing the block exchanges the two analyses: (wx, wy) -> (wy, wx), alpha unchanged
    (Eq. 12 with G^T is Eq. 13 with G, given z_x = exp(-j wx))."""
    for Lp in (1, 3, 6):
        for seed in range(3):
            G = _noisy_block(Lp, 400 + 10 * Lp + seed)
            a, b = O.square_window(G), O.square_window(G.T)
            assert abs(a["wx"] - b["wy"]) < 1e-10 and abs(a["wy"] - b["wx"]) < 1e-10
            assert abs(_wrap(a["alpha"] - b["alpha"])) < 1e-10


def test_square_global_phase_and_scale():
    """G -> s exp(j theta) G (s > 0) leaves both angles unchanged and adds theta to alpha."""
    for seed in range(3):
        G = _noisy_block(3, 500 + seed)
        a = O.square_window(G)
        b = O.square_window(2.5 * np.exp(1j * 0.9) * G)
        assert abs(a["wx"] - b["wx"]) < 1e-10 and abs(a["wy"] - b["wy"]) < 1e-10
        assert abs(_wrap(b["alpha"] - a["alpha"] - 0.9)) < 1e-10


def test_square_modulation_shifts_angles():
    """Modulating the block by exp(j(tx x + ty y)) adds tx, ty to the angles and leaves alpha
    (centred coordinates) unchanged: the rotation of Eq. 12-13's roots is exact."""
    Lp = 3
    y, x = np.mgrid[-Lp:Lp + 1, -Lp:Lp + 1]
    for seed in range(3):
        G = _noisy_block(Lp, 600 + seed, sigma=0.4)
        a = O.square_window(G)
        b = O.square_window(G * np.exp(1j * (0.3 * x - 0.2 * y)))
        assert abs(_wrap(b["wx"] - a["wx"] - 0.3)) < 1e-10
        assert abs(_wrap(b["wy"] - a["wy"] + 0.2)) < 1e-10
        assert abs(_wrap(b["alpha"] - a["alpha"])) < 1e-10


def test_square_carrier_removal_on_complex_frames():
    """A complex frame with carrier exp(j 2 pi f0 x) and carrier_freq = f0 gives the maps of the
    same frame without the carrier and carrier_freq = 0 (complex frames are not band-passed)."""
    rng = np.random.default_rng(7)
    H, W, f0 = 30, 40, 0.13
    y, x = np.mgrid[0:H, 0:W]
    phi = 0.02 * (x - 20) ** 2 / 4 + 0.1 * y
    base = np.exp(1j * phi) + 0.3 * (rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W)))
    mod = base * np.exp(1j * TWO_PI * f0 * x)
    a = O.square_demodulate(base.astype(np.complex128), O.make_params(carrier_freq=0.0), 3)
    b = O.square_demodulate(mod.astype(np.complex128), O.make_params(carrier_freq=f0), 3)
    ok = a[3] == O.STATUS_OK
    assert (b[3] == a[3]).all() and ok.sum() > 0
    for i in range(3):
        assert np.abs(_wrap(a[i][ok] - b[i][ok])).max() < 1e-9


def test_square_sampled_equals_full():
    rng = np.random.default_rng(8)
    img = (0.5 + 0.4 * np.cos(TWO_PI * 0.12 * np.arange(48)[None, :] + rng.normal(size=(40, 48)) * 0.3))
    img = img.astype(np.float32)
    p = O.make_params(carrier_freq=0.12)
    full = O.square_demodulate(img, p, 4)
    ys = rng.integers(0, 40, 60)
    xs = rng.integers(0, 48, 60)
    smp = O.square_demodulate_pixels(img, p, 4, ys, xs)
    for i in range(3):
        np.testing.assert_array_equal(smp[i], full[i][ys, xs])
    np.testing.assert_array_equal(smp[3], full[3][ys, xs])
