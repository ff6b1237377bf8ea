"""Pins for the FP64 oracle: each test checks it against something other than itself -- a closed
form from the paper's model, a textbook special case, a library routine computing the same
mathematical object by another method, or an invariance of the estimator.

Paper: Ramaiah et al., arXiv:1910.11872, Sec. 3 (Eq. 2-15) and Algorithm 1.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_11872_gb300 import synth

TWO_PI = 2 * np.pi


def _wrap(a):
    return (np.asarray(a) + np.pi) % TWO_PI - np.pi


# ----------------------------------------------------------------------------------------------
# Step 2: analytic signal (Sec. 2, Eq. 1)
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("W", [64, 77, 128, 200])
def test_analytic_line_matches_fft_bandpass(W):
    """The direct-DFT band-pass equals numpy's FFT with the same one-sided band mask."""
    rng = np.random.default_rng(W)
    v = rng.normal(size=W) + 0.5
    f0, B = 0.12, 0.06
    X = np.fft.fft(v)
    k = np.arange(W)
    mask = (k >= 1) & (2 * k < W) & (np.abs(k / W - f0) < B)
    ref = np.fft.ifft(np.where(mask, X, 0))
    got = O.analytic_line(v, f0, B)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_analytic_line_closed_form_periodic_cosine():
    """a + b cos(2 pi k0 n / W + p) with k0 inside the band -> (b/2) exp(j(2 pi k0 n / W + p))."""
    W, k0, p = 128, 14, 0.7
    n = np.arange(W)
    v = 0.5 + 0.4 * np.cos(TWO_PI * k0 * n / W + p)
    got = O.analytic_line(v, 0.1)
    assert np.abs(got - 0.2 * np.exp(1j * (TWO_PI * k0 * n / W + p))).max() < 1e-13
    # a component outside the band vanishes
    v2 = v + 0.3 * np.cos(TWO_PI * 40 * n / W)
    assert np.abs(O.analytic_line(v2, 0.1) - got).max() < 1e-13


def test_analytic_frame_axes():
    """Carrier along y is the carrier-along-x result of the transposed frame."""
    rng = np.random.default_rng(3)
    img = rng.normal(size=(24, 40))
    gx = O.analytic_frame(img, 0.1, carrier_axis=0)
    gy = O.analytic_frame(np.ascontiguousarray(img.T), 0.1, carrier_axis=1)
    assert np.abs(gx - gy.T).max() < 1e-14


# ----------------------------------------------------------------------------------------------
# Step 4: covariance (Sec. 3, Eq. 4-8)
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fb", [0, 1])
@pytest.mark.parametrize("N,L", [(12, 3), (32, 8), (24, 6), (48, 12)])
def test_covariance_rank_one_for_exponential(N, L, fb):
    """Eq. 6-8: a window A exp(j(w n + a)) has R = A^2 u1 u1^H, R[m][l] = A^2 exp(j w (m - l))."""
    A, w, a = 0.7, 0.9, 0.4
    n = np.arange(N)
    R = O.covariance(A * np.exp(1j * (w * n + a)), L, fb)
    m = np.arange(L)
    ref = A * A * np.exp(1j * w * (m[:, None] - m[None, :]))
    assert np.abs(R - ref).max() < 1e-14


def test_covariance_structure_noise():
    """Hermitian, positive semidefinite, trace = mean snapshot energy, FB is centro-Hermitian."""
    rng = np.random.default_rng(5)
    N, L = 32, 8
    K = N - L + 1
    w = rng.normal(size=N) + 1j * rng.normal(size=N)
    Rf = O.covariance(w, L, 0)
    R = O.covariance(w, L, 1)
    J = np.eye(L)[::-1]
    for M in (Rf, R):
        assert np.abs(M - M.conj().T).max() < 1e-15
        assert np.linalg.eigvalsh(M).min() > -1e-13
    energy = sum(np.sum(np.abs(w[i:i + L]) ** 2) for i in range(K)) / K
    assert abs(np.trace(Rf).real - energy) < 1e-12
    assert np.abs(J @ R.conj() @ J - R).max() < 1e-15
    assert np.abs(R - 0.5 * (Rf + J @ Rf.conj() @ J)).max() < 1e-15


# ----------------------------------------------------------------------------------------------
# Step 5: eigen-decomposition (Sec. 3, Eq. 8-11; the paper uses an SVD)
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 5, 8, 12])
def test_eig_matches_lapack(L):
    rng = np.random.default_rng(L)
    X = rng.normal(size=(L, 3 * L)) + 1j * rng.normal(size=(L, 3 * L))
    R = X @ X.conj().T / (3 * L)
    ev, V, sweeps = O.eig_hermitian(R)
    assert sweeps > 0
    ref = np.linalg.eigvalsh(R)
    assert np.abs(np.sort(ev) - ref).max() < 1e-12 * ref.max()
    j = np.argmax(ev)
    u = V[:, j]
    assert np.linalg.norm(R @ u - ev[j] * u) < 1e-13 * np.linalg.norm(R)
    w, U = np.linalg.eigh(R)
    # same eigenvector up to a unit phase
    assert abs(abs(np.vdot(U[:, -1], u)) - 1.0) < 1e-12
    assert np.abs(V.conj().T @ V - np.eye(L)).max() < 1e-13


def test_eig_eigenvalues_signal_plus_noise():
    """Eq. 10: R = A^2 u u^H + s^2 I has eigenvalues L A^2 + s^2 and s^2 (L-1 times)."""
    L, A, s2, w = 8, 0.6, 0.05, -1.1
    a = np.exp(1j * w * np.arange(L))
    R = A * A * np.outer(a, a.conj()) + s2 * np.eye(L)
    ev, V, _ = O.eig_hermitian(R)
    ev = np.sort(ev)
    assert abs(ev[-1] - (L * A * A + s2)) < 1e-13
    assert np.abs(ev[:-1] - s2).max() < 1e-13


# ----------------------------------------------------------------------------------------------
# Step 6: root-MUSIC polynomial (Sec. 3, Eq. 12-14)
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 4, 8, 12])
def test_music_poly_on_circle_equals_noise_projection(L):
    """On |z| = 1, Q(z) z^-(L-1) = a(w)^H (I - u u^H) a(w) = L - |u^H a(w)|^2 (real, >= 0)."""
    rng = np.random.default_rng(10 + L)
    u = rng.normal(size=L) + 1j * rng.normal(size=L)
    u /= np.linalg.norm(u)
    q = O.music_poly(u)
    for w in np.linspace(-np.pi, np.pi, 37):
        a = np.exp(1j * w * np.arange(L))
        ref = L - abs(np.vdot(u, a)) ** 2
        z = np.exp(1j * w)
        val = np.polyval(q[::-1], z) * z ** (-(L - 1))
        assert abs(val - ref) < 1e-12
        assert ref >= -1e-12


def test_music_poly_closed_form_steering_vector():
    """u = a(w0)/sqrt(L): c_k = L d_k - (L - |k|)/L exp(-j w0 k)."""
    L, w0 = 8, 0.77
    u = np.exp(1j * w0 * np.arange(L)) / np.sqrt(L)
    q = O.music_poly(u)
    k = np.arange(-(L - 1), L)
    ref = L * (k == 0) - (L - np.abs(k)) / L * np.exp(-1j * w0 * k)
    assert np.abs(q - ref).max() < 1e-14


# ----------------------------------------------------------------------------------------------
# Step 7: roots (the paper solves with companion-matrix eigenvalues)
# ----------------------------------------------------------------------------------------------
def _match(a, b):
    """Max distance of the best one-to-one matching of two root sets (greedy, small sets)."""
    a, b = list(a), list(b)
    worst = 0.0
    for z in a:
        j = int(np.argmin([abs(z - t) for t in b]))
        worst = max(worst, abs(z - b[j]))
        b.pop(j)
    return worst


@pytest.mark.parametrize("seed", range(6))
def test_roots_match_companion_matrix(seed):
    """All roots equal numpy's companion-matrix eigenvalues (the paper's method)."""
    rng = np.random.default_rng(100 + seed)
    L = [2, 4, 6, 8, 12, 8][seed]
    u = rng.normal(size=L) + 1j * rng.normal(size=L)
    u /= np.linalg.norm(u)
    q = O.music_poly(u)
    r, nc = O.poly_roots(q)
    assert not nc and r.size == 2 * L - 2
    ref = np.roots(q[::-1])
    assert _match(r, ref) < 1e-9
    # residual at the rounding level
    for z in r:
        assert abs(np.polyval(q[::-1], z)) < 1e-12 * np.polyval(np.abs(q[::-1]), abs(z))


def _near_pair_polynomial(L, eps, theta):
    """Conjugate-self-reciprocal polynomial of degree 2L - 2 (the root-MUSIC structure, Eq. 12-14)
    with planted roots: a near pair (1 - eps) e^{j theta} and its mirror 1/(1 - eps) e^{j theta},
    2 eps apart across the unit circle, and L - 2 further inner roots at radius 0.55 / 0.7 with
    their mirrors. Returns the ascending coefficients (rounded to FP64)."""
    inner = [(1 - eps) * np.exp(1j * theta)]
    for k in range(1, L - 1):
        inner.append((0.55 if k % 2 else 0.7) * np.exp(1j * (theta + TWO_PI * k / (L - 1))))
    inner = np.array(inner)
    return np.poly(np.concatenate([inner, 1 / np.conj(inner)]))[::-1]


@pytest.mark.parametrize("L", [4, 6, 8, 12])
def test_roots_near_pair_at_rounding_level(L):
    """Roots of polynomials whose signal root and its mirror straddle the unit circle 2e-3, 2e-4 and
    2e-5 apart (the configuration the selection of Sec. 3 has to resolve on high-SNR windows) are as
    accurate as the FP64 coefficients allow: each root is within 3 x its first-order condition bound
    eps_64 sum_k |q_k| |z|^k / |Q'(z)| of the exact root of the same FP64 coefficients, computed
    independently with mpmath's polyroots in 60-digit arithmetic. A root finder stopped at the
    residual level alone leaves the near pair 20-45 x its condition bound off."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    worst = 0.0
    for eps in (1e-3, 1e-4, 1e-5):
        for theta in (0.3, 2.0, -1.1):
            q = _near_pair_polynomial(L, eps, theta)
            exact = np.array([complex(z) for z in mpmath.polyroots([mpmath.mpc(complex(c)) for c in q[::-1]],
                                                                   maxsteps=400, extraprec=400)])
            got, nc = O.poly_roots(q)
            assert not nc and got.size == 2 * L - 2
            d = np.abs(got[:, None] - exact[None, :])
            j = d.argmin(axis=1)
            assert len(set(j.tolist())) == got.size  # one computed root per exact root
            k = np.arange(q.size)
            for z, e in zip(exact[j], d.min(axis=1)):
                bound = np.finfo(float).eps * np.sum(np.abs(q) * np.abs(z) ** k) / abs(np.sum(k[1:] * q[1:] * z ** (k[1:] - 1)))
                worst = max(worst, e / bound)
    assert worst <= 3.0, worst


@pytest.mark.parametrize("L", [3, 8, 12])
def test_roots_conjugate_reciprocal_pairs(L):
    """c_-k = conj(c_k) makes the root set closed under z -> 1/conj(z)."""
    rng = np.random.default_rng(7 * L)
    u = rng.normal(size=L) + 1j * rng.normal(size=L)
    u /= np.linalg.norm(u)
    r, _ = O.poly_roots(O.music_poly(u))
    assert _match(r, 1.0 / np.conj(r)) < 1e-9


def test_roots_generic_polynomial_and_zero_coefficients():
    q = np.array([0, 0, 2.0, -3.0 + 1j, 1.0, 0.5j, 0, 0], dtype=complex)  # two roots at 0, two at inf
    r, _ = O.poly_roots(q)
    assert r.size == 5
    assert sum(abs(z) == 0 for z in r) == 2
    assert _match([z for z in r if z != 0], np.roots(q[2:6][::-1])) < 1e-12


# ----------------------------------------------------------------------------------------------
# Step 8: selection (Sec. 3; Algorithm 1)
# ----------------------------------------------------------------------------------------------
def test_selection_hand_cases():
    q_dummy = np.array([1.0, 0.0, 1.0], dtype=complex)
    # inside and closest to the circle wins over an outside root that is closer
    roots = [0.5 + 0j, 0.9 * np.exp(0.3j), 1.02 * np.exp(-0.2j), 3.0 + 0j]
    assert O.select_root(q_dummy, roots) == pytest.approx(0.9 * np.exp(0.3j))
    # a root just outside within 1e-9 still counts (split double root on the circle)
    roots = [0.8 + 0j, (1 + 5e-10) * np.exp(1.1j), 2.0 + 0j]
    assert O.select_root(q_dummy, roots) == pytest.approx((1 + 5e-10) * np.exp(1.1j))
    # nothing inside: no candidate
    assert O.select_root(q_dummy, [1.5 + 0j, 2.0j]) is None


def test_selection_split_double_root_is_relocated_on_q_prime():
    """A double root at z0 perturbed into two roots 1e-8 apart is returned as z0."""
    z0 = np.exp(0.6j)
    others = [0.3 + 0.1j, 2.5 - 1j]
    q = np.poly([z0, z0] + others)[::-1]  # ascending
    split = [z0 * (1 + 1e-8 * np.exp(0.4j)), z0 * (1 - 1e-8 * np.exp(0.4j))]
    z = O.select_root(q, split + others)
    assert abs(z - z0) < 1e-14


# ----------------------------------------------------------------------------------------------
# End to end (steps 1-9)
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fb", [0, 1])
@pytest.mark.parametrize("N,L", [(32, 2), (32, 3), (32, 8), (24, 6), (48, 12), (33, 8)])
def test_p1_noise_free_linear_phase_exact(N, L, fb):
    """Noise-free periodic fringe (W f integer): the analytic signal is one exponential, Q has a
    double root at exp(j 2 pi f), and the output is 2 pi (f - f0) at every valid pixel."""
    H, W, f, f0 = 6, 128, 16 / 128, 0.1
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = 0.5 + 0.4 * np.cos(TWO_PI * f * x + 0.3)
    out, st, _ = O.demodulate(img, O.make_params(N, L, fb, 0, 0, f0))
    valid = st == O.STATUS_OK
    assert valid.sum() == H * (W - N + 1)
    assert np.all(st[~valid] == O.STATUS_BORDER) and np.all(np.isnan(out[~valid]))
    assert np.abs(out[valid] - TWO_PI * (f - f0)).max() < 1e-12
    # the valid columns are exactly those whose window stays inside the line
    cols = np.where(valid[0])[0]
    assert cols[0] == N // 2 and cols[-1] == W - N + N // 2


@pytest.mark.parametrize("gy", [0.03, -0.05])
def test_p1_noise_free_tilt_along_y(gy):
    """Carrier along x, windows along y: the output is the y phase slope 2 pi gy (no carrier)."""
    H, W = 64, 128
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = 0.5 + 0.4 * np.cos(TWO_PI * (16 / 128) * x + TWO_PI * gy * y + 0.3)
    out, st, _ = O.demodulate(img, O.make_params(32, 8, 1, 1, 0, 0.1))
    valid = st == 0
    assert valid.sum() == W * (H - 32 + 1)
    assert np.abs(out[valid] - TWO_PI * gy).max() < 1e-12


@pytest.mark.parametrize("fb", [0, 1])
def test_p2_order_two_is_pulse_pair(fb):
    """L = 2: root-MUSIC reduces to the lag-one autocorrelation estimator arg sum w[i+1] conj w[i]."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        N = int(rng.integers(4, 40))
        w0 = rng.uniform(-3, 3)
        n = np.arange(N)
        w = np.exp(1j * w0 * n) + 0.7 * (rng.normal(size=N) + 1j * rng.normal(size=N))
        ref_angle = 0.4
        got = O.window_derivative(w, 2, fb, ref_angle)["deriv"]
        pp = np.angle(np.sum(w[1:] * np.conj(w[:-1])))
        assert abs(_wrap(got - (pp - ref_angle))) < 1e-10


def test_p4_carrier_rotation():
    """Multiplying the window by exp(-j t n) rotates every root by exp(-j t): output shifts by -t."""
    rng = np.random.default_rng(12)
    N, L = 32, 8
    n = np.arange(N)
    w = 0.4 * np.exp(1j * (0.8 * n + 0.01 * n ** 2)) + 0.1 * (rng.normal(size=N) + 1j * rng.normal(size=N))
    for fb in (0, 1):
        base = O.window_derivative(w, L, fb)["deriv"]
        for t in (0.3, -1.2, 2.0):
            got = O.window_derivative(w * np.exp(-1j * t * n), L, fb)["deriv"]
            assert abs(_wrap(got - (base - t))) < 1e-10


def test_p5_invariances():
    """Affine intensity change, global phase, and transposition with the axes swapped."""
    fr = synth.small_gaussian_frame(H=48, W=64)
    img = fr.image.astype(np.float64)
    p = O.make_params(32, 8, 1, 0, 0, 0.1)
    base, st, _ = O.demodulate(img, p)
    v = st == 0
    aff, _, _ = O.demodulate(3.7 * img - 1.1, p)
    assert np.abs(aff[v] - base[v]).max() < 1e-9
    pt = O.make_params(32, 8, 1, 1, 1, 0.1)
    tr, stt, _ = O.demodulate(np.ascontiguousarray(img.T), pt)
    assert np.array_equal(stt.T, st)
    assert np.abs(tr.T[v] - base[v]).max() < 1e-9
    rng = np.random.default_rng(2)
    w = np.exp(0.5j * np.arange(32)) + 0.3 * rng.normal(size=32)
    a = O.window_derivative(w, 8, 1)["deriv"]
    b = O.window_derivative(w * np.exp(1.3j), 8, 1)["deriv"]
    assert abs(a - b) < 1e-11


@pytest.mark.parametrize("L", [2, 3, 4])
def test_p7_noise_free_root_is_pseudospectrum_minimum(L):
    """Noise-free: the selected root's angle is where P(w) = a^H C a vanishes on the circle,
    found by brute-force grid search (tiny windows, non-periodic frequencies)."""
    rng = np.random.default_rng(20 + L)
    for _ in range(5):
        N = int(rng.integers(L + 2, 13))
        w0 = rng.uniform(-3, 3)
        w = 0.3 * np.exp(1j * (w0 * np.arange(N) + 0.2))
        res = O.window_derivative(w, L, 1)
        grid = np.linspace(-np.pi, np.pi, 1_000_001)
        u = res["u1"]
        A = np.exp(1j * np.outer(grid, np.arange(L)))
        P = L - np.abs(A @ u.conj()) ** 2
        assert abs(_wrap(grid[np.argmin(P)] - res["deriv"])) <= 2 * (grid[1] - grid[0])
        assert abs(_wrap(res["deriv"] - w0)) < 1e-10


def test_p7_noisy_selection_by_enumeration():
    """Noisy windows: the oracle's root set equals the companion-matrix roots, and the selected
    root is the inside root nearest the circle found by enumerating numpy's roots."""
    rng = np.random.default_rng(31)
    for _ in range(40):
        L = int(rng.choice([2, 3, 4, 6, 8]))
        N = int(rng.integers(L + 1, 3 * L + 4))
        w = np.exp(1j * rng.uniform(-3, 3) * np.arange(N)) + 0.8 * (rng.normal(size=N) + 1j * rng.normal(size=N))
        res = O.window_derivative(w, L, int(rng.integers(2)))
        ref = np.roots(res["q"][::-1])
        # near-double roots (the pair z, 1/conj(z) close to the circle) are only determined to
        # about sqrt(eps) by either root finder
        assert _match(res["roots"], ref) < 1e-6
        inside = [z for z in ref if abs(z) <= 1 + 1e-9]
        best = min(inside, key=lambda z: abs(abs(z) - 1))
        assert abs(_wrap(np.angle(best) - res["deriv"])) < 1e-6


def test_p8_accuracy_against_analytic_derivative():
    """Gaussian-bump fringe: the derivative follows the closed-form dphi/dx away from the line
    ends. The local linear-phase model (Sec. 3, Eq. 3) leaves a window-averaging bias, so the
    output sits closer to the mean slope across the window than to the pointwise slope."""
    fr = synth.small_gaussian_frame(sigma=0.0)
    out, st, _ = O.demodulate(fr.image, O.make_params(32, 8, 1, 0, 0, 0.1))
    inner = np.zeros_like(st, dtype=bool)
    inner[:, 32:96] = True
    v = inner & (st == 0)
    e = (out - fr.truth)[v]
    assert np.sqrt(np.mean(e ** 2)) < 1e-2
    phi, _, _ = synth.gaussian_bump(128, 128, 3.0, 64.0, 64.0, 20.0)
    slope = np.full_like(phi, np.nan)
    slope[:, 16:113] = (phi[:, 31:128] - phi[:, 0:97]) / 31.0   # window [n-16, n+15]
    em = (out - slope)[v]
    assert np.sqrt(np.mean(em ** 2)) < 4e-3
    assert np.sqrt(np.mean(em ** 2)) < 0.6 * np.sqrt(np.mean(e ** 2))
    fr = synth.small_gaussian_frame(sigma=0.02)
    out2, st2, _ = O.demodulate(fr.image, O.make_params(32, 8, 1, 0, 0, 0.1))
    e2 = (out2 - fr.truth)[inner & (st2 == 0)]
    assert np.sqrt(np.mean(e2 ** 2)) < 1e-2


def test_degenerate_zero_frame_and_parameters():
    img = np.zeros((8, 64), dtype=np.float32)
    out, st, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, 0.1))
    assert np.all(np.isnan(out))
    assert set(np.unique(st)) <= {O.STATUS_BORDER, O.STATUS_DEGENERATE}
    assert (st == O.STATUS_DEGENERATE).sum() == 8 * (64 - 32 + 1)
    with pytest.raises(ValueError):
        O.demodulate(img, O.make_params(8, 12, 1, 0, 0, 0.1))


def test_sampled_pixels_equal_full_frame():
    fr = synth.diffusion_frame(3, T=10, H=96, W=64)
    p = O.make_params(32, 8, 1, 1, 0, 0.1)
    full, st, _ = O.demodulate(fr.image, p)
    rng = np.random.default_rng(0)
    ys = rng.integers(0, 96, 50)
    xs = rng.integers(0, 64, 50)
    vals, sst, _ = O.demodulate_pixels(fr.image, p, ys, xs)
    assert np.array_equal(sst, st[ys, xs])
    np.testing.assert_array_equal(vals, full[ys, xs])
