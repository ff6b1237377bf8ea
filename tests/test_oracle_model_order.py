"""Pins for the oracle's model order p > 1 on real fringes without the analytic step (Sec. 3 with p
exponentials per window: a real cosine carries exp(+-j omega), a local offset one more at zero
frequency). Checked against closed forms (exact frequencies of noise-free cosines, with and without
offsets), an independent evaluation (LAPACK eigenvectors, the pseudospectrum's Fourier
coefficients, numpy's companion-matrix roots and an enumeration of the selection rule), and the
p = 1 special case."""
import numpy as np
import pytest

import oracle as O

TWO_PI = 2 * np.pi


@pytest.mark.parametrize("L,fb", [(6, 0), (8, 1), (12, 1)])
def test_p2_noise_free_real_cosine_exact(L, fb):
    H, W, f, f0 = 6, 128, 16 / 128, 0.1
    y, x = np.mgrid[0:H, 0:W]
    img = 0.5 + 0.4 * np.cos(TWO_PI * f * x + 0.3 * y)  # the line mean is exactly 0.5
    out, st, _ = O.demodulate(img, O.make_params(32, L, fb, 0, 0, f0, model_order=2, raw_input=1))
    v = st == 0
    assert v.sum() == H * (W - 31)
    assert np.abs(out[v] - TWO_PI * (f - f0)).max() < 1e-9


def test_p3_models_a_local_offset():
    """Windows inside one half of a line with a step offset hold a constant plus a cosine: three
    exponentials, recovered exactly with p = 3 and biased with p = 2."""
    H, W, f, f0 = 4, 128, 16 / 128, 0.1
    y, x = np.mgrid[0:H, 0:W]
    img = 0.5 + 0.3 * (x < W // 2) + 0.4 * np.cos(TWO_PI * f * x + 0.3 * y)
    xs = np.arange(W)
    inside = ((xs - 16 >= 0) & (xs + 15 < W // 2)) | ((xs - 16 >= W // 2) & (xs + 15 < W))
    o3, s3, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, f0, model_order=3, raw_input=1))
    v = (s3 == 0) & inside[None, :]
    assert v.sum() == H * inside.sum()
    assert np.abs(o3[v] - TWO_PI * (f - f0)).max() < 1e-9
    o2, s2, _ = O.demodulate(img, O.make_params(32, 8, 1, 0, 0, f0, model_order=2, raw_input=1))
    v2 = (s2 == 0) & inside[None, :]
    assert np.abs(o2[v2] - TWO_PI * (f - f0)).max() > 1e-3


def _reference_p(w, L, p, fb, omega_ref):
    """Independent evaluation for one window: LAPACK eigenvectors of R, the polynomial's Laurent
    coefficients from the pseudospectrum a(z)^H C a(z) sampled on the circle, numpy's roots, and
    the selection rule enumerated."""
    N = w.size
    K = N - L + 1
    S = np.array([w[i:i + L] for i in range(K)])
    R = S.T @ S.conj() / K
    if fb:
        J = np.eye(L)[::-1]
        R = 0.5 * (R + J @ R.conj() @ J)
    ev, V = np.linalg.eigh(R)
    U = V[:, ::-1][:, :p]
    C = np.eye(L) - U @ U.conj().T
    M = 4 * L
    th = TWO_PI * np.arange(M) / M
    A = np.exp(1j * np.outer(np.arange(L), th))
    P = np.real(np.einsum("im,ij,jm->m", A.conj(), C, A))
    c = np.fft.fft(P) / M
    coef = np.array([c[k % M] for k in range(-(L - 1), L)])
    roots = np.roots(coef[::-1])
    cand = [r for r in roots if abs(r) <= 1 + 1e-9]
    cand.sort(key=lambda r: abs(abs(r) - 1))
    chosen = []
    for r in cand:
        if len(chosen) == p:
            break
        if all(abs(r - q) >= 1e-6 for q in chosen):
            chosen.append(r)
    z = min(chosen, key=lambda r: abs(np.angle(r * np.exp(-1j * omega_ref))))
    return float(np.angle(z * np.exp(-1j * omega_ref)))


@pytest.mark.parametrize("p", [2, 3])
def test_p_noisy_windows_by_enumeration(p):
    rng = np.random.default_rng(p)
    for trial in range(8):
        n = np.arange(24)
        w = np.cos(0.7 * n + rng.uniform(0, 6)) + (0.4 if p == 3 else 0.0) + 0.2 * rng.normal(size=24)
        r = O.window_derivative_p(w.astype(complex), 8, p, fb=1, omega_ref=0.6)
        assert r["status"] == O.STATUS_OK
        assert abs(r["deriv"] - _reference_p(w.astype(complex), 8, p, 1, 0.6)) < 1e-8


def test_p1_is_the_papers_estimator():
    rng = np.random.default_rng(9)
    for _ in range(5):
        w = np.exp(1j * 0.9 * np.arange(32)) + 0.3 * (rng.normal(size=32) + 1j * rng.normal(size=32))
        a = O.window_derivative_p(w, 8, 1, fb=1, omega_ref=0.5)
        b = O.window_derivative(w, 8, fb=1, omega_ref=0.5)
        assert a["deriv"] == b["deriv"]
