"""The row solver's Rouche root-count certificate (roots_device.cuh, rouche_certify), on the CPU.

The certificate replaces the Schur-Cohn count of the roots inside |z| < rho = |z_s| - 0.02 where it
can: it deflates the selected root and its mirror from the root-MUSIC polynomial (Sec. 3, Eq. 12-14)
and compares what is left with the noise-free polynomial G_L on |w| = rho. These tests check the
constants it is built on (the committed rouche_table.h is what gen_rouche_table.py writes; G_L is the
deflated steering-vector polynomial; the tabulated bounds are below min |G_L| on the circles) and the
soundness of the test itself: a float32 restatement of the device test, run on polynomials of noisy
steering vectors, random vectors and pairs of exponentials, never certifies a root count that numpy's
companion-matrix roots contradict.
"""
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1910_11872_gb300", "csrc")
f32 = np.float32


def _gen():
    spec = importlib.util.spec_from_file_location("gen_rouche_table", os.path.join(CSRC, "gen_rouche_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _header():
    return open(os.path.join(CSRC, "rouche_table.h")).read()


def _g(txt, L):
    m = re.search(r"constexpr float rouche_g%d\(int k\) \{ switch \(k\) \{ (.*?) default" % L, txt)
    return np.array([float(v.rstrip("f;")) for v in re.findall(r"return ([^;]+);", m.group(1))], dtype=np.float32)


def _mins(txt, L):
    m = re.search(r"kRcMin%d\[\d+\] = \{([^}]*)\}" % L, txt)
    return np.array([float(x.strip().rstrip("f")) for x in m.group(1).split(",")], dtype=np.float32)


def test_committed_table_is_the_generators_output():
    assert _header() == _gen().header_text()


@pytest.mark.parametrize("L", list(range(3, 13)))
def test_g_is_the_deflated_steering_vector_polynomial(L):
    """G_L (w - 1)^2 equals the root-MUSIC polynomial of u = a(0) / sqrt(L) (Eq. 12-14: c_0 = L - 1,
    c_k = -(L - |k|) / L), and G_L has L - 2 roots inside the unit circle and their mirrors outside."""
    g = _g(_header(), L).astype(np.float64)
    u = np.ones(L) / np.sqrt(L)
    C = np.eye(L) - np.outer(u, u)
    q = np.array([np.trace(C, offset=k) for k in range(-(L - 1), L)])  # ascending powers
    back = np.convolve(g, [1.0, -2.0, 1.0])
    assert np.abs(back - q).max() < 1e-6
    r = np.abs(np.roots(g[::-1]))
    assert (r < 1).sum() == L - 2 and (r > 1).sum() == L - 2


@pytest.mark.parametrize("L", list(range(3, 13)))
def test_tabulated_bounds_are_below_the_minimum_modulus(L):
    txt = _header()
    g = _g(txt, L).astype(np.float64)
    lo = _mins(txt, L)
    rho0 = float(re.search(r"kRcRho0 = ([0-9.]+)f", txt).group(1))
    step = float(re.search(r"kRcStep = ([0-9.]+)f", txt).group(1))
    rin = np.abs(np.roots(g[::-1]))
    rin = rin[rin < 1].max()
    th = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    rng = np.random.default_rng(L)
    for i in np.flatnonzero(lo > 0):
        a = rho0 + i * step
        assert a > rin  # the interval's annulus holds no zero of G_L
        for rho in (a, a + step, a + rng.uniform(0, step)):
            assert np.abs(np.polyval(g[::-1], rho * np.exp(1j * th))).min() >= lo[i]


def _certify32(c, zs, r, L, txt):
    """float32 restatement of rouche_certify: True when Q provably has L - 2 roots in |z| < r - 0.02."""
    lo, g = _mins(txt, L), _g(txt, L)
    n = 2 * L - 2
    rho = f32(r - f32(0.02))
    ft = (rho - f32(0.4)) * f32(1 / 0.005)
    if not (0 <= ft < lo.size) or not lo[int(ft)] > 0:
        return False
    ir = f32(1) / f32(r)
    e = np.complex64(zs * ir)
    ch, ep = [np.complex64(c[0])], e
    for k in range(1, L):
        ch.append(np.complex64(c[k] * ep))
        ep = np.complex64(ep * e)

    def qh(i):
        k = i - (L - 1)
        return ch[0] if k == 0 else (ch[k] if k > 0 else np.conj(ch[-k]))

    sig = f32(r + ir)
    b2 = b1 = np.complex64(0)
    s = f32(0)
    for k in range(n - 2, -1, -1):
        q = qh(k + 2)
        b = np.complex64(complex(f32(sig * b1.real + q.real) - b2.real, f32(sig * b1.imag + q.imag) - b2.imag))
        s = f32(s * rho + (abs(f32(b.real - g[k])) + abs(b.imag)))
        b2, b1 = b1, b
    q1, q0 = qh(1), qh(0)
    R1 = complex(f32(sig * b1.real + q1.real) - b2.real, f32(sig * b1.imag + q1.imag) - b2.imag)
    Rr = complex(f32(R1.real * r + f32(q0.real - b1.real)), f32(R1.imag * r + f32(q0.imag - b1.imag)))
    qmin = f32((r - rho) * (ir - rho))
    qsum = f32(L - 1 + 2 * sum(abs(ck) for ck in c[1:]))
    lhs = f32(s + (abs(R1.real) + abs(R1.imag)) / f32(ir - rho) + (abs(Rr.real) + abs(Rr.imag) + 4e-6 * qsum) / qmin)
    return bool(lhs < f32(0.9) * lo[int(ft)])


def _coefs32(u, L):
    u = u.astype(np.complex64)
    inu2 = f32((1 - 2e-6) / f32(np.sum(np.abs(u) ** 2)))
    return [np.complex64(L - 1)] + [np.complex64(-inu2 * np.sum(u[:L - k] * np.conj(u[k:]))) for k in range(1, L)]


@pytest.mark.parametrize("L", [3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_certificate_never_certifies_a_wrong_count(L):
    txt = _header()
    rng = np.random.default_rng(100 + L)
    certified = 0
    for trial in range(600):
        kind = trial % 3
        m = np.arange(L)
        if kind == 0:  # a noisy steering vector (the estimator's normal case)
            u = np.exp(1j * rng.uniform(-np.pi, np.pi) * m) + rng.uniform(0, 0.6) * (rng.normal(size=L) + 1j * rng.normal(size=L))
        elif kind == 1:  # no structure at all
            u = rng.normal(size=L) + 1j * rng.normal(size=L)
        else:  # two exponentials: a second root can come near the circle
            w1, w2 = rng.uniform(-np.pi, np.pi, 2)
            u = np.exp(1j * w1 * m) + rng.uniform(0.2, 1.0) * np.exp(1j * w2 * m)
        c = _coefs32(u, L)
        q = np.array([np.conj(c[L - 1 - i]) if i < L - 1 else c[i - (L - 1)] for i in range(2 * L - 1)], complex)
        roots = np.roots(q[::-1])
        inner = roots[np.abs(roots) < 1]
        zs = inner[np.argmax(np.abs(inner))]
        r = abs(zs)
        if r <= 0.5:
            continue
        if _certify32(c, np.complex64(zs), f32(r), L, txt):
            certified += 1
            assert int(np.sum(np.abs(roots) < r - 0.02)) == L - 2, (L, kind, r)
    assert certified >= 20  # the test is exercised, not vacuous
