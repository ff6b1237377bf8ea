"""Writes rouche_table.h: the constants of the row solver's Rouche root-count certificate
(roots_device.cuh, rouche_certify).

For covariance order L the noise-free (single steering vector) root-MUSIC polynomial, rotated so that
its double root sits at w = 1, has the real coefficients q_k = L - 1 (k = 0) and -(L - |k|) / L
(0 < |k| < L) at w^(k + L - 1) (Sec. 3, Eq. 12-14 with u = a(w)/sqrt(L)). Dividing out (w - 1)^2
leaves G_L(w) of degree 2L - 4 with L - 2 roots inside the unit circle and their mirrors outside.
The certificate compares a window's deflated polynomial with G_L on the circle |w| = rho and needs a
lower bound of min |G_L(w)| there. This script tabulates, for rho in [kRho0, kRho0 + kN kStep), a
lower bound valid on each interval [rho_i, rho_i + kStep]: G_L has no zeros in that annulus (checked
against its roots), so by the minimum modulus principle its minimum over the annulus is attained on
one of the two boundary circles; on each circle the minimum over 8192 equally spaced points, less a
bound on the derivative along the circle times the half spacing, is a lower bound. Entries where the
annulus contains a zero of G_L, or the bound is not positive, are 0 (the certificate then fails and
the Schur-Cohn count decides).

    python gen_rouche_table.py     (writes rouche_table.h next to this script)
"""
import os

import numpy as np

ORDERS = tuple(range(3, 13))  # every covariance order the row solvers take, but 2 (nothing to certify)
RHO0, STEP, NRHO = 0.40, 0.005, 120
NPTS = 8192


def g_std(L: int) -> np.ndarray:
    q = np.array([(L - 1.0) if k == 0 else -(L - abs(k)) / L for k in range(-(L - 1), L)])  # ascending
    g, rem = np.polydiv(q[::-1], np.poly([1.0, 1.0]))
    assert np.abs(rem).max() < 1e-12
    return g[::-1]  # ascending, degree 2L - 4


def min_modulus_lower_bound(g: np.ndarray, rho: float) -> float:
    th = np.arange(NPTS) * (2 * np.pi / NPTS)
    w = rho * np.exp(1j * th)
    v = np.abs(np.polyval(g[::-1], w)).min()
    k = np.arange(g.size)
    dmax = np.sum(k * np.abs(g) * rho ** k)  # |d G(rho e^{jt}) / dt| <= sum k |g_k| rho^k
    return v - dmax * (np.pi / NPTS)


def table(L: int):
    g = g_std(L)
    radii = np.abs(np.roots(g[::-1]))
    lo = []
    for i in range(NRHO):
        a, b = RHO0 + i * STEP, RHO0 + (i + 1) * STEP
        if np.any((radii >= a - 1e-9) & (radii <= b + 1e-9)) or np.any(radii[radii < 1] >= a):
            lo.append(0.0)
            continue
        m = min(min_modulus_lower_bound(g, a), min_modulus_lower_bound(g, b))
        lo.append(max(m, 0.0))
    lo = np.array(lo, dtype=np.float32)
    lo = np.where(lo > 0, np.nextafter(lo, np.float32(0)), 0).astype(np.float32)  # round down
    return g, lo, radii[radii < 1].max()


def header_text() -> str:
    lines = ["// rouche_table.h -- written by gen_rouche_table.py (do not edit): the noise-free deflated",
             "// root-MUSIC polynomials G_L and lower bounds of min |G_L| on the circles |w| = rho, for the row",
             "// solver's Rouche certificate (roots_device.cuh).",
             "#pragma once", "", "namespace rmusic {", "",
             f"constexpr float kRcRho0 = {RHO0}f;", f"constexpr float kRcStep = {STEP}f;",
             f"constexpr int kRcN = {NRHO};", ""]
    for L in ORDERS:
        g, lo, rin = table(L)
        lines.append(f"// L = {L}: inner roots of G_L up to |w| = {rin:.4f}")
        # G_L's coefficients as a constexpr function: indexed with compile-time k they fold into
        # immediate operands (no loads)
        cases = " ".join(f"case {k}: return {v:.9e}f;" for k, v in enumerate(g))
        lines.append(f"__host__ __device__ constexpr float rouche_g{L}(int k) {{ switch (k) {{ {cases} default: return 0.f; }} }}")
        body = ", ".join(f"{v:.7e}f" for v in lo)
        lines.append(f"__device__ const float kRcMin{L}[{NRHO}] = {{{body}}};")
        lines.append("")
    lines += ["}  // namespace rmusic", ""]
    return "\n".join(lines)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "rouche_table.h"), "w") as f:
        f.write(header_text())


if __name__ == "__main__":
    main()
