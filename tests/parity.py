"""Element-wise comparison of GPU maps with the FP64 oracle's, shared by the GPU parity tests.

The rule (Sec. 3 and Algorithm 1 fix one selected root per pixel):
  * border pixels (status 1) are decided by integer geometry and must be identical;
  * every other status must be identical too, and every pixel that both sides call ok must agree
    to within `tol` rad/pixel, unless the oracle itself shows that the pixel's decision lies within
    the FP32 resolution of the GPU path -- an "excused" pixel:
      - near tie: among the oracle's roots of that window the two candidates of the selection
        (|z| <= 1 + 1e-9, nearest the circle) differ in their distance to the circle by less than
        TIE_RES, and the GPU's value is the other candidate's angle (within `tol`);
      - near degenerate: the oracle's eigen-gap l1 - l2 is below GAP_RES l1 (the FP32 path's
        degenerate threshold is 4e-6 l1) and the GPU called the pixel degenerate.
    Excused pixels are counted and may be at most `max_excused` of the compared pixels.
"""
from __future__ import annotations

import numpy as np

import oracle as O

TWO_PI = 2 * np.pi
# Distance-to-circle difference below which two roots are a tie at FP32 resolution: the FP32
# coefficients' relative rounding (~1e-6 after the eigenvector) moves a root's modulus by a few
# 1e-6 on well-conditioned windows; 2e-5 leaves a factor of five above the largest deviation of the
# FP32 path's selected roots from the oracle's seen on noisy 1024^2 frames (4e-6).
TIE_RES = 2e-5
GAP_RES = 1e-5


def _wrap(a):
    return (np.asarray(a) + np.pi) % TWO_PI - np.pi


class Window:
    """The oracle's analytic-signal window of one pixel, for the excuse checks."""

    def __init__(self, image, N, L, fb, deriv_axis, carrier_axis, f0, B=0.0):
        self.image, self.N, self.L, self.fb = image, N, L, fb
        self.deriv_axis, self.carrier_axis, self.f0, self.B = deriv_axis, carrier_axis, f0, B
        self._gamma = None

    def gamma(self):
        if self._gamma is None:
            self._gamma = O.analytic_frame(self.image, self.f0, self.B, self.carrier_axis)
        return self._gamma

    def window(self, y, x):
        g, N = self.gamma(), self.N
        if self.deriv_axis == 0:
            return g[y, x - N // 2: x - N // 2 + N]
        return g[y - N // 2: y - N // 2 + N, x]

    def omega_ref(self):
        return TWO_PI * self.f0 if self.deriv_axis == self.carrier_axis else 0.0


def _excuse(win: Window, y, x, g_val, g_st, tol):
    """Why the oracle allows this pixel's GPU result, or None."""
    w = win.window(y, x)
    r = O.window_derivative(w, win.L, win.fb, win.omega_ref())
    if g_st == 2:
        R = O.covariance(w, win.L, win.fb)
        ev, _, _ = O.eig_hermitian(R)
        ev = np.sort(ev)[::-1]
        if ev[0] <= 0 or ev[0] - ev[1] <= GAP_RES * ev[0]:
            return "near degenerate"
        return None
    roots = r["roots"]
    cand = roots[np.abs(roots) <= 1 + 1e-9]
    if cand.size < 2 or g_st != 0 or not np.isfinite(g_val):
        return None
    d = np.abs(np.abs(cand) - 1.0)
    order = np.argsort(d)
    z1, z2 = cand[order[0]], cand[order[1]]
    if d[order[1]] - d[order[0]] > TIE_RES:
        return None
    # a split double root (the two nearest roots form one root) is one candidate, not a tie
    if abs(z1 - z2) < 4e-3:
        return None
    alt = _wrap(np.angle(z2) - win.omega_ref())
    if abs(_wrap(g_val - alt)) <= tol:
        return "near tie"
    return None


def check(g, gs, o, os_, tol, win: Window | None = None, ys=None, xs=None, max_excused=1e-4, what=""):
    """Assert parity of GPU values g / statuses gs with the oracle's o / os_ (same shapes: whole maps,
    or the sampled pixels at (ys, xs)). Returns a small report (compared pixels, max and p99.9 of
    |gpu - oracle| on pixels both call ok, excused pixels by reason)."""
    g = np.asarray(g, dtype=np.float64).ravel()
    gs = np.asarray(gs).ravel()
    o = np.asarray(o, dtype=np.float64).ravel()
    os_ = np.asarray(os_).ravel()
    assert np.array_equal(gs == 1, os_ == 1), f"{what}: border maps differ"
    both = (gs == 0) & (os_ == 0)
    d = np.full(g.shape, np.inf)
    d[both] = np.abs(_wrap(g[both] - o[both]))
    bad = (gs != os_) | (both & (d > tol))
    excused = {}
    if bad.any():
        assert win is not None, (f"{what}: {int(bad.sum())} pixels disagree (statuses {np.unique(gs[bad])} vs "
                                 f"{np.unique(os_[bad])}, max {np.max(d[bad & both], initial=0):.3e})")
        for i in np.flatnonzero(bad):
            if ys is None:
                y, x = np.unravel_index(i, win.image.shape)
            else:
                y, x = int(np.ravel(ys)[i]), int(np.ravel(xs)[i])
            why = _excuse(win, int(y), int(x), g[i], gs[i], tol)
            assert why is not None, (f"{what}: pixel ({y}, {x}) gpu {g[i]:.7f} (status {gs[i]}) vs oracle "
                                     f"{o[i]:.7f} (status {os_[i]}): not a near tie or near-degenerate window")
            excused[why] = excused.get(why, 0) + 1
    n = int((os_ != 1).sum())
    assert sum(excused.values()) <= max(1, max_excused * n), f"{what}: {excused} excused of {n}"
    ok = both & ~bad
    dd = d[ok]
    return {"compared": n, "max": float(dd.max()) if dd.size else 0.0,
            "p999": float(np.quantile(dd, 0.999)) if dd.size else 0.0, "excused": excused}


def rms_check(g, o, truth, mask, rel=0.01, what=""):
    """The GPU's RMS error against the closed-form derivative is within `rel` of the oracle's."""
    rms_o = np.sqrt(np.mean((np.asarray(o, dtype=np.float64)[mask] - truth[mask]) ** 2))
    rms_g = np.sqrt(np.mean((np.asarray(g, dtype=np.float64)[mask] - truth[mask]) ** 2))
    assert abs(rms_g - rms_o) <= rel * rms_o, f"{what}: rms gpu {rms_g:.6e} oracle {rms_o:.6e}"
    return rms_g, rms_o
