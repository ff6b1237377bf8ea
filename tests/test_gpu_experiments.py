"""The paper's accuracy experiments (Sec. 4: Table 1, Fig. 4) through the GPU path on full
512 x 512 frames of the synthetic stand-in, with the statistic cross-checked against the oracle on
sampled pixels. Trend checks as in test_oracle_experiments.py, plus the unwrapped phase: at L = 1
unwrapping slips make the phase error large (the paper's Table 1 gives 5.4 rad there)."""
import numpy as np
import pytest

import oracle as O
from paper_1910_11872_gb300 import experiments as E
from paper_1910_11872_gb300 import synth

pytestmark = pytest.mark.gpu


def test_half_width_sweep_u_shape_and_oracle_agreement():
    rows = E.rmse_vs_half_width(range(1, 9), snr_db=0.0, size=512, hi=150.0)
    a = [r["alpha_rmse"] for r in rows]
    p = [r["phase_rmse"] for r in rows]
    best = int(np.argmin(a)) + 1
    assert 3 <= best <= 5, a
    assert a[0] > 4 * min(a) and a[-1] > 1.5 * min(a), a
    assert p[0] > 10 * min(p[1:]), p            # slips at the smallest window
    assert int(np.argmin(p)) + 1 == best or abs(p[best - 1] - min(p)) < 0.02 * min(p), (p, a)
    # the GPU statistic against the oracle's on the same pixels
    fr = synth.complex_fringe_frame(0.0, 512, 512, 150.0)
    rng = np.random.default_rng(1)
    ys, xs = rng.integers(8, 504, 1000), rng.integers(8, 504, 1000)
    for Lp in (2, 4, 7):
        g = E.square_maps(fr.image, Lp)[2][ys, xs]
        _, _, o, _, _ = O.square_demodulate_pixels(fr.image, O.make_params(carrier_freq=0.0), Lp, ys, xs)
        eg, eo = E.wrapped_rmse(g, fr.meta["phi"][ys, xs]), E.wrapped_rmse(o, fr.meta["phi"][ys, xs])
        assert abs(eg - eo) <= 0.01 * eo, (Lp, eg, eo)


def test_snr_sweep_monotone():
    rows = E.rmse_vs_snr((-5.0, 0.0, 5.0, 10.0, 15.0, 20.0), Lp=4, size=512, hi=150.0)
    for key in ("alpha_rmse", "phase_rmse", "dx_rmse", "dy_rmse"):
        v = [r[key] for r in rows]
        assert all(v[i] > v[i + 1] for i in range(len(v) - 1)), (key, v)
