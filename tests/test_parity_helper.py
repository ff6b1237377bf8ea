"""The GPU-vs-oracle comparison rule itself (tests/parity.py), exercised on the CPU with the oracle's
own maps and planted disagreements: a changed value or status that the oracle's roots and
eigenvalues do not excuse must be rejected."""
import numpy as np
import pytest

import oracle as O
import parity
from paper_1910_11872_gb300 import synth


@pytest.fixture(scope="module")
def maps():
    fr = synth.peaks_frame(10, 0.1, H=12, W=160)
    o, st, _ = O.demodulate(fr.image, O.make_params(32, 8, 1, 0, 0, 0.1))
    return fr, o, st


def test_identical_maps_pass(maps):
    fr, o, st = maps
    rep = parity.check(o.astype(np.float32), st, o, st, 1e-4, parity.Window(fr.image, 32, 8, 1, 0, 0, 0.1))
    assert rep["excused"] == {} and rep["max"] <= 1e-7
    assert rep["compared"] == (st != 1).sum()


def test_planted_value_error_is_rejected(maps):
    fr, o, st = maps
    g = o.copy()
    y, x = 5, 80
    assert st[y, x] == 0
    g[y, x] += 3e-4  # not another root of the window
    with pytest.raises(AssertionError, match="not a near tie"):
        parity.check(g, st, o, st, 1e-4, parity.Window(fr.image, 32, 8, 1, 0, 0, 0.1))
    # without a window to consult, any disagreement fails
    with pytest.raises(AssertionError, match="disagree"):
        parity.check(g, st, o, st, 1e-4)


def test_planted_status_errors_are_rejected(maps):
    fr, o, st = maps
    win = parity.Window(fr.image, 32, 8, 1, 0, 0, 0.1)
    for new in (2, 3):  # degenerate on a well-separated window; not converged
        gs = st.copy()
        gs[6, 90] = new
        with pytest.raises(AssertionError):
            parity.check(o, gs, o, st, 1e-4, win)
    gs = st.copy()
    gs[0, 3] = 0  # a border pixel called ok
    with pytest.raises(AssertionError, match="border"):
        parity.check(o, gs, o, st, 1e-4, win)


def test_rms_check(maps):
    fr, o, st = maps
    v = st == 0
    parity.rms_check(o, o, fr.truth, v)
    with pytest.raises(AssertionError):
        parity.rms_check(o + 0.05 * np.sign(o - fr.truth), o, fr.truth, v)
