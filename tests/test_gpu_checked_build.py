"""The checked build (RMUSIC_CHECKS): the solvers test their work items' data-dependent indices and
count failures instead of touching memory out of range -- the stand-in for a device memory checker,
which this pool does not offer. On ragged and tiny frames, every covariance order, row and column
windows, the exhaustive root finder, every square half-width class and the asynchronous host entry,
no test may fail, and the maps must be those of the ordinary build: identical statuses, values within
FP32 rounding (the extra tests can change the compiler's instruction selection, as between the
solver's register-cap variants)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _child(mode, path):
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_build_child.py"), mode, path],
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_finds_no_bad_index_and_matches(tmp_path):
    pytest.importorskip("torch")
    plain = str(tmp_path / "plain.npz")
    checked = str(tmp_path / "checked.npz")
    vp = _child("plain", plain)
    vc = _child("checked", checked)
    assert all(v == 0 for v in vp.values()), vp  # the ordinary build counts nothing
    assert all(v == 0 for v in vc.values()), vc
    a, b = np.load(plain), np.load(checked)
    assert sorted(a.files) == sorted(b.files)
    for name in a.files:
        if name.endswith("_st"):
            assert np.array_equal(a[name], b[name]), name
    for name in a.files:
        if name.endswith("_out"):
            x, y = a[name], b[name]
            assert np.array_equal(np.isnan(x), np.isnan(y)), name
            ok = ~np.isnan(x)
            d = np.abs(((x[ok] - y[ok]) + np.pi) % (2 * np.pi) - np.pi)
            assert d.max(initial=0.0) <= 3e-5, (name, d.max())
