"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every function that
include/rmusic.h declares, its structs have the layout the binding assumes, and argument checks
that return before any CUDA call behave as documented. No GPU work is done here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1910_11872_gb300 import build, rmusic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rmusic_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rmusic_create", "rmusic_demodulate_frames", "rmusic_destroy", "rmusic_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_library_is_built_for_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert all("sm_" not in f or "sm_103a" in f for f in build.FLAGS)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rmusic.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu\\n", sizeof(rmusic_params), offsetof(rmusic_params, carrier_freq),'
        " offsetof(rmusic_params, precision), offsetof(rmusic_params, use_graph), sizeof(rmusic_frame_desc));\n"
        'printf("%zu %zu %zu\\n", offsetof(rmusic_frame_desc, out_offset), offsetof(rmusic_frame_desc, cov_order),'
        " sizeof(rmusic_stats));\n"
        'printf("%zu %zu %zu %zu\\n", offsetof(rmusic_params, geometry), offsetof(rmusic_params, half_width),'
        " offsetof(rmusic_params, unwrap), offsetof(rmusic_params, band_cross));\n"
        'printf("%zu\\n", offsetof(rmusic_params, raw_input));\n'
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b, c, d = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:4]
    P, D, S = rmusic.rmusic_params, rmusic.rmusic_frame_desc, rmusic.rmusic_stats
    assert list(map(int, a.split())) == [ctypes.sizeof(P), P.carrier_freq.offset, P.precision.offset,
                                         P.use_graph.offset, ctypes.sizeof(D)]
    assert list(map(int, b.split())) == [D.out_offset.offset, D.cov_order.offset, ctypes.sizeof(S)]
    assert list(map(int, c.split())) == [P.geometry.offset, P.half_width.offset, P.unwrap.offset,
                                         P.band_cross.offset]
    assert int(d) == P.raw_input.offset


def test_argument_checks_without_cuda(lib):
    L = rmusic.load_library()
    assert L.rmusic_create(None, 0, 0, None) == rmusic.RMUSIC_EINVAL
    p = rmusic.make_params()
    assert L.rmusic_create(ctypes.byref(p), 0, 0, None) == rmusic.RMUSIC_EINVAL
    assert L.rmusic_demodulate_frames(None, None, None, 1, None, None, None) == rmusic.RMUSIC_EINVAL
    assert L.rmusic_get_stats(None, None) == rmusic.RMUSIC_EINVAL
    L.rmusic_destroy(None)
    assert rmusic.rmusic_strerror(rmusic.RMUSIC_ENOMEM).startswith("out of memory")
    assert rmusic.rmusic_strerror(12345) == "unknown error"
    bad = rmusic.make_params(model_order=4)
    ctx = ctypes.c_void_p()
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EUNSUPPORTED
    bad = rmusic.make_params(model_order=2)  # the batched model-order solver takes raw real lines only
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EUNSUPPORTED
    bad = rmusic.make_params(model_order=2, precision="plain_fp32", raw_input=1, deriv_axis=1)
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EINVAL
    bad = rmusic.make_params(window_len=8, cov_order=12)
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EINVAL
    # the square block: half-width 1 .. 8, FP32-batched only
    for hw in (0, 9):
        bad = rmusic.make_params(geometry="square", half_width=hw)
        assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EINVAL
    bad = rmusic.make_params(geometry="square", half_width=5, precision="plain_fp32")
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EUNSUPPORTED
    bad = rmusic.make_params(geometry=2)
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EINVAL
    bad = rmusic.make_params(unwrap=1)  # phase assembly needs the square geometry's alpha maps
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EINVAL
    assert L.rmusic_unwrap_phase(None, None, None, 1, None, None) == rmusic.RMUSIC_EINVAL
    assert L.rmusic_unwrap_phase_sched(None, None, None, 1, None, -1, None) == rmusic.RMUSIC_EINVAL
    bad = rmusic.make_params(band_cross=0.5)
    assert L.rmusic_create(ctypes.byref(bad), 0, 0, ctypes.byref(ctx)) == rmusic.RMUSIC_EINVAL
