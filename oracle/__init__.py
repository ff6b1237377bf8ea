"""FP64 CPU oracle for the sliding-window root-MUSIC phase-derivative path (arXiv:1910.11872).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package. The product path (the CUDA library and its binding)
never calls it and shares no code with it.

The arithmetic lives in ``rmusic_oracle.c`` (plain C99, double precision, one function per
step of the method, each citing the section or equation it follows). This module only compiles
it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmusic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, U16, F64, C64, C128 = 0, 1, 2, 3, 4
STATUS_OK, STATUS_BORDER, STATUS_DEGENERATE, STATUS_NOT_CONVERGED = 0, 1, 2, 3


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in rmusic_oracle.c."""

    _fields_ = [
        ("window_len", ctypes.c_int32),
        ("cov_order", ctypes.c_int32),
        ("model_order", ctypes.c_int32),
        ("forward_backward", ctypes.c_int32),
        ("deriv_axis", ctypes.c_int32),
        ("carrier_axis", ctypes.c_int32),
        ("carrier_freq", ctypes.c_double),
        ("band_halfwidth", ctypes.c_double),
        ("band_cross", ctypes.c_double),
        ("raw_input", ctypes.c_int32),
    ]


def make_params(window_len=32, cov_order=8, forward_backward=1, deriv_axis=0, carrier_axis=0,
                carrier_freq=0.1, band_halfwidth=0.0, model_order=1, band_cross=0.0, raw_input=0) -> Params:
    return Params(window_len, cov_order, model_order, forward_backward, deriv_axis, carrier_axis,
                  float(carrier_freq), float(band_halfwidth), float(band_cross), int(raw_input))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available). Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


class use_library:
    """Context manager that routes every call in this module to another build of the oracle
    (used by the mutation tests, which plant a mistake in a copy of the source)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        with _lock:
            self._saved = _lib
            _lib = ctypes.CDLL(self.path)
            _declare(_lib)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a (modified) copy of the oracle source to ``out_path`` (no OpenMP)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-std=c11", "-O1", "-ffp-contract=off", "-fPIC", "-shared", src, "-o",
                    out_path, "-lm"], check=True, capture_output=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _declare(L: ctypes.CDLL) -> None:
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    i32 = ctypes.c_int32
    L.orc_analytic_line.argtypes = [dp, i32, ctypes.c_double, ctypes.c_double, dp]
    L.orc_analytic_frame.argtypes = [ctypes.c_void_p, i32, i32, i32, i32, ctypes.c_double,
                                     ctypes.c_double, dp]
    L.orc_cross_band.argtypes = [dp, i32, i32, i32, ctypes.c_double]
    L.orc_window_derivative_p_ri.argtypes = [dp, i32, i32, i32, i32, ctypes.c_double, dp, dp]
    L.orc_covariance_ri.argtypes = [dp, i32, i32, i32, dp]
    L.orc_covariance_ri.restype = None
    L.orc_eig_hermitian_ri.argtypes = [dp, i32, dp, dp]
    L.orc_music_poly_ri.argtypes = [dp, i32, dp]
    L.orc_music_poly_ri.restype = None
    L.orc_poly_roots_ri.argtypes = [dp, i32, dp, ip]
    L.orc_select_root_ri.argtypes = [dp, i32, dp, i32, ctypes.c_double, dp]
    L.orc_window_derivative_ri.argtypes = [dp, i32, i32, i32, ctypes.c_double, dp, dp, dp, dp,
                                           ip, dp]
    L.orc_demodulate.argtypes = [ctypes.c_void_p, i32, i32, i32, ctypes.POINTER(Params), dp,
                                 ctypes.c_void_p, i32]
    L.orc_demodulate_pixels.argtypes = [ctypes.c_void_p, i32, i32, i32, ctypes.POINTER(Params),
                                        i32, ip, ip, dp, ctypes.c_void_p, i32]
    L.orc_max_threads.argtypes = []
    fp = ctypes.POINTER(ctypes.c_float)
    L.orc_unwrap_reliability.argtypes = [fp, i32, i32, fp]
    L.orc_unwrap_reliability.restype = None
    L.orc_unwrap.argtypes = [fp, i32, i32, dp, ip]
    L.orc_square_window_ri.argtypes = [dp, i32, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
    L.orc_square_demodulate.argtypes = [ctypes.c_void_p, i32, i32, i32, ctypes.POINTER(Params), i32,
                                        dp, dp, dp, ctypes.c_void_p, i32]
    L.orc_square_demodulate_pixels.argtypes = [ctypes.c_void_p, i32, i32, i32, ctypes.POINTER(Params),
                                               i32, i32, ip, ip, dp, dp, dp, ctypes.c_void_p, i32]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c2ri(z) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    return np.ascontiguousarray(z.view(np.float64))


def _ri2c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a).view(np.complex128)


def _dtype_code(frame: np.ndarray) -> int:
    if frame.dtype == np.float32:
        return F32
    if frame.dtype == np.uint16:
        return U16
    if frame.dtype == np.float64:
        return F64
    if frame.dtype == np.complex64:
        return C64
    if frame.dtype == np.complex128:
        return C128
    raise TypeError(f"unsupported frame dtype {frame.dtype}")


# ---------------------------------------------------------------------------------------------
# Step-level entry points (pin tests)
# ---------------------------------------------------------------------------------------------
def analytic_line(v, f0: float, B: float = 0.0) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(2 * v.size)
    rc = lib().orc_analytic_line(_dp(v), v.size, f0, B, _dp(out))
    assert rc == 0
    return _ri2c(out)


def analytic_frame(frame: np.ndarray, f0: float, B: float = 0.0, carrier_axis: int = 0) -> np.ndarray:
    frame = np.ascontiguousarray(frame)
    H, W = frame.shape
    if B <= 0:
        B = 0.5 * f0
    out = np.zeros(2 * H * W)
    rc = lib().orc_analytic_frame(frame.ctypes.data, _dtype_code(frame), H, W, carrier_axis, f0, B,
                                  _dp(out))
    assert rc == 0
    return _ri2c(out).reshape(H, W)


def cross_band(gamma, Bc: float, carrier_axis: int = 0) -> np.ndarray:
    """The 2-D variant's second pass on an analytic-signal frame: low-pass |k / len| < Bc across
    the carrier lines."""
    g = np.ascontiguousarray(np.asarray(gamma, dtype=np.complex128))
    H, W = g.shape
    buf = np.ascontiguousarray(g.view(np.float64).ravel())
    rc = lib().orc_cross_band(_dp(buf), H, W, carrier_axis, float(Bc))
    assert rc == 0
    return buf.view(np.complex128).reshape(H, W)


def covariance(w, L: int, fb: int = 1) -> np.ndarray:
    w = _c2ri(w)
    N = w.size // 2
    R = np.zeros(2 * L * L)
    lib().orc_covariance_ri(_dp(w), N, L, fb, _dp(R))
    return _ri2c(R).reshape(L, L)


def eig_hermitian(R) -> tuple[np.ndarray, np.ndarray, int]:
    R = np.asarray(R, dtype=np.complex128)
    L = R.shape[0]
    ev = np.zeros(L)
    V = np.zeros(2 * L * L)
    sweeps = lib().orc_eig_hermitian_ri(_dp(_c2ri(R)), L, _dp(ev), _dp(V))
    return ev, _ri2c(V).reshape(L, L), sweeps


def music_poly(u) -> np.ndarray:
    u = _c2ri(u)
    L = u.size // 2
    q = np.zeros(2 * (2 * L - 1))
    lib().orc_music_poly_ri(_dp(u), L, _dp(q))
    return _ri2c(q)


def poly_roots(q) -> tuple[np.ndarray, bool]:
    """Roots of sum_i q[i] z^i (ascending powers)."""
    qr = _c2ri(q)
    deg = qr.size // 2 - 1
    out = np.zeros(2 * max(deg, 1))
    nc = ctypes.c_int32(0)
    n = lib().orc_poly_roots_ri(_dp(qr), deg, _dp(out), ctypes.byref(nc))
    return _ri2c(out)[:n].copy(), bool(nc.value)


def select_root(q, roots, omega_ref: float = 0.0) -> complex | None:
    """Selected root of the polynomial with ascending coefficients q, given its roots."""
    qr = _c2ri(q)
    r = _c2ri(roots)
    z = np.zeros(2)
    rc = lib().orc_select_root_ri(_dp(qr), qr.size // 2 - 1, _dp(r), r.size // 2, omega_ref, _dp(z))
    return None if rc != 0 else complex(z[0], z[1])


def window_derivative(w, L: int, fb: int = 1, omega_ref: float = 0.0) -> dict:
    """Steps 4-9 for one analytic-signal window. Returns a dict of all intermediates."""
    wr = _c2ri(w)
    N = wr.size // 2
    d = np.zeros(1)
    u = np.zeros(2 * L)
    q = np.zeros(2 * (2 * L - 1))
    r = np.zeros(2 * (2 * L - 2))
    nr = ctypes.c_int32(0)
    z = np.zeros(2)
    st = lib().orc_window_derivative_ri(_dp(wr), N, L, fb, omega_ref, _dp(d), _dp(u), _dp(q),
                                        _dp(r), ctypes.byref(nr), _dp(z))
    return {"deriv": float(d[0]), "status": int(st), "u1": _ri2c(u), "q": _ri2c(q),
            "roots": _ri2c(r)[: nr.value].copy(), "zsel": complex(z[0], z[1])}


def window_derivative_p(w, L: int, p: int, fb: int = 1, omega_ref: float = 0.0) -> dict:
    """Steps 4-9 with model order p (1..3) for one window."""
    wr = _c2ri(w)
    d = np.zeros(1)
    z = np.zeros(2)
    st = lib().orc_window_derivative_p_ri(_dp(wr), wr.size // 2, L, fb, p, omega_ref, _dp(d), _dp(z))
    return {"deriv": float(d[0]), "status": int(st), "zsel": complex(z[0], z[1])}


# ---------------------------------------------------------------------------------------------
# Frame-level entry points
# ---------------------------------------------------------------------------------------------
def demodulate(frame: np.ndarray, params: Params, nthreads: int = 0) -> tuple[np.ndarray, np.ndarray, int]:
    """Derivative map (float64, NaN where undefined), status map (uint8), threads used."""
    frame = np.ascontiguousarray(frame)
    H, W = frame.shape
    out = np.empty(H * W)
    st = np.empty(H * W, dtype=np.uint8)
    used = lib().orc_demodulate(frame.ctypes.data, _dtype_code(frame), H, W, ctypes.byref(params),
                                _dp(out), st.ctypes.data, nthreads)
    if used < 0:
        raise ValueError(f"oracle rejected the input (code {used})")
    return out.reshape(H, W), st.reshape(H, W), used


def demodulate_pixels(frame: np.ndarray, params: Params, ys, xs, nthreads: int = 0):
    """Derivative at the listed pixels only. Returns (values, status, threads used)."""
    frame = np.ascontiguousarray(frame)
    H, W = frame.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.empty(ys.size)
    st = np.empty(ys.size, dtype=np.uint8)
    ip = ctypes.POINTER(ctypes.c_int32)
    used = lib().orc_demodulate_pixels(frame.ctypes.data, _dtype_code(frame), H, W,
                                       ctypes.byref(params), ys.size, ys.ctypes.data_as(ip),
                                       xs.ctypes.data_as(ip), _dp(out), st.ctypes.data, nthreads)
    if used < 0:
        raise ValueError(f"oracle rejected the input (code {used})")
    return out, st, used


# ---------------------------------------------------------------------------------------------
# The paper's square block geometry (Sec. 3, Eq. 4-15, Algorithm 1)
# ---------------------------------------------------------------------------------------------
def square_window(G, ref_x: float = 0.0, ref_y: float = 0.0) -> dict:
    """One (2Lp+1) x (2Lp+1) block G (rows: y, columns: x). Returns the raw angles omega_x,
    omega_y (carrier included), alpha, the status and the intermediates u1, v1, zx, zy."""
    G = np.asarray(G, dtype=np.complex128)
    M = G.shape[0]
    assert G.shape == (M, M) and M % 2 == 1
    Lp = (M - 1) // 2
    out = np.zeros(3)
    u = np.zeros(2 * M)
    v = np.zeros(2 * M)
    z = np.zeros(4)
    st = lib().orc_square_window_ri(_dp(_c2ri(G.ravel())), Lp, ref_x, ref_y, _dp(out), _dp(u), _dp(v), _dp(z))
    return {"wx": float(out[0]), "wy": float(out[1]), "alpha": float(out[2]), "status": int(st),
            "u1": _ri2c(u), "v1": _ri2c(v), "zx": complex(z[0], z[1]), "zy": complex(z[2], z[3])}


def square_demodulate(frame: np.ndarray, params: Params, Lp: int, nthreads: int = 0):
    """Paper geometry over a whole frame: (dx, dy, alpha, status, threads used); maps are
    float64 with NaN where undefined."""
    frame = np.ascontiguousarray(frame)
    H, W = frame.shape
    dx, dy, al = np.empty(H * W), np.empty(H * W), np.empty(H * W)
    st = np.empty(H * W, dtype=np.uint8)
    used = lib().orc_square_demodulate(frame.ctypes.data, _dtype_code(frame), H, W, ctypes.byref(params),
                                       Lp, _dp(dx), _dp(dy), _dp(al), st.ctypes.data, nthreads)
    if used < 0:
        raise ValueError(f"oracle rejected the input (code {used})")
    return dx.reshape(H, W), dy.reshape(H, W), al.reshape(H, W), st.reshape(H, W), used


def square_demodulate_pixels(frame: np.ndarray, params: Params, Lp: int, ys, xs, nthreads: int = 0):
    """Paper geometry at the listed pixels only: (dx, dy, alpha, status, threads used)."""
    frame = np.ascontiguousarray(frame)
    H, W = frame.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    n = ys.size
    dx, dy, al = np.empty(n), np.empty(n), np.empty(n)
    st = np.empty(n, dtype=np.uint8)
    ip = ctypes.POINTER(ctypes.c_int32)
    used = lib().orc_square_demodulate_pixels(frame.ctypes.data, _dtype_code(frame), H, W,
                                              ctypes.byref(params), Lp, n, ys.ctypes.data_as(ip),
                                              xs.ctypes.data_as(ip), _dp(dx), _dp(dy), _dp(al),
                                              st.ctypes.data, nthreads)
    if used < 0:
        raise ValueError(f"oracle rejected the input (code {used})")
    return dx, dy, al, st, used


# ---------------------------------------------------------------------------------------------
# Phase assembly: the reliability-sorting unwrapper the paper cites (Sec. 3)
# ---------------------------------------------------------------------------------------------
def unwrap_reliability(phi) -> np.ndarray:
    """Reliability map (float32) of a wrapped float32 map (NaN = no value)."""
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    H, W = phi.shape
    R = np.empty_like(phi)
    fp = ctypes.POINTER(ctypes.c_float)
    lib().orc_unwrap_reliability(phi.ctypes.data_as(fp), H, W, R.ctypes.data_as(fp))
    return R


def unwrap(phi):
    """Unwrap a wrapped float32 map (NaN = no value). Returns (unwrapped float64, k int32 with
    unwrapped = phi + 2 pi k, number of groups left)."""
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    H, W = phi.shape
    out = np.empty((H, W))
    k = np.empty((H, W), dtype=np.int32)
    fp = ctypes.POINTER(ctypes.c_float)
    n = lib().orc_unwrap(phi.ctypes.data_as(fp), H, W, _dp(out), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if n < 0:
        raise MemoryError("oracle unwrap: allocation failed")
    return out, k, n


def max_threads() -> int:
    return int(lib().orc_max_threads())
