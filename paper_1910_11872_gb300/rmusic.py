"""ctypes binding of the C ABI in ``include/rmusic.h``.

The functions here carry the C names and only marshal arguments: every step of the computation
runs in the CUDA library ``_lib/librmusic.so``. There is no CPU or PyTorch fallback: if the
library cannot be loaded (or built), importing the binding's entry points raises.

PyTorch is used only as a source of device memory and streams (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``) by the convenience wrapper ``Demodulator``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

from . import build as _build

RMUSIC_OK = 0
RMUSIC_EINVAL = -1
RMUSIC_ENOMEM = -2
RMUSIC_EUNSUPPORTED = -3
RMUSIC_ETIMEDOUT = -4
RMUSIC_ECUDA = -5
RMUSIC_EAGAIN = -6

RMUSIC_PLAIN_FP64 = 0
RMUSIC_PLAIN_FP32 = 1
RMUSIC_FP32_BATCHED = 2

RMUSIC_DTYPE_F32 = 0
RMUSIC_DTYPE_U16 = 1
RMUSIC_DTYPE_C64 = 2

RMUSIC_GEOM_ROW = 0
RMUSIC_GEOM_SQUARE = 1
GEOMETRIES = {"row": RMUSIC_GEOM_ROW, "square": RMUSIC_GEOM_SQUARE}

STATUS_OK, STATUS_BORDER, STATUS_DEGENERATE, STATUS_NOT_CONVERGED = 0, 1, 2, 3

PRECISIONS = {"plain_fp64": RMUSIC_PLAIN_FP64, "plain_fp32": RMUSIC_PLAIN_FP32,
              "batched": RMUSIC_FP32_BATCHED}


class rmusic_params(ctypes.Structure):
    _fields_ = [
        ("window_len", ctypes.c_int32),
        ("cov_order", ctypes.c_int32),
        ("model_order", ctypes.c_int32),
        ("forward_backward", ctypes.c_int32),
        ("deriv_axis", ctypes.c_int32),
        ("carrier_axis", ctypes.c_int32),
        ("carrier_freq", ctypes.c_double),
        ("band_halfwidth", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("max_sweeps", ctypes.c_int32),
        ("max_root_iters", ctypes.c_int32),
        ("polish_fp64", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("geometry", ctypes.c_int32),
        ("half_width", ctypes.c_int32),
        ("unwrap", ctypes.c_int32),
        ("band_cross", ctypes.c_double),
        ("raw_input", ctypes.c_int32),
        ("exhaustive", ctypes.c_int32),
    ]


class rmusic_frame_desc(ctypes.Structure):
    _fields_ = [
        ("offset_bytes", ctypes.c_uint64),
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("pitch_elems", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("out_offset", ctypes.c_uint64),
        ("window_len", ctypes.c_int32),
        ("cov_order", ctypes.c_int32),
    ]


class rmusic_stats(ctypes.Structure):
    _fields_ = [
        ("kernel_launches", ctypes.c_int32),
        ("graph_replayed", ctypes.c_int32),
        ("workspace_bytes", ctypes.c_uint64),
        ("pixels", ctypes.c_uint64),
        ("mean_sweeps", ctypes.c_double),
        ("mean_root_iters", ctypes.c_double),
        ("mean_root_updates", ctypes.c_double),
        ("mean_root_evals", ctypes.c_double),
        ("bandpass_ms", ctypes.c_float),
        ("solver_ms", ctypes.c_float),
        ("solver_ctas_per_sm", ctypes.c_int32),
        ("solver_variant", ctypes.c_int32),
        ("mean_power_steps", ctypes.c_double),
        ("eig_fallback_frac", ctypes.c_double),
        ("mean_newton_steps", ctypes.c_double),
        ("root_fallback_frac", ctypes.c_double),
        ("mean_polish_steps", ctypes.c_double),
        ("check_violations", ctypes.c_uint64),
        ("wait_timeouts", ctypes.c_uint64),
    ]


class RmusicError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)


_lock = threading.Lock()
_lib: ctypes.CDLL | None = None
_checked = False


def use_checked_build() -> None:
    """Make this process load the checked build (RMUSIC_CHECKS) instead of the ordinary one. Must be
    called before the library is first loaded; for tests that look for out-of-range indices."""
    global _checked
    with _lock:
        if _lib is not None and not _checked:
            raise RuntimeError("the ordinary build is already loaded in this process")
        _checked = True


def library_path() -> str:
    return _build.CHECKED_LIB if _checked else _build.LIB


def load_library(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load librmusic.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.CHECKED_LIB if _checked else _build.LIB
        if build_if_needed:
            _build.build(checked=_checked)
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        lib.rmusic_create.argtypes = [ctypes.POINTER(rmusic_params), ctypes.c_int, ctypes.c_size_t,
                                      ctypes.POINTER(vp)]
        lib.rmusic_create.restype = ctypes.c_int
        lib.rmusic_demodulate_frames.argtypes = [vp, vp, ctypes.POINTER(rmusic_frame_desc), i32, vp, vp, vp]
        lib.rmusic_demodulate_frames.restype = ctypes.c_int
        lib.rmusic_demodulate_frames_host.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(rmusic_frame_desc),
                                                      i32, vp, vp, vp]
        lib.rmusic_demodulate_frames_host.restype = ctypes.c_int
        lib.rmusic_demodulate_frames_host_async.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(rmusic_frame_desc),
                                                      i32, vp, vp, vp]
        lib.rmusic_demodulate_frames_host_async.restype = ctypes.c_int
        lib.rmusic_demodulate_frames_noalloc.argtypes = [ctypes.POINTER(rmusic_params), ctypes.c_int, vp,
                                                         ctypes.POINTER(rmusic_frame_desc), i32, vp, vp, vp]
        lib.rmusic_demodulate_frames_noalloc.restype = ctypes.c_int
        lib.rmusic_autotune.argtypes = [vp, vp, ctypes.POINTER(rmusic_frame_desc), i32, vp, vp, vp]
        lib.rmusic_autotune.restype = ctypes.c_int
        lib.rmusic_reserve.argtypes = [vp, ctypes.c_uint64, i32]
        lib.rmusic_reserve.restype = ctypes.c_int
        lib.rmusic_destroy.argtypes = [vp]
        lib.rmusic_destroy.restype = None
        lib.rmusic_strerror.argtypes = [ctypes.c_int]
        lib.rmusic_strerror.restype = ctypes.c_char_p
        lib.rmusic_last_cuda_error.argtypes = [vp]
        lib.rmusic_last_cuda_error.restype = ctypes.c_char_p
        lib.rmusic_checked_build.argtypes = []
        lib.rmusic_checked_build.restype = ctypes.c_int
        lib.rmusic_set_solver_variant.argtypes = [vp, i32, i32]
        lib.rmusic_set_solver_variant.restype = ctypes.c_int
        lib.rmusic_unwrap_phase.argtypes = [vp, vp, ctypes.POINTER(rmusic_frame_desc), i32, vp, vp]
        lib.rmusic_unwrap_phase.restype = ctypes.c_int
        lib.rmusic_unwrap_phase_sched.argtypes = [vp, vp, ctypes.POINTER(rmusic_frame_desc), i32, vp, i32, vp]
        lib.rmusic_unwrap_phase_sched.restype = ctypes.c_int
        lib.rmusic_get_stats.argtypes = [vp, ctypes.POINTER(rmusic_stats)]
        lib.rmusic_get_stats.restype = ctypes.c_int
        _lib = lib
        return lib


# ------------------------------------------------------------------------------------------
# C entry points, same names
# ------------------------------------------------------------------------------------------
def rmusic_strerror(code: int) -> str:
    return load_library().rmusic_strerror(int(code)).decode()


strerror = rmusic_strerror


def rmusic_create(params: rmusic_params, device: int = 0, hbm_budget_bytes: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    rc = load_library().rmusic_create(ctypes.byref(params), int(device), int(hbm_budget_bytes), ctypes.byref(ctx))
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_create")
    return ctx


def _desc_array(descs: Sequence[rmusic_frame_desc]):
    if isinstance(descs, ctypes.Array):
        return descs
    arr = (rmusic_frame_desc * max(len(descs), 1))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def rmusic_demodulate_frames(ctx, d_frames: int, descs, n_frames: int, d_out: int, d_status: int | None,
                             cuda_stream: int | None) -> int:
    arr = _desc_array(descs)
    rc = load_library().rmusic_demodulate_frames(ctx, d_frames or None, arr, int(n_frames), d_out or None,
                                                 d_status or None, cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_demodulate_frames", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_demodulate_frames_host(ctx, h_frames: int, in_bytes: int, descs, n_frames: int, h_out: int,
                                  h_status: int | None, cuda_stream: int | None) -> int:
    arr = _desc_array(descs)
    rc = load_library().rmusic_demodulate_frames_host(ctx, h_frames or None, int(in_bytes), arr, int(n_frames),
                                                      h_out or None, h_status or None, cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_demodulate_frames_host", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_demodulate_frames_host_async(ctx, h_frames: int, in_bytes: int, descs, n_frames: int, h_out: int,
                                        h_status: int | None, cuda_stream: int | None) -> int:
    arr = _desc_array(descs)
    rc = load_library().rmusic_demodulate_frames_host_async(ctx, h_frames or None, int(in_bytes), arr, int(n_frames),
                                                            h_out or None, h_status or None, cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_demodulate_frames_host_async", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_demodulate_frames_noalloc(params: rmusic_params, device: int, d_frames: int, descs, n_frames: int,
                                     d_out: int, d_status: int | None, cuda_stream: int | None) -> int:
    """The context-free FP32-batched entry point that allocates no device memory (for callers
    that cannot allocate); its scratch is a fixed array inside the library (see rmusic.h)."""
    arr = _desc_array(descs)
    rc = load_library().rmusic_demodulate_frames_noalloc(ctypes.byref(params), int(device), d_frames or None, arr,
                                                         int(n_frames), d_out or None, d_status or None,
                                                         cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_demodulate_frames_noalloc")
    return rc


def rmusic_reserve(ctx, max_pixels: int, max_frames: int) -> int:
    rc = load_library().rmusic_reserve(ctx, int(max_pixels), int(max_frames))
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_reserve", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_autotune(ctx, d_frames: int, descs, n_frames: int, d_out: int, d_status: int | None,
                    cuda_stream: int | None) -> int:
    arr = _desc_array(descs)
    rc = load_library().rmusic_autotune(ctx, d_frames or None, arr, int(n_frames), d_out or None, d_status or None,
                                        cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_autotune", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_unwrap_phase(ctx, d_phase: int, descs, n_frames: int, d_out: int, cuda_stream: int | None) -> int:
    arr = _desc_array(descs)
    rc = load_library().rmusic_unwrap_phase(ctx, d_phase or None, arr, int(n_frames), d_out or None,
                                            cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_unwrap_phase", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_unwrap_phase_sched(ctx, d_phase: int, descs, n_frames: int, d_out: int, launched_rounds: int,
                              cuda_stream: int | None) -> int:
    arr = _desc_array(descs)
    rc = load_library().rmusic_unwrap_phase_sched(ctx, d_phase or None, arr, int(n_frames), d_out or None,
                                                  int(launched_rounds), cuda_stream or None)
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_unwrap_phase_sched", rmusic_last_cuda_error(ctx))
    return rc


def rmusic_set_solver_variant(ctx, order: int, variant: int) -> int:
    rc = load_library().rmusic_set_solver_variant(ctx, int(order), int(variant))
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_set_solver_variant")
    return rc


def rmusic_destroy(ctx) -> None:
    if ctx:
        load_library().rmusic_destroy(ctx)


def rmusic_last_cuda_error(ctx) -> str:
    r = load_library().rmusic_last_cuda_error(ctx)
    return r.decode() if r else ""


def rmusic_get_stats(ctx) -> rmusic_stats:
    st = rmusic_stats()
    rc = load_library().rmusic_get_stats(ctx, ctypes.byref(st))
    if rc != RMUSIC_OK:
        raise RmusicError(rc, "rmusic_get_stats")
    return st


# ------------------------------------------------------------------------------------------
# Convenience wrapper over torch tensors (marshalling only)
# ------------------------------------------------------------------------------------------
def make_params(window_len=32, cov_order=8, forward_backward=1, deriv_axis=0, carrier_axis=0,
                carrier_freq=0.1, band_halfwidth=0.0, precision="batched", max_sweeps=0,
                max_root_iters=0, polish_fp64=0, use_graph=0, timing=0, autotune=0,
                model_order=1, geometry="row", half_width=0, unwrap=0, band_cross=0.0,
                raw_input=0, exhaustive=0) -> rmusic_params:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    geom = GEOMETRIES[geometry] if isinstance(geometry, str) else int(geometry)
    return rmusic_params(window_len, cov_order, model_order, forward_backward, deriv_axis, carrier_axis,
                         float(carrier_freq), float(band_halfwidth), prec, max_sweeps, max_root_iters,
                         polish_fp64, use_graph, timing, autotune, geom, half_width, unwrap, float(band_cross),
                         int(raw_input), int(exhaustive))


def frame_descs(shapes, dtype_code: int, elem_bytes: int, windows=None, maps: int = 1):
    """Descriptors for frames packed back to back (frame f after frame f-1) and maps packed the same
    way. ``shapes`` is a list of (H, W); ``windows`` an optional list of (N, L) per frame; ``maps``
    the maps a frame writes (3 in the square geometry: d/dx, d/dy, alpha)."""
    descs = (rmusic_frame_desc * max(len(shapes), 1))()
    off = 0
    oo = 0
    for i, (H, W) in enumerate(shapes):
        N, L = windows[i] if windows is not None else (0, 0)
        descs[i] = rmusic_frame_desc(off, H, W, 0, dtype_code, oo, N, L)
        off += H * W * elem_bytes
        oo += maps * H * W
    return descs, off, oo


class Demodulator:
    """Owns one rmusic context. ``run`` takes a CUDA tensor of frames (T, H, W) or a list of 2-D
    CUDA tensors of uneven sizes (float32, uint16 or complex64), and returns the flat map buffer,
    the status buffer and the shapes. Row geometry: one derivative map per frame. Square geometry:
    three maps per frame (d/dx, d/dy, alpha; a fourth, the unwrapped phase, with unwrap=1), frame
    f's block after frame f-1's; the status buffer has the same length, frame f's status map at the
    start of its block."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, **params):
        self.params = make_params(**params)
        self.device = device
        self.ctx = rmusic_create(self.params, device, hbm_budget_bytes)

    def close(self):
        if getattr(self, "ctx", None):
            rmusic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> rmusic_stats:
        return rmusic_get_stats(self.ctx)

    def reserve(self, max_pixels: int, max_frames: int) -> None:
        """Pre-allocate the workspace for calls of up to max_pixels pixels in max_frames frames."""
        rmusic_reserve(self.ctx, max_pixels, max_frames)

    def run(self, frames, windows=None, with_status: bool = True, stream=None, out=None, status=None):
        import torch

        if isinstance(frames, torch.Tensor):
            frames = frames if frames.dim() == 3 else frames.unsqueeze(0)
            flat = frames.contiguous()
            shapes = [tuple(flat.shape[1:])] * flat.shape[0]
        else:
            shapes = [tuple(f.shape) for f in frames]
            flat = torch.cat([f.contiguous().reshape(-1) for f in frames])
        if flat.dtype == torch.float32:
            code, esz = RMUSIC_DTYPE_F32, 4
        elif flat.dtype == torch.uint16 if hasattr(torch, "uint16") else False:
            code, esz = RMUSIC_DTYPE_U16, 2
        elif flat.dtype == torch.int16:
            code, esz = RMUSIC_DTYPE_U16, 2
        elif flat.dtype == torch.complex64:
            code, esz = RMUSIC_DTYPE_C64, 8
        else:
            raise TypeError(f"frames must be float32, uint16 or complex64, got {flat.dtype}")
        maps = 3 + self.params.unwrap if self.params.geometry == RMUSIC_GEOM_SQUARE else 1
        descs, _, nout = frame_descs(shapes, code, esz, windows, maps)
        dev = flat.device
        if out is None:
            out = torch.empty(nout, dtype=torch.float32, device=dev)
        if with_status and status is None:
            status = torch.empty(nout, dtype=torch.uint8, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        rmusic_demodulate_frames(self.ctx, flat.data_ptr(), descs, len(shapes), out.data_ptr(),
                                 status.data_ptr() if with_status else None, s.cuda_stream)
        return out, status, shapes
