"""ctypes binding of the serving loop's C ABI (``include/rmusic_serve.h``): same function names,
argument marshalling only. ``Server`` is a small convenience wrapper."""
from __future__ import annotations

import ctypes

from . import rmusic as _rm


class rmusic_serve_config(ctypes.Structure):
    _fields_ = [
        ("max_streams", ctypes.c_int32),
        ("ring_depth", ctypes.c_int32),
        ("max_batch_frames", ctypes.c_int32),
        ("inflight_batches", ctypes.c_int32),
        ("max_batch_pixels", ctypes.c_uint64),
        ("hbm_budget_bytes", ctypes.c_uint64),
    ]


class rmusic_completion(ctypes.Structure):
    _fields_ = [
        ("stream_id", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("tag", ctypes.c_uint64),
        ("t_submit", ctypes.c_double),
        ("t_launch", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("batch_frames", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
    ]


class rmusic_serve_stats(ctypes.Structure):
    _fields_ = [
        ("frames_done", ctypes.c_uint64),
        ("pixels_done", ctypes.c_uint64),
        ("batches", ctypes.c_uint64),
        ("submits_rejected", ctypes.c_uint64),
        ("opens_rejected", ctypes.c_uint64),
        ("device_bytes", ctypes.c_uint64),
        ("arena_free_pixels", ctypes.c_uint64),
        ("streams_open", ctypes.c_int32),
        ("frames_queued", ctypes.c_int32),
        ("batches_inflight", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
    ]


_declared = False


def _lib():
    global _declared
    lib = _rm.load_library()
    if not _declared:
        vp = ctypes.c_void_p
        lib.rmusic_serve_create.argtypes = [ctypes.POINTER(_rm.rmusic_params), ctypes.c_int,
                                            ctypes.POINTER(rmusic_serve_config), ctypes.POINTER(vp)]
        lib.rmusic_serve_open_stream.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_int32)]
        lib.rmusic_serve_submit.argtypes = [vp, ctypes.c_int32, vp, vp, vp, ctypes.c_uint64]
        lib.rmusic_serve_poll.argtypes = [vp, ctypes.POINTER(rmusic_completion), ctypes.c_int32, ctypes.c_int32]
        lib.rmusic_serve_close_stream.argtypes = [vp, ctypes.c_int32]
        lib.rmusic_serve_get_stats.argtypes = [vp, ctypes.POINTER(rmusic_serve_stats)]
        lib.rmusic_serve_destroy.argtypes = [vp]
        lib.rmusic_serve_destroy.restype = None
        for f in ("rmusic_serve_create", "rmusic_serve_open_stream", "rmusic_serve_submit", "rmusic_serve_poll",
                  "rmusic_serve_close_stream", "rmusic_serve_get_stats"):
            getattr(lib, f).restype = ctypes.c_int
        _declared = True
    return lib


def _check(rc: int, where: str) -> int:
    if rc < 0 and rc != _rm.RMUSIC_EAGAIN:
        raise _rm.RmusicError(rc, where)
    return rc


def rmusic_serve_create(params: _rm.rmusic_params, device: int, cfg: rmusic_serve_config):
    srv = ctypes.c_void_p()
    _check(_lib().rmusic_serve_create(ctypes.byref(params), int(device), ctypes.byref(cfg), ctypes.byref(srv)),
           "rmusic_serve_create")
    return srv


def rmusic_serve_open_stream(srv, height: int, width: int, dtype: int) -> int:
    sid = ctypes.c_int32()
    _check(_lib().rmusic_serve_open_stream(srv, height, width, dtype, ctypes.byref(sid)), "rmusic_serve_open_stream")
    return sid.value


def rmusic_serve_submit(srv, stream_id: int, h_frame: int, h_out: int, h_status: int | None, tag: int) -> int:
    """Returns RMUSIC_OK or RMUSIC_EAGAIN (ring full); raises on other errors."""
    return _check(_lib().rmusic_serve_submit(srv, stream_id, h_frame, h_out, h_status or None, tag),
                  "rmusic_serve_submit")


def rmusic_serve_poll(srv, max_n: int, timeout_ms: int):
    arr = (rmusic_completion * max(max_n, 1))()
    n = _check(_lib().rmusic_serve_poll(srv, arr, max_n, timeout_ms), "rmusic_serve_poll")
    return [arr[i] for i in range(n)]


def rmusic_serve_close_stream(srv, stream_id: int) -> None:
    _check(_lib().rmusic_serve_close_stream(srv, stream_id), "rmusic_serve_close_stream")


def rmusic_serve_get_stats(srv) -> rmusic_serve_stats:
    st = rmusic_serve_stats()
    _check(_lib().rmusic_serve_get_stats(srv, ctypes.byref(st)), "rmusic_serve_get_stats")
    return st


def rmusic_serve_destroy(srv) -> None:
    if srv:
        _lib().rmusic_serve_destroy(srv)


def make_config(max_streams=16, ring_depth=4, max_batch_frames=32, inflight_batches=2,
                max_batch_pixels=16 << 20, hbm_budget_bytes=4 << 30) -> rmusic_serve_config:
    return rmusic_serve_config(max_streams, ring_depth, max_batch_frames, inflight_batches, max_batch_pixels,
                               hbm_budget_bytes)


class Server:
    """Owns one rmusic server. Host buffers passed to submit must stay alive until polled."""

    def __init__(self, device: int = 0, cfg: rmusic_serve_config | None = None, **params):
        params.setdefault("precision", "batched")
        self.params = _rm.make_params(**params)
        self.cfg = cfg or make_config()
        self.srv = rmusic_serve_create(self.params, device, self.cfg)

    def open_stream(self, height: int, width: int, dtype: int = _rm.RMUSIC_DTYPE_F32) -> int:
        return rmusic_serve_open_stream(self.srv, height, width, dtype)

    def submit(self, stream_id: int, h_frame: int, h_out: int, h_status: int | None = None, tag: int = 0) -> int:
        return rmusic_serve_submit(self.srv, stream_id, h_frame, h_out, h_status, tag)

    def poll(self, max_n: int = 256, timeout_ms: int = 0):
        return rmusic_serve_poll(self.srv, max_n, timeout_ms)

    def close_stream(self, stream_id: int) -> None:
        rmusic_serve_close_stream(self.srv, stream_id)

    def stats(self) -> rmusic_serve_stats:
        return rmusic_serve_get_stats(self.srv)

    def close(self) -> None:
        if getattr(self, "srv", None):
            rmusic_serve_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
