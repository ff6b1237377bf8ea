"""Failures injected on the host into the serving loop (no GPU fault, no hang): bad arguments are
rejected with error codes before any work is queued; a stream closed while its frames are queued or
on the GPU waits for them, and their completions stay available and correct; a stream that stalls
(opened, never fed) holds up no one; destroying the server with frames in flight finishes them; a
client that stops polling loses nothing until it polls again."""
import numpy as np
import pytest

from paper_1910_11872_gb300 import rmusic, serve, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    assert torch.cuda.is_available()
    return torch


def _alone(frame):
    torch = _torch()
    dem = rmusic.Demodulator()
    try:
        out, st, _ = dem.run(torch.from_numpy(frame).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy().reshape(frame.shape)
    finally:
        dem.close()


def _frames(n, H=64, W=256):
    return [synth.peaks_frame(20.0, 0.1, H=H, W=W, stream=k).image for k in range(n)]


def test_bad_arguments_are_rejected():
    torch = _torch()
    srv = serve.Server(cfg=serve.make_config(max_streams=2, ring_depth=2))
    try:
        with pytest.raises(rmusic.RmusicError) as e:
            srv.open_stream(0, 256)
        assert e.value.code in (rmusic.RMUSIC_EINVAL, rmusic.RMUSIC_ENOMEM)
        with pytest.raises(rmusic.RmusicError):
            srv.open_stream(64, 256, dtype=99)
        a = srv.open_stream(64, 256)
        fr = torch.from_numpy(_frames(1)[0]).pin_memory()
        out = torch.empty(fr.numel()).pin_memory()
        for bad in (-1, a + 7, 4096):
            with pytest.raises(rmusic.RmusicError) as e:
                srv.submit(bad, fr.data_ptr(), out.data_ptr(), None, 1)
            assert e.value.code == rmusic.RMUSIC_EINVAL
        srv.close_stream(a)
        with pytest.raises(rmusic.RmusicError) as e:   # a closed stream takes no more frames
            srv.submit(a, fr.data_ptr(), out.data_ptr(), None, 2)
        assert e.value.code == rmusic.RMUSIC_EINVAL
        with pytest.raises(rmusic.RmusicError):
            srv.close_stream(a)                         # nor a second close
        assert srv.stats().frames_done == 0
    finally:
        srv.close()


def test_close_with_frames_in_flight_and_a_stalled_stream():
    torch = _torch()
    frames = _frames(4)
    srv = serve.Server(cfg=serve.make_config(max_streams=4, ring_depth=4, inflight_batches=2))
    try:
        stalled = srv.open_stream(128, 512)            # opened, never fed
        a = srv.open_stream(64, 256)
        ins = [torch.from_numpy(f).pin_memory() for f in frames]
        outs = [torch.full((f.size,), -5.0).pin_memory() for f in frames]
        for k, (i, o) in enumerate(zip(ins, outs)):
            assert srv.submit(a, i.data_ptr(), o.data_ptr(), None, 100 + k) == rmusic.RMUSIC_OK
        srv.close_stream(a)                             # waits for the four frames
        done = srv.poll(16, 0)                          # their completions are still there
        assert sorted(c.tag for c in done) == [100, 101, 102, 103]
        for f, o in zip(frames, outs):
            assert np.array_equal(o.numpy().reshape(f.shape), _alone(f), equal_nan=True)
        assert srv.stats().frames_done == 4
        srv.close_stream(stalled)
    finally:
        srv.close()


def test_destroy_with_frames_in_flight_and_late_polling():
    torch = _torch()
    frames = _frames(3, H=128, W=1024)
    ins = [torch.from_numpy(f).pin_memory() for f in frames]
    outs = [torch.full((f.size,), -5.0).pin_memory() for f in frames]
    srv = serve.Server(cfg=serve.make_config(max_streams=2, ring_depth=4))
    a = srv.open_stream(128, 1024)
    for k, (i, o) in enumerate(zip(ins, outs)):
        assert srv.submit(a, i.data_ptr(), o.data_ptr(), None, k) == rmusic.RMUSIC_OK
    srv.close()                                         # finishes the submitted frames, then frees
    for f, o in zip(frames, outs):
        assert np.array_equal(o.numpy().reshape(f.shape), _alone(f), equal_nan=True)
