"""Serving loop on the GPU (include/rmusic_serve.h): frames from several streams, submitted while
others run, come back identical to single-frame calls of the regular entry point; stream admission
follows the HBM budget; a full ring applies back-pressure; batches form continuously."""
import argparse

import numpy as np
import pytest

from paper_1910_11872_gb300 import rmusic, serve, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    assert torch.cuda.is_available()
    return torch


def _single(frame, **params):
    torch = _torch()
    dem = rmusic.Demodulator(**params)
    try:
        x = torch.from_numpy(frame.view(np.int16) if frame.dtype == np.uint16 else frame).cuda()
        out, st, _ = dem.run(x)
        torch.cuda.synchronize()
        return out.cpu().numpy().reshape(frame.shape), st.cpu().numpy().reshape(frame.shape)
    finally:
        dem.close()


def test_mix_equals_alone():
    torch = _torch()
    rng = np.random.default_rng(9)
    specs = [((64, 256), np.float32), ((128, 160), np.float32), ((96, 300), np.uint16), ((33, 512), np.float32)]
    frames = {}
    for s, ((H, W), dt) in enumerate(specs):
        for k in range(3):
            phi, _, _ = synth.gaussian_sum(rng, H, W)
            img = synth.add_noise(synth.fringe(phi, 0.1), 0.02, rng)
            frames[(s, k)] = synth.quantize12(img) if dt == np.uint16 else img.astype(np.float32)
    cfg = serve.make_config(max_streams=8, ring_depth=4, max_batch_frames=5, inflight_batches=2,
                            max_batch_pixels=1 << 20, hbm_budget_bytes=256 << 20)
    srv = serve.Server(cfg=cfg)
    try:
        ids = [srv.open_stream(H, W, rmusic.RMUSIC_DTYPE_U16 if dt == np.uint16 else rmusic.RMUSIC_DTYPE_F32)
               for (H, W), dt in specs]
        keep, outs, sts = [], {}, {}
        tag = 0
        tags = {}
        for k in range(3):                       # interleave the streams
            for s in range(len(specs)):
                f = frames[(s, k)]
                h_in = torch.from_numpy(f.view(np.int16) if f.dtype == np.uint16 else f).pin_memory()
                o = torch.empty(f.size, dtype=torch.float32).pin_memory()
                st = torch.empty(f.size, dtype=torch.uint8).pin_memory()
                keep += [h_in, o, st]
                assert srv.submit(ids[s], h_in.data_ptr(), o.data_ptr(), st.data_ptr(), tag) == rmusic.RMUSIC_OK
                tags[tag] = (s, k)
                outs[(s, k)], sts[(s, k)] = o, st
                tag += 1
        done = []
        while len(done) < tag:
            done += srv.poll(64, 2000)
        assert all(c.status == rmusic.RMUSIC_OK for c in done)
        assert sorted(c.tag for c in done) == list(range(tag))
        assert all(c.t_submit <= c.t_launch <= c.t_done for c in done)
        for (s, k), f in frames.items():
            g_alone, s_alone = _single(f)
            g = outs[(s, k)].numpy().reshape(f.shape)
            st = sts[(s, k)].numpy().reshape(f.shape)
            assert np.array_equal(st, s_alone)
            assert np.array_equal(g, g_alone, equal_nan=True)
        stats = srv.stats()
        assert stats.frames_done == tag and stats.batches <= tag
    finally:
        srv.close()


def test_admission_and_backpressure():
    torch = _torch()
    # budget: two batch workspaces (8 B x 4 M pixels + 1 MiB each) and 5 M - 1024 pixel slots
    cfg = serve.make_config(max_streams=4, ring_depth=1, max_batch_frames=4, inflight_batches=2,
                            max_batch_pixels=4 << 20,
                            hbm_budget_bytes=(2 * (8 * (4 << 20) + (1 << 20))) + 9 * ((5 << 20) - 1024))
    srv = serve.Server(cfg=cfg)
    try:
        a = srv.open_stream(2048, 2048)             # 4 M slots: fits
        with pytest.raises(rmusic.RmusicError) as e:
            srv.open_stream(1024, 1024)             # 1 M more does not fit in ~5 M
        assert e.value.code == rmusic.RMUSIC_ENOMEM
        with pytest.raises(rmusic.RmusicError):
            srv.open_stream(4096, 2048)             # larger than max_batch_pixels
        fr = synth.peaks_frame(20, 0.1, H=2048, W=2048).image
        h_in = torch.from_numpy(fr).pin_memory()
        o1 = torch.empty(fr.size).pin_memory()
        o2 = torch.empty(fr.size).pin_memory()
        assert srv.submit(a, h_in.data_ptr(), o1.data_ptr(), None, 1) == rmusic.RMUSIC_OK
        # the ring holds one frame: a second submit while the first runs is pushed back
        assert srv.submit(a, h_in.data_ptr(), o2.data_ptr(), None, 2) == rmusic.RMUSIC_EAGAIN
        done = []
        while not done:
            done = srv.poll(4, 5000)
        assert srv.stats().submits_rejected == 1
        srv.close_stream(a)
        b = srv.open_stream(1024, 1024)             # the closed ring's space is free again
        assert b >= 0
        g_alone, _ = _single(fr)
        assert np.array_equal(o1.numpy().reshape(fr.shape), g_alone, equal_nan=True)
    finally:
        srv.close()


def test_continuous_batching_forms_multi_frame_batches():
    torch = _torch()
    cfg = serve.make_config(max_streams=8, ring_depth=8, max_batch_frames=16, inflight_batches=1,
                            max_batch_pixels=8 << 20, hbm_budget_bytes=1 << 30)
    srv = serve.Server(cfg=cfg)
    try:
        ids = [srv.open_stream(512, 512) for _ in range(6)]
        fr = synth.peaks_frame(15, 0.1, H=512, W=512).image
        h_in = torch.from_numpy(fr).pin_memory()
        outs = [torch.empty(fr.size).pin_memory() for _ in range(48)]
        n = 0
        for k in range(8):
            for s in ids:
                assert srv.submit(s, h_in.data_ptr(), outs[n].data_ptr(), None, n) == rmusic.RMUSIC_OK
                n += 1
        done = []
        while len(done) < n:
            done += srv.poll(64, 2000)
        # with one batch slot, frames that arrived during a batch were taken together afterwards
        assert max(c.batch_frames for c in done) > 1
        assert srv.stats().batches < n
        ref = outs[0].numpy()
        for o in outs[1:]:
            assert np.array_equal(o.numpy(), ref, equal_nan=True)
    finally:
        srv.close()


def test_serve_bench_short_run():
    from paper_1910_11872_gb300 import serve_bench

    args = argparse.Namespace(streams=4, rate=100.0, seconds=1.0, pool=1, ring_depth=4, max_batch_frames=8,
                              max_batch_mpx=16, inflight=2, budget_gb=2.0, device=0)
    r = serve_bench.run(args)
    assert r["frames_done"] > 0
    assert r["frames_done"] + r["frames_rejected"] == r["frames_offered"]
    assert 0 < r["latency_ms"]["p50"] <= r["latency_ms"]["p99"]
