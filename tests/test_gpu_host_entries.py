"""Host-buffer entries beyond the row-geometry cases of test_gpu_parity: the asynchronous entry in
the paper's square geometry with phase assembly (maps staged on the device and copied back), after
a workspace reservation (no allocation while calls are in flight), and its argument errors."""
import numpy as np
import pytest

from paper_1910_11872_gb300 import rmusic, synth

pytestmark = pytest.mark.gpu


def _torch():
    return pytest.importorskip("torch")


def test_async_square_with_phase_assembly_equals_sync():
    torch = _torch()
    frames = [synth.complex_fringe_frame(5.0, H=72, W=96, hi=6.0, stream=i).image for i in range(2)]
    flat = np.concatenate([f.reshape(-1) for f in frames])
    descs, nbytes, nout = rmusic.frame_descs([f.shape for f in frames], rmusic.RMUSIC_DTYPE_C64, 8, maps=4)
    kw = dict(geometry="square", half_width=3, carrier_freq=0.0, unwrap=1)
    dem = rmusic.Demodulator(**kw)
    try:
        ref = np.empty(nout, np.float32)
        ref_st = np.empty(nout, np.uint8)
        rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, 2, ref.ctypes.data,
                                             ref_st.ctypes.data, None)
    finally:
        dem.close()
    hin = torch.from_numpy(flat.view(np.float32)).pin_memory()
    hout = torch.full((nout,), 7.0).pin_memory()
    hst = torch.full((nout,), 9, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    dem = rmusic.Demodulator(use_graph=1, **kw)
    try:
        for _ in range(2):  # the second call replays the captured graph
            rmusic.rmusic_demodulate_frames_host_async(dem.ctx, hin.data_ptr(), nbytes, descs, 2, hout.data_ptr(),
                                                       hst.data_ptr(), s.cuda_stream)
            s.synchronize()
            assert np.array_equal(hout.numpy(), ref, equal_nan=True)
            for d in list(descs)[:2]:  # a frame's status map: the first H*W entries of its block
                o, n = d.out_offset, d.height * d.width
                assert np.array_equal(hst.numpy()[o:o + n], ref_st[o:o + n])
    finally:
        dem.close()


def test_async_after_reserve_allocates_nothing():
    torch = _torch()
    shapes = [(48, 256), (32, 512)]
    steps = [[synth.peaks_frame(snr, 0.1, H=h, W=w, stream=k).image for h, w in shapes]
             for k, snr in enumerate((25.0, 8.0, 40.0))]
    descs, nbytes, nout = rmusic.frame_descs(shapes, rmusic.RMUSIC_DTYPE_F32, 4)
    total = sum(h * w for h, w in shapes)
    dem = rmusic.Demodulator()
    try:
        ref = []
        for fr in steps:
            flat = np.concatenate([f.ravel() for f in fr]).astype(np.float32)
            out = np.empty(nout, np.float32)
            rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, 2, out.ctypes.data, None,
                                                 None)
            ref.append(out)
    finally:
        dem.close()
    dem = rmusic.Demodulator(use_graph=1)
    s = torch.cuda.Stream()
    try:
        # the analytic signal of both frames; the staged frames grow the workspace on the first call
        dem.reserve(total, 2)
        hins = [torch.from_numpy(np.concatenate([f.ravel() for f in fr]).astype(np.float32)).pin_memory()
                for fr in steps]
        houts = [torch.empty(nout).pin_memory() for _ in steps]
        rmusic.rmusic_demodulate_frames_host_async(dem.ctx, hins[0].data_ptr(), nbytes, descs, 2,
                                                   houts[0].data_ptr(), None, s.cuda_stream)
        s.synchronize()
        held = dem.stats().workspace_bytes
        for k in range(1, len(steps)):  # queued back to back on one stream
            rmusic.rmusic_demodulate_frames_host_async(dem.ctx, hins[k].data_ptr(), nbytes, descs, 2,
                                                       houts[k].data_ptr(), None, s.cuda_stream)
        s.synchronize()
        assert dem.stats().workspace_bytes == held
        for k in range(len(steps)):
            assert np.array_equal(houts[k].numpy(), ref[k], equal_nan=True), k
    finally:
        dem.close()


def test_async_rejects_bad_arguments_and_stays_usable():
    torch = _torch()
    fr = synth.peaks_frame(20.0, 0.1, H=16, W=128).image
    flat = fr.ravel().astype(np.float32)
    descs, nbytes, nout = rmusic.frame_descs([fr.shape], rmusic.RMUSIC_DTYPE_F32, 4)
    out = np.empty(nout, np.float32)
    dem = rmusic.Demodulator()
    s = torch.cuda.Stream()
    try:
        # the frame runs past the input buffer
        with pytest.raises(rmusic.RmusicError) as e:
            rmusic.rmusic_demodulate_frames_host_async(dem.ctx, flat.ctypes.data, nbytes - 4, descs, 1,
                                                       out.ctypes.data, None, s.cuda_stream)
        assert e.value.code == rmusic.RMUSIC_EINVAL
        with pytest.raises(rmusic.RmusicError) as e:
            rmusic.rmusic_demodulate_frames_host_async(dem.ctx, 0, nbytes, descs, 1, out.ctypes.data, None,
                                                       s.cuda_stream)
        assert e.value.code == rmusic.RMUSIC_EINVAL
        rmusic.rmusic_demodulate_frames_host_async(dem.ctx, flat.ctypes.data, nbytes, descs, 1, out.ctypes.data,
                                                   None, s.cuda_stream)
        s.synchronize()
        ref = np.empty(nout, np.float32)
        rmusic.rmusic_demodulate_frames_host(dem.ctx, flat.ctypes.data, nbytes, descs, 1, ref.ctypes.data, None,
                                             None)
        assert np.array_equal(out, ref, equal_nan=True)
    finally:
        dem.close()
