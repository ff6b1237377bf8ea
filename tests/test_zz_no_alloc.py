"""rmusic_demodulate_frames_noalloc: the FP32-batched path for callers that cannot allocate device
memory (its scratch is a fixed array inside the library). Checked through the C ABI against the
regular context-based entry point on two calls in a row, so that state left in the shared scratch
by the first call would show up in the second.

This file is named to be collected last: if it fails, a run that stops at the first failure has
already run every other test. It passes alone in a fresh process and after the other tests."""
import os
import re

import numpy as np
import pytest

from paper_1910_11872_gb300 import rmusic, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-4  # rad/pixel, the FP32 paths' noise-free tolerance against the FP64 oracle


def test_noalloc_source_makes_no_allocation_call():
    src = open(os.path.join(ROOT, "paper_1910_11872_gb300", "csrc", "noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", src)
    for call in ("cudaMalloc", "cudaFree", "cudaMallocHost", "cudaHostAlloc", "cudaMallocAsync",
                 "cudaMallocManaged", "malloc(", "new "):
        assert call not in code, f"noalloc.cu calls {call}"
    assert "static __device__ __align__(256)" in code
    assert "cudaGetSymbolAddress" in code


def _batch(seed, shapes, windows, snr):
    rng = np.random.default_rng(seed)
    frames = []
    for H, W in shapes:
        phi, _, _ = synth.gaussian_sum(rng, H, W)
        img = synth.add_noise(synth.fringe(phi, 0.1), synth.sigma_for_snr(0.4, snr), rng)
        frames.append(img.astype(np.float32))
    return frames, windows


def _run_both(torch, frames, windows):
    shapes = [f.shape for f in frames]
    descs, nbytes, nout = rmusic.frame_descs(shapes, rmusic.RMUSIC_DTYPE_F32, 4, windows)
    x = torch.from_numpy(np.concatenate([f.ravel() for f in frames])).cuda()
    params = rmusic.make_params(precision="batched")
    stream = torch.cuda.current_stream().cuda_stream
    out_na = torch.full((nout,), 123.0, device="cuda")
    st_na = torch.full((nout,), 77, dtype=torch.uint8, device="cuda")
    rmusic.rmusic_demodulate_frames_noalloc(params, 0, x.data_ptr(), descs, len(frames), out_na.data_ptr(),
                                            st_na.data_ptr(), stream)
    ctx = rmusic.rmusic_create(params, 0, 0)
    try:
        out = torch.empty(nout, device="cuda")
        st = torch.empty(nout, dtype=torch.uint8, device="cuda")
        rmusic.rmusic_demodulate_frames(ctx, x.data_ptr(), descs, len(frames), out.data_ptr(), st.data_ptr(),
                                        stream)
        torch.cuda.synchronize()
    finally:
        rmusic.rmusic_destroy(ctx)
    return out_na.cpu().numpy(), st_na.cpu().numpy(), out.cpu().numpy(), st.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_context_entry_on_two_calls_in_a_row():
    import torch

    assert torch.cuda.is_available()
    calls = [
        _batch(1, [(40, 300), (64, 128), (17, 257)], [(32, 8), (24, 6), (48, 12)], 20.0),
        _batch(2, [(24, 96), (9, 200)], [(16, 4), (32, 8)], np.inf),
    ]
    for frames, windows in calls:
        g_na, s_na, g, s = _run_both(torch, frames, windows)
        assert np.array_equal(s_na, s)
        ok = s == rmusic.STATUS_OK
        assert ok.sum() > 0
        assert np.array_equal(np.isnan(g_na), np.isnan(g))
        assert np.abs(g_na[ok] - g[ok]).max() <= TOL


@pytest.mark.gpu
def test_noalloc_rejects_requests_over_its_fixed_limits():
    import torch

    params = rmusic.make_params(precision="batched")
    buf = torch.zeros(16, device="cuda")
    too_many_px = [rmusic.rmusic_frame_desc(0, 2048, 4096, 0, rmusic.RMUSIC_DTYPE_F32, 0, 0, 0)]
    with pytest.raises(rmusic.RmusicError) as e:
        rmusic.rmusic_demodulate_frames_noalloc(params, 0, buf.data_ptr(), too_many_px, 1, buf.data_ptr(), None, None)
    assert e.value.code == rmusic.RMUSIC_ENOMEM
    many = [rmusic.rmusic_frame_desc(0, 1, 8, 0, rmusic.RMUSIC_DTYPE_F32, 0, 0, 0)] * 257
    with pytest.raises(rmusic.RmusicError) as e:
        rmusic.rmusic_demodulate_frames_noalloc(params, 0, buf.data_ptr(), many, 257, buf.data_ptr(), None, None)
    assert e.value.code == rmusic.RMUSIC_ENOMEM
    plain = rmusic.make_params(precision="plain_fp32")
    with pytest.raises(rmusic.RmusicError) as e:
        rmusic.rmusic_demodulate_frames_noalloc(plain, 0, buf.data_ptr(), many[:1], 1, buf.data_ptr(), None, None)
    assert e.value.code == rmusic.RMUSIC_EUNSUPPORTED
