"""rmusic_demodulate_frames_noalloc: the FP32-batched path for callers that cannot allocate device
memory (its scratch is a fixed array inside the library). Checked through the C ABI against the
regular context-based entry point on two calls in a row, so that state left in the shared scratch
by the first call would show up in the second, and against the FP64 oracle.

This file is named to be collected last: if it fails, a run that stops at the first failure has
already run every other test. It passes alone in a fresh process and after the other tests."""
import os
import re

import numpy as np
import pytest

from paper_1910_11872_gb300 import rmusic, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1910_11872_gb300", "csrc")
TOL = 1e-4  # rad/pixel, the FP32 paths' tolerance against the FP64 oracle
ALLOC_CALLS = ("cudaMalloc", "cudaFree", "cudaMallocHost", "cudaHostAlloc", "cudaMallocAsync", "cudaMallocManaged",
               "cudaMallocPitch", "cudaMalloc3D", "cudaMallocArray", "cuMemAlloc", "cuMemCreate", "malloc(",
               "calloc(", "realloc(", "new ", "std::vector", "std::string")


def _code(path):
    return re.sub(r"//[^\n]*", "", open(path).read())


# The solver variant the entry point runs for each covariance order: the library's untuned default
# (batched_variants.h: 4 CTAs per SM for L = 8, the middle register cap otherwise).
def _default_variant(L):
    return 0 if L == 8 else 1


def test_noalloc_source_makes_no_allocation_call():
    """Neither the entry point nor any code it reaches allocates: noalloc.cu itself, the band-pass and
    solver translation units and headers whose launchers it calls (init_analytic, band_assign,
    launch_analytic, launch_batched, batched_grid), and the shared validation in capi.cu
    (params_check, describe_frame)."""
    code = _code(os.path.join(CSRC, "noalloc.cu"))
    assert "static __device__ __align__(256)" in code
    assert "cudaGetSymbolAddress" in code
    reached = ["noalloc.cu", "analytic.cu", "batched.cu", "batched_kernel.cuh", "roots_device.cuh", "rmusic_device.cuh",
               "rmusic_launch.h", "rmusic_validate.h", "batched_variants.h"]
    reached += [f for f in os.listdir(CSRC) if f.startswith("batched_l") and f.endswith(".cu")]
    for f in reached:
        c = _code(os.path.join(CSRC, f))
        for call in ALLOC_CALLS:
            assert call not in c, f"{f} calls {call}"
    capi = _code(os.path.join(CSRC, "capi.cu"))
    start = capi.index("namespace rmusic {")
    shared = capi[start: capi.index("namespace {", start)]
    assert "int params_check(" in shared and "int describe_frame(" in shared
    for call in ALLOC_CALLS:
        assert call not in shared, f"capi.cu's shared validation calls {call}"


def _batch(seed, shapes, windows, snr):
    rng = np.random.default_rng(seed)
    frames = []
    for H, W in shapes:
        phi, _, _ = synth.gaussian_sum(rng, H, W)
        img = synth.add_noise(synth.fringe(phi, 0.1), synth.sigma_for_snr(0.4, snr), rng)
        frames.append(img.astype(np.float32))
    return frames, windows


def _inputs(torch, frames, windows):
    shapes = [f.shape for f in frames]
    descs, nbytes, nout = rmusic.frame_descs(shapes, rmusic.RMUSIC_DTYPE_F32, 4, windows)
    x = torch.from_numpy(np.concatenate([f.ravel() for f in frames])).cuda()
    return descs, nout, x


def _noalloc(torch, frames, descs, x, out, st):
    params = rmusic.make_params(precision="batched")
    rmusic.rmusic_demodulate_frames_noalloc(params, 0, x.data_ptr(), descs, len(frames), out.data_ptr(),
                                            st.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _context(torch, frames, windows, descs, x):
    """The regular entry point with every covariance order pinned to the default variant."""
    params = rmusic.make_params(precision="batched")
    ctx = rmusic.rmusic_create(params, 0, 0)
    try:
        for L in {w[1] for w in windows}:
            rmusic.rmusic_set_solver_variant(ctx, L, _default_variant(L))
        nout = sum(f.size for f in frames)
        out = torch.empty(nout, device="cuda")
        st = torch.empty(nout, dtype=torch.uint8, device="cuda")
        rmusic.rmusic_demodulate_frames(ctx, x.data_ptr(), descs, len(frames), out.data_ptr(), st.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        rmusic.rmusic_destroy(ctx)
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_context_entry_on_two_calls_in_a_row():
    """Two different calls in a row: each one's maps and statuses equal, bit for bit, those of a
    context pinned to the same solver variant; the noise-free call's maps also agree with the FP64
    oracle within 1e-4 rad/pixel with identical status maps."""
    import torch

    import oracle as O

    assert torch.cuda.is_available()
    calls = [
        _batch(1, [(40, 300), (64, 128), (17, 257)], [(32, 8), (24, 6), (48, 12)], 20.0),
        _batch(2, [(24, 96), (9, 200)], [(16, 4), (32, 8)], np.inf),
    ]
    for k, (frames, windows) in enumerate(calls):
        descs, nout, x = _inputs(torch, frames, windows)
        out_na = torch.full((nout,), 123.0, device="cuda")
        st_na = torch.full((nout,), 77, dtype=torch.uint8, device="cuda")
        _noalloc(torch, frames, descs, x, out_na, st_na)
        torch.cuda.synchronize()
        g_na, s_na = out_na.cpu().numpy(), st_na.cpu().numpy()
        g, s = _context(torch, frames, windows, descs, x)
        assert np.array_equal(s_na, s), k
        assert (s == rmusic.STATUS_OK).sum() > 0
        assert np.array_equal(g_na, g, equal_nan=True), k
        if k == 1:  # noise-free: against the oracle
            o_off = 0
            for f, (N, L) in zip(frames, windows):
                o, os_, _ = O.demodulate(f, O.make_params(N, L, 1, 0, 0, 0.1))
                gg = g_na[o_off:o_off + f.size].reshape(f.shape)
                ss = s_na[o_off:o_off + f.size].reshape(f.shape)
                assert np.array_equal(ss, os_)
                v = os_ == 0
                assert np.abs(gg[v].astype(np.float64) - o[v]).max() <= TOL
                o_off += f.size


@pytest.mark.gpu
def test_noalloc_repeated_calls_leave_device_memory_unchanged():
    """After one warm-up call (which loads the code and looks the scratch address up), further
    calls change neither the device's free memory nor the maps."""
    import torch

    frames, windows = _batch(3, [(48, 256), (20, 512)], [(32, 8), (24, 6)], 15.0)
    descs, nout, x = _inputs(torch, frames, windows)
    out = torch.empty(nout, device="cuda")
    st = torch.empty(nout, dtype=torch.uint8, device="cuda")
    _noalloc(torch, frames, descs, x, out, st)
    torch.cuda.synchronize()
    first = out.cpu().numpy()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc(torch, frames, descs, x, out, st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert np.array_equal(out.cpu().numpy(), first, equal_nan=True)


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
    # the validation every entry point shares: the codes rmusic_create returns
    for bad, code in ((dict(unwrap=1), rmusic.RMUSIC_EINVAL), (dict(exhaustive=2), rmusic.RMUSIC_EINVAL),
                      (dict(model_order=0), rmusic.RMUSIC_EINVAL), (dict(model_order=2), rmusic.RMUSIC_EUNSUPPORTED)):
        p = rmusic.make_params(precision="batched", **bad)
        with pytest.raises(rmusic.RmusicError) as e:
            rmusic.rmusic_demodulate_frames_noalloc(p, 0, buf.data_ptr(), many[:1], 1, buf.data_ptr(), None, None)
        assert e.value.code == code, bad
        with pytest.raises(rmusic.RmusicError) as e:
            rmusic.rmusic_create(p, 0, 0)
        assert e.value.code == code, bad
