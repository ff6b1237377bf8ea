"""Child process of tests/test_gpu_checked_build.py: runs a fixed set of workloads through the
ordinary or the checked build of the library and saves the maps, statuses and index-check counts.

    python tests/checked_build_child.py {plain|checked} OUT.npz
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1910_11872_gb300 import rmusic, synth  # noqa: E402


def main():
    mode, path = sys.argv[1], sys.argv[2]
    if mode == "checked":
        rmusic.use_checked_build()
    import torch

    lib = rmusic.load_library()
    assert lib.rmusic_checked_build() == (1 if mode == "checked" else 0)
    res, viol = {}, {}

    def record(name, dem, out, st):
        torch.cuda.synchronize()
        viol[name] = int(dem.stats().check_violations)
        res[name + "_out"] = out.cpu().numpy() if hasattr(out, "cpu") else out
        res[name + "_st"] = st.cpu().numpy() if hasattr(st, "cpu") else st

    # row windows: ragged and tiny frames, every covariance order, per-frame windows in one call
    shapes = [(8, 40), (16, 64), (33, 300), (20, 1024), (12, 512), (40, 256)]
    windows = [(24, 6), (32, 8), (48, 12), (16, 4), (64, 12), (12, 2)]
    frames = [synth.peaks_frame(15.0, 0.1, H=h, W=w, stream=i).image for i, (h, w) in enumerate(shapes)]
    for axis in (0, 1):
        dem = rmusic.Demodulator(deriv_axis=axis, carrier_axis=0)
        try:
            out, st, _ = dem.run([torch.from_numpy(f).cuda() for f in frames], windows=windows)
            record(f"row_axis{axis}", dem, out, st)
        finally:
            dem.close()
    # the exhaustive root finder and the Jacobi fallback on the same frames
    dem = rmusic.Demodulator(exhaustive=1)
    try:
        out, st, _ = dem.run([torch.from_numpy(f).cuda() for f in frames], windows=windows)
        record("row_exhaustive", dem, out, st)
    finally:
        dem.close()
    # the paper's square block, every half-width class
    cf = [synth.complex_fringe_frame(5.0, H=40, W=72, hi=6.0, stream=i).image for i in range(2)]
    nsq = 3 * sum(f.size for f in cf)  # three maps per frame; a frame's status fills its first map's span
    for lp in (1, 3, 5, 8):
        dem = rmusic.Demodulator(geometry="square", half_width=lp, carrier_freq=0.0)
        try:
            out = torch.zeros(nsq, device="cuda")
            st = torch.zeros(nsq, dtype=torch.uint8, device="cuda")
            dem.run([torch.from_numpy(f).cuda() for f in cf], out=out, status=st)
            record(f"square_lp{lp}", dem, out, st)
        finally:
            dem.close()
    # the asynchronous host entry on pinned buffers
    hs = [(24, 256), (16, 512)]
    hf = [synth.peaks_frame(10.0, 0.1, H=h, W=w, stream=7 + i).image for i, (h, w) in enumerate(hs)]
    descs, nbytes, nout = rmusic.frame_descs(hs, rmusic.RMUSIC_DTYPE_F32, 4)
    hin = torch.from_numpy(np.concatenate([f.ravel() for f in hf]).astype(np.float32)).pin_memory()
    hout = torch.empty(nout).pin_memory()
    hst = torch.empty(nout, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    dem = rmusic.Demodulator(use_graph=1)
    try:
        rmusic.rmusic_demodulate_frames_host_async(dem.ctx, hin.data_ptr(), nbytes, descs, 2, hout.data_ptr(),
                                                   hst.data_ptr(), s.cuda_stream)
        s.synchronize()
        record("host_async", dem, hout.numpy().copy(), hst.numpy().copy())
    finally:
        dem.close()
    np.savez(path, **res)
    print(json.dumps(viol))


if __name__ == "__main__":
    main()
