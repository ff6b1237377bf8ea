// batched_fwd_variants.h -- the forward-estimate solver's instantiations per covariance order (two
// register-cap variants each, batched_fwd_kernel.cuh), compiled in batched_fwd_l*.cu and dispatched
// by batched_fwd.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

#define RMUSIC_DECLARE_FWD(L)                                                                             \
    cudaError_t launch_fwd_l##L(int v, const FrameDev* d_frames, int nframes, int64_t total_items,        \
                                unsigned long long* d_counter, const float2* d_gamma, float* d_out,       \
                                uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream);         \
    int occupancy_fwd_l##L(int v);
RMUSIC_DECLARE_FWD(2)
RMUSIC_DECLARE_FWD(3)
RMUSIC_DECLARE_FWD(4)
RMUSIC_DECLARE_FWD(5)
RMUSIC_DECLARE_FWD(6)
RMUSIC_DECLARE_FWD(7)
RMUSIC_DECLARE_FWD(8)
RMUSIC_DECLARE_FWD(9)
RMUSIC_DECLARE_FWD(10)
RMUSIC_DECLARE_FWD(11)
RMUSIC_DECLARE_FWD(12)
#undef RMUSIC_DECLARE_FWD

}  // namespace rmusic
