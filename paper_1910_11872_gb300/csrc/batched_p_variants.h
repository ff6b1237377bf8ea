// batched_p_variants.h -- the model-order solver's instantiations (batched_p_kernel.cuh; p = 2 for
// L = 3 .. 12, p = 3 for L = 4 .. 12), compiled in batched_p_l*.cu and dispatched by batched_p.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

#define RMUSIC_DECLARE_P(PM, L)                                                                             \
    cudaError_t launch_p##PM##_l##L(const FrameDev* d_frames, int nframes, int64_t total_items,           \
                                    unsigned long long* d_counter, const float2* d_gamma, float* d_out,   \
                                    uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t s);          \
    int occupancy_p##PM##_l##L();
RMUSIC_DECLARE_P(2, 3)
RMUSIC_DECLARE_P(2, 4)
RMUSIC_DECLARE_P(2, 5)
RMUSIC_DECLARE_P(2, 6)
RMUSIC_DECLARE_P(2, 7)
RMUSIC_DECLARE_P(2, 8)
RMUSIC_DECLARE_P(2, 9)
RMUSIC_DECLARE_P(2, 10)
RMUSIC_DECLARE_P(2, 11)
RMUSIC_DECLARE_P(2, 12)
RMUSIC_DECLARE_P(3, 4)
RMUSIC_DECLARE_P(3, 5)
RMUSIC_DECLARE_P(3, 6)
RMUSIC_DECLARE_P(3, 7)
RMUSIC_DECLARE_P(3, 8)
RMUSIC_DECLARE_P(3, 9)
RMUSIC_DECLARE_P(3, 10)
RMUSIC_DECLARE_P(3, 11)
RMUSIC_DECLARE_P(3, 12)
#undef RMUSIC_DECLARE_P

}  // namespace rmusic
