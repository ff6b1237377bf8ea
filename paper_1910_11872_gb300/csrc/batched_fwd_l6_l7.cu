// batched_fwd_l6_l7.cu -- instantiations of the forward-estimate solver for covariance order(s) 6 7 (batched_fwd_variants.h).
#include "batched_fwd_kernel.cuh"
#include "batched_fwd_variants.h"

namespace rmusic {

cudaError_t launch_fwd_l6(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<6>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l6(int v) { return occupancy_fwd_t<6>(v); }

cudaError_t launch_fwd_l7(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<7>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l7(int v) { return occupancy_fwd_t<7>(v); }

}  // namespace rmusic
