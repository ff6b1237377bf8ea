// batched_fwd_l2_l5.cu -- instantiations of the forward-estimate solver for covariance order(s) 2 3 4 5 (batched_fwd_variants.h).
#include "batched_fwd_kernel.cuh"
#include "batched_fwd_variants.h"

namespace rmusic {

cudaError_t launch_fwd_l2(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<2>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l2(int v) { return occupancy_fwd_t<2>(v); }

cudaError_t launch_fwd_l3(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<3>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l3(int v) { return occupancy_fwd_t<3>(v); }

cudaError_t launch_fwd_l4(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<4>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l4(int v) { return occupancy_fwd_t<4>(v); }

cudaError_t launch_fwd_l5(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<5>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l5(int v) { return occupancy_fwd_t<5>(v); }

}  // namespace rmusic
