// batched_fwd_l11_l12.cu -- instantiations of the forward-estimate solver for covariance order(s) 11 12 (batched_fwd_variants.h).
#include "batched_fwd_kernel.cuh"
#include "batched_fwd_variants.h"

namespace rmusic {

cudaError_t launch_fwd_l11(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<11>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l11(int v) { return occupancy_fwd_t<11>(v); }

cudaError_t launch_fwd_l12(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_fwd_t<12>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                           stream);
}

int occupancy_fwd_l12(int v) { return occupancy_fwd_t<12>(v); }

}  // namespace rmusic
