// batched_p_l10_l12.cu -- instantiations of the model-order solver (batched_p_kernel.cuh) for covariance orders 10 .. 12.
#include "batched_p_kernel.cuh"
#include "batched_p_variants.h"

namespace rmusic {

cudaError_t launch_p2_l10(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<10, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l10() { return occupancy_p_t<10, 2>(); }

cudaError_t launch_p3_l10(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<10, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l10() { return occupancy_p_t<10, 3>(); }

cudaError_t launch_p2_l11(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<11, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l11() { return occupancy_p_t<11, 2>(); }

cudaError_t launch_p3_l11(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<11, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l11() { return occupancy_p_t<11, 3>(); }

cudaError_t launch_p2_l12(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<12, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l12() { return occupancy_p_t<12, 2>(); }

cudaError_t launch_p3_l12(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<12, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l12() { return occupancy_p_t<12, 3>(); }

}  // namespace rmusic
