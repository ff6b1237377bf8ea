// batched_p_l7_l9.cu -- instantiations of the model-order solver (batched_p_kernel.cuh) for covariance orders 7 .. 9.
#include "batched_p_kernel.cuh"
#include "batched_p_variants.h"

namespace rmusic {

cudaError_t launch_p2_l7(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<7, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l7() { return occupancy_p_t<7, 2>(); }

cudaError_t launch_p3_l7(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<7, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l7() { return occupancy_p_t<7, 3>(); }

cudaError_t launch_p2_l8(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<8, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l8() { return occupancy_p_t<8, 2>(); }

cudaError_t launch_p3_l8(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<8, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l8() { return occupancy_p_t<8, 3>(); }

cudaError_t launch_p2_l9(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<9, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l9() { return occupancy_p_t<9, 2>(); }

cudaError_t launch_p3_l9(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<9, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l9() { return occupancy_p_t<9, 3>(); }

}  // namespace rmusic
