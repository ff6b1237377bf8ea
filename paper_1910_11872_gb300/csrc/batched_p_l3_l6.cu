// batched_p_l3_l6.cu -- instantiations of the model-order solver (batched_p_kernel.cuh) for covariance orders 3 .. 6.
#include "batched_p_kernel.cuh"
#include "batched_p_variants.h"

namespace rmusic {

cudaError_t launch_p2_l3(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<3, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l3() { return occupancy_p_t<3, 2>(); }

cudaError_t launch_p2_l4(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<4, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l4() { return occupancy_p_t<4, 2>(); }

cudaError_t launch_p3_l4(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<4, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l4() { return occupancy_p_t<4, 3>(); }

cudaError_t launch_p2_l5(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<5, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l5() { return occupancy_p_t<5, 2>(); }

cudaError_t launch_p3_l5(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<5, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l5() { return occupancy_p_t<5, 3>(); }

cudaError_t launch_p2_l6(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<6, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p2_l6() { return occupancy_p_t<6, 2>(); }

cudaError_t launch_p3_l6(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                          const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                          cudaStream_t s) {
    return launch_p_t<6, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
}
int occupancy_p3_l6() { return occupancy_p_t<6, 3>(); }

}  // namespace rmusic
