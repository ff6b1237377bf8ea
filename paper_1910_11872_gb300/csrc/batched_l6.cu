// batched_l6.cu -- instantiations of the FP32-batched solver for covariance order(s) 6, all variants (see batched_variants.h).
#include "batched_kernel.cuh"
#include "batched_variants.h"

namespace rmusic {

cudaError_t launch_solver_l6(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                             uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    return launch_solver_t<6>(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid,
                              stream);
}

int occupancy_solver_l6(int v) { return occupancy_solver_t<6>(v); }

}  // namespace rmusic
