// batched_l6.cu -- instantiations of the FP32-batched solver for covariance order(s) 6, all register-cap variants (see batched_variants.h).
#include "batched_kernel.cuh"
#include "batched_variants.h"

namespace rmusic {

template <int V>
static cudaError_t launch_l6_v(const FrameDev* d_frames, int nframes, int64_t total_items,
                                unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                                uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    batched_kernel<6, solver_variant_ctas(6, V)><<<grid, kBatThreads, 0, stream>>>(
        d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a);
    return cudaGetLastError();
}

template <int V>
static int occupancy_l6_v() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_kernel<6, solver_variant_ctas(6, V)>,
                                                      kBatThreads, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_solver_l6(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                               unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                               uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    switch (v) {
        case 0: return launch_l6_v<0>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 1: return launch_l6_v<1>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 2: return launch_l6_v<2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

int occupancy_solver_l6(int v) {
    switch (v) {
        case 0: return occupancy_l6_v<0>();
        case 1: return occupancy_l6_v<1>();
        case 2: return occupancy_l6_v<2>();
        default: return 1;
    }
}

}  // namespace rmusic
