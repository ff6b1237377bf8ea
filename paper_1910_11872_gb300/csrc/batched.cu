// batched.cu -- dispatch of the FP32-batched solver: which covariance orders it supports, its
// register-cap variants, grid sizes and launches. The kernel itself is in batched_kernel.cuh.
#include "batched_variants.h"
#include "rmusic_launch.h"

namespace rmusic {

bool batched_supports(int L) { return L == 2 || L == 4 || L == 6 || L == 8 || L == 10 || L == 12; }

int batched_num_variants(int L) { return solver_num_variants(L); }

int batched_default_variant(int L) { return solver_default_variant(L); }

int batched_variant_ctas(int L, int v) { return solver_variant_ctas(L, v); }

static int occupancy(int L, int v) {
    switch (L) {
        case 2: return occupancy_solver_l2(v);
        case 4: return occupancy_solver_l4(v);
        case 6: return occupancy_solver_l6(v);
        case 8: return occupancy_solver_l8(v);
        case 10: return occupancy_solver_l10(v);
        case 12: return occupancy_solver_l12(v);
        default: return 1;
    }
}

int batched_grid(int L, int v, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * occupancy(L, v);
}

cudaError_t init_batched(int) { return cudaSuccess; }

cudaError_t launch_batched(int L, int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                           unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                           uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    switch (L) {
        case 2: return launch_solver_l2(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 4: return launch_solver_l4(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 6: return launch_solver_l6(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 8: return launch_solver_l8(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 10: return launch_solver_l10(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        case 12: return launch_solver_l12(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rmusic
