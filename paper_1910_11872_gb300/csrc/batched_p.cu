// batched_p.cu -- dispatch of the FP32-batched model-order solver (batched_p_kernel.cuh): the model
// orders and covariance orders it supports, grid sizes and launches.
#include "batched_p_kernel.cuh"
#include "batched_p_variants.h"

namespace rmusic {

bool batched_p_supports(int p, int L) { return (p == 2 || p == 3) && L > p && L <= kMaxL; }

int batched_p_ctas(int L) { return p_ctas(L); }

static int occupancy_p(int p, int L) {
#define RMUSIC_P_OCC(PM, LL) \
    if (p == PM && L == LL) return occupancy_p##PM##_l##LL();
    RMUSIC_P_OCC(2, 3)
    RMUSIC_P_OCC(2, 4)
    RMUSIC_P_OCC(2, 5)
    RMUSIC_P_OCC(2, 6)
    RMUSIC_P_OCC(2, 7)
    RMUSIC_P_OCC(2, 8)
    RMUSIC_P_OCC(2, 9)
    RMUSIC_P_OCC(2, 10)
    RMUSIC_P_OCC(2, 11)
    RMUSIC_P_OCC(2, 12)
    RMUSIC_P_OCC(3, 4)
    RMUSIC_P_OCC(3, 5)
    RMUSIC_P_OCC(3, 6)
    RMUSIC_P_OCC(3, 7)
    RMUSIC_P_OCC(3, 8)
    RMUSIC_P_OCC(3, 9)
    RMUSIC_P_OCC(3, 10)
    RMUSIC_P_OCC(3, 11)
    RMUSIC_P_OCC(3, 12)
#undef RMUSIC_P_OCC
    return 1;
}

int batched_p_grid(int p, int L, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * occupancy_p(p, L);
}

cudaError_t launch_batched_p(int p, int L, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out, uint8_t* d_status,
                             BatchedArgs a, int grid, cudaStream_t s) {
#define RMUSIC_P_CASE(PM, LL)   \
    if (p == PM && L == LL) \
        return launch_p##PM##_l##LL(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
    RMUSIC_P_CASE(2, 3)
    RMUSIC_P_CASE(2, 4)
    RMUSIC_P_CASE(2, 5)
    RMUSIC_P_CASE(2, 6)
    RMUSIC_P_CASE(2, 7)
    RMUSIC_P_CASE(2, 8)
    RMUSIC_P_CASE(2, 9)
    RMUSIC_P_CASE(2, 10)
    RMUSIC_P_CASE(2, 11)
    RMUSIC_P_CASE(2, 12)
    RMUSIC_P_CASE(3, 4)
    RMUSIC_P_CASE(3, 5)
    RMUSIC_P_CASE(3, 6)
    RMUSIC_P_CASE(3, 7)
    RMUSIC_P_CASE(3, 8)
    RMUSIC_P_CASE(3, 9)
    RMUSIC_P_CASE(3, 10)
    RMUSIC_P_CASE(3, 11)
    RMUSIC_P_CASE(3, 12)
#undef RMUSIC_P_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rmusic
