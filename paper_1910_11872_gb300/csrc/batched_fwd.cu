// batched_fwd.cu -- dispatch of the forward-estimate FP32-batched solver (batched_fwd_kernel.cuh): the
// covariance orders it supports, its register-cap variants, grid sizes and launches.
#include "batched_fwd_kernel.cuh"
#include "batched_fwd_variants.h"

namespace rmusic {

bool batched_fwd_supports(int L) { return L >= 2 && L <= kMaxL; }

int batched_fwd_num_variants(int) { return 2; }

// the variant with the smaller register cap where shared memory holds both, else the larger one
int batched_fwd_default_variant(int L) { return L <= 8 ? 1 : 0; }

int batched_fwd_variant_ctas(int L, int v) { return fwd_variant_ctas(L, v); }

static int occupancy_fwd(int L, int v) {
    switch (L) {
        case 2: return occupancy_fwd_l2(v);
        case 3: return occupancy_fwd_l3(v);
        case 4: return occupancy_fwd_l4(v);
        case 5: return occupancy_fwd_l5(v);
        case 6: return occupancy_fwd_l6(v);
        case 7: return occupancy_fwd_l7(v);
        case 8: return occupancy_fwd_l8(v);
        case 9: return occupancy_fwd_l9(v);
        case 10: return occupancy_fwd_l10(v);
        case 11: return occupancy_fwd_l11(v);
        case 12: return occupancy_fwd_l12(v);
        default: return 1;
    }
}

int batched_fwd_grid(int L, int v, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * occupancy_fwd(L, v);
}

cudaError_t launch_batched_fwd(int L, int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                               unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                               uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t s) {
#define RMUSIC_FWD_CASE(LL) \
    case LL: return launch_fwd_l##LL(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
    switch (L) {
        RMUSIC_FWD_CASE(2)
        RMUSIC_FWD_CASE(3)
        RMUSIC_FWD_CASE(4)
        RMUSIC_FWD_CASE(5)
        RMUSIC_FWD_CASE(6)
        RMUSIC_FWD_CASE(7)
        RMUSIC_FWD_CASE(8)
        RMUSIC_FWD_CASE(9)
        RMUSIC_FWD_CASE(10)
        RMUSIC_FWD_CASE(11)
        RMUSIC_FWD_CASE(12)
        default: return cudaErrorInvalidValue;
    }
#undef RMUSIC_FWD_CASE
}

}  // namespace rmusic
