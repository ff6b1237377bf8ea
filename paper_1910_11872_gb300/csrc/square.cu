// square.cu -- dispatch of the square-block FP32 solver (the paper's geometry): supported
// half-widths, register-cap variants, grid sizes and launches. The kernel is in square_kernel.cuh.
#include "rmusic_launch.h"
#include "square_variants.h"

namespace rmusic {

bool square_supports(int Lp) { return Lp >= 1 && Lp <= kMaxSquareLp; }

int square_num_variants(int) { return kSquareVariants; }

int square_default_variant(int) { return kSquareDefaultVariant; }

int square_variant_ctas(int Lp, int v) { return square_ctas(Lp, v); }

static int occupancy(int Lp, int v) {
    switch (Lp) {
        case 1: return occupancy_square_l1(v);
        case 2: return occupancy_square_l2(v);
        case 3: return occupancy_square_l3(v);
        case 4: return occupancy_square_l4(v);
        case 5: return occupancy_square_l5(v);
        case 6: return occupancy_square_l6(v);
        case 7: return occupancy_square_l7(v);
        case 8: return occupancy_square_l8(v);
        default: return 1;
    }
}

int square_grid(int Lp, int v, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * occupancy(Lp, v);
}

cudaError_t launch_square(int Lp, int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                          unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                          uint8_t* d_status, SquareArgs a, int grid, cudaStream_t stream) {
#define RM_SQ(LP) \
    case LP: return launch_square_l##LP(v, d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, stream);
    switch (Lp) {
        RM_SQ(1)
        RM_SQ(2)
        RM_SQ(3)
        RM_SQ(4)
        RM_SQ(5)
        RM_SQ(6)
        RM_SQ(7)
        RM_SQ(8)
        default: return cudaErrorInvalidValue;
    }
#undef RM_SQ
}

}  // namespace rmusic
