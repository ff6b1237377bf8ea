// square_variants.h -- register-cap variants of the square-block solver per half-width Lp, and
// the instantiation boilerplate shared by square_l*.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

constexpr int kSquareVariants = 2;
constexpr int kSquareDefaultVariant = 0;

// Resident 128-thread CTAs per SM of variant v for half-width Lp (block side M = 2 Lp + 1).
__host__ __device__ constexpr int square_ctas(int Lp, int v) {
    return Lp == 1 ? (v == 0 ? 8 : 12)
         : Lp == 2 ? (v == 0 ? 6 : 8)
         : Lp == 3 ? (v == 0 ? 4 : 6)
         : Lp <= 5 ? (v == 0 ? 3 : 4)
         : (v == 0 ? 2 : 3);
}

#define RMUSIC_DECLARE_SQUARE(LP)                                                                           \
    cudaError_t launch_square_l##LP(int v, const FrameDev* d_frames, int nframes, int64_t total_items,      \
                                    unsigned long long* d_counter, const float2* d_gamma, float* d_out,     \
                                    uint8_t* d_status, SquareArgs a, int grid, cudaStream_t stream);        \
    int occupancy_square_l##LP(int v);
RMUSIC_DECLARE_SQUARE(1)
RMUSIC_DECLARE_SQUARE(2)
RMUSIC_DECLARE_SQUARE(3)
RMUSIC_DECLARE_SQUARE(4)
RMUSIC_DECLARE_SQUARE(5)
RMUSIC_DECLARE_SQUARE(6)
RMUSIC_DECLARE_SQUARE(7)
RMUSIC_DECLARE_SQUARE(8)
#undef RMUSIC_DECLARE_SQUARE

// Defines launch_square_l<LP> and occupancy_square_l<LP> for both variants (in square_l*.cu). The
// kernel's dynamic shared memory may exceed the 48 KB default: its limit is raised before every
// launch and occupancy query (a cheap host call).
#define RMUSIC_DEFINE_SQUARE(LP)                                                                              \
    static cudaError_t square_smem_attr_l##LP(int v) {                                                        \
        return v == 0 ? cudaFuncSetAttribute(square_kernel<LP, square_ctas(LP, 0)>,                           \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,                     \
                                             (int)square_smem_bytes(LP))                                      \
                      : cudaFuncSetAttribute(square_kernel<LP, square_ctas(LP, 1)>,                           \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,                     \
                                             (int)square_smem_bytes(LP));                                     \
    }                                                                                                         \
    cudaError_t launch_square_l##LP(int v, const FrameDev* d_frames, int nframes, int64_t total_items,        \
                                    unsigned long long* d_counter, const float2* d_gamma, float* d_out,       \
                                    uint8_t* d_status, SquareArgs a, int grid, cudaStream_t stream) {         \
        if (v != 0 && v != 1) return cudaErrorInvalidValue;                                                   \
        cudaError_t e = square_smem_attr_l##LP(v);                                                            \
        if (e != cudaSuccess) return e;                                                                       \
        if (v == 0)                                                                                           \
            square_kernel<LP, square_ctas(LP, 0)><<<grid, kSqThreads, square_smem_bytes(LP), stream>>>(       \
                d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a);                      \
        else                                                                                                  \
            square_kernel<LP, square_ctas(LP, 1)><<<grid, kSqThreads, square_smem_bytes(LP), stream>>>(       \
                d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a);                      \
        return cudaGetLastError();                                                                            \
    }                                                                                                         \
    int occupancy_square_l##LP(int v) {                                                                       \
        int nb = 0;                                                                                           \
        if (square_smem_attr_l##LP(v) != cudaSuccess) return 1;                                               \
        cudaError_t e = v == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                               \
                                     &nb, square_kernel<LP, square_ctas(LP, 0)>, kSqThreads,                  \
                                     square_smem_bytes(LP))                                                   \
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                               \
                                     &nb, square_kernel<LP, square_ctas(LP, 1)>, kSqThreads,                  \
                                     square_smem_bytes(LP));                                                  \
        return (e == cudaSuccess && nb > 0) ? nb : 1;                                                         \
    }

}  // namespace rmusic
