// batched_variants.h -- variants of the FP32-batched solver per covariance order: register caps
// (how many 128-thread CTAs stay resident per SM, the __launch_bounds__ minimum) and, for L <= 8,
// the warp-per-matrix schedule of the eigenvalue sweeps; the autotuner in capi.cu times them and
// keeps the fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

// Variants 0 .. 2 of every L differ only in their register cap (identical arithmetic); variant 3
// (L <= 8) runs the eigenvalue sweeps with the warp-per-matrix schedule at variant 1's cap.
constexpr int kSolverVariants = 3;
constexpr int kSolverWarpVariant = 3;
constexpr int kSolverMidVariant = 1;

// The variant used without tuning: the measured fastest on a GB300 for L = 8 (4 CTAs/SM: the
// certified solver with its fallbacks out of line runs best at 128 registers), the middle cap
// otherwise.
__host__ __device__ constexpr int solver_default_variant(int L) { return L == 8 ? 0 : kSolverMidVariant; }

__host__ __device__ constexpr int solver_num_variants(int L) { return L <= 8 ? 4 : 3; }
__host__ __device__ constexpr bool solver_variant_warp(int v) { return v == kSolverWarpVariant; }

// Resident CTAs per SM of variant v for covariance order L.
__host__ __device__ constexpr int solver_variant_ctas(int L, int v) {
    return v == kSolverWarpVariant ? solver_variant_ctas(L, kSolverMidVariant)
         : L == 2 ? (v == 0 ? 8 : v == 1 ? 12 : 16)
         : L == 4 ? (v == 0 ? 6 : v == 1 ? 8 : 12)
         : L == 6 ? (v == 0 ? 4 : v == 1 ? 6 : 8)
         : L == 8 ? (v == 0 ? 4 : v == 1 ? 6 : 8)
         : L == 10 ? (v == 0 ? 2 : v == 1 ? 3 : 4)
         : (v == 0 ? 1 : v == 1 ? 2 : 3);
}

#define RMUSIC_DECLARE_SOLVER(L)                                                                            \
    cudaError_t launch_solver_l##L(int v, const FrameDev* d_frames, int nframes, int64_t total_items,       \
                                   unsigned long long* d_counter, const float2* d_gamma, float* d_out,      \
                                   uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream);        \
    int occupancy_solver_l##L(int v);
RMUSIC_DECLARE_SOLVER(2)
RMUSIC_DECLARE_SOLVER(4)
RMUSIC_DECLARE_SOLVER(6)
RMUSIC_DECLARE_SOLVER(8)
RMUSIC_DECLARE_SOLVER(10)
RMUSIC_DECLARE_SOLVER(12)
#undef RMUSIC_DECLARE_SOLVER

}  // namespace rmusic
