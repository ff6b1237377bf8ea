// rmusic_launch.h -- host-side launchers of the library's kernels (internal interface between
// the C ABI in capi.cu and the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"

namespace rmusic {

// Band-pass analytic signal of every carrier line (Sec. 2, Eq. 1). init_analytic must run once per
// device (it also uploads the twiddle table). band_assign picks a frame's band-pass schedule
// (F->band_r) and returns the CTAs it takes; frames' line_start values are the running sums of
// those counts, total_ctas their sum, schedules the kBand* bits of the schedules the frames take.
constexpr int kBandPerLine = 1, kBandWarpFft = 2;
cudaError_t init_analytic();
int64_t band_assign(FrameDev* F, bool fp64);
inline int band_schedule_bit(const FrameDev& F) { return F.band_r ? kBandWarpFft : kBandPerLine; }
// fp64 = true writes complex128 (plain FP64 path), otherwise complex64.
cudaError_t launch_analytic(const FrameDev* d_frames, int nframes, int64_t total_ctas, int max_len, int schedules,
                            const void* d_in, void* d_gamma, bool fp64, cudaStream_t stream);

// 2-D band-pass variant: low-pass |k / len| < B_c across the carrier lines of the workspace, in
// place (signed bins -cross_kc .. cross_kc). One CTA per 32 cross lines of a frame.
constexpr int kMaxCrossKc = 180;
cudaError_t init_crossband();
cudaError_t launch_crossband(const FrameDev* d_frames, int nframes, int64_t total_groups, int max_kc,
                             void* d_gamma, bool fp64, cudaStream_t stream);

// Plain path: one thread per pixel of one frame, T = float or double (Sec. 3; Algorithm 1).
constexpr int kMaxModelOrder = 3;
struct PlainArgs {
    int fb;
    int max_sweeps;
    int max_iters;
    int p;  // model order 1 .. kMaxModelOrder
};
cudaError_t launch_plain_fp64(const FrameDev* d_frame, const FrameDev& h_frame, const double2* d_gamma,
                              float* d_out, uint8_t* d_status, PlainArgs a, cudaStream_t stream);
cudaError_t launch_plain_fp32(const FrameDev* d_frame, const FrameDev& h_frame, const float2* d_gamma,
                              float* d_out, uint8_t* d_status, PlainArgs a, cudaStream_t stream);

// Statistics slots of the solvers' counters array (the BatchedArgs / SquareArgs lists below).
constexpr int kStatSlots = 10;
// Slot after the statistics: index checks that failed (checked builds only).
constexpr int kCheckSlot = kStatSlots;
// Slot after it: grid-wide waits of the phase assembly that gave up.
constexpr int kWaitSlot = kStatSlots + 1;

#ifdef __CUDACC__
// Checked builds (-DRMUSIC_CHECKS) test the solvers' data-dependent indices: rm_check(ok, counters)
// counts a failed test in counters[kCheckSlot] and returns false, so that the caller skips the
// access instead of faulting. Ordinary builds compile it to true and keep nothing of it.
#ifdef RMUSIC_CHECKS
__device__ __forceinline__ bool rm_check(bool ok, unsigned long long* counters) {
    if (!ok && counters) atomicAdd(counters + kCheckSlot, 1ull);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool rm_check(bool, unsigned long long*) { return true; }
#endif
#endif

// Batched FP32 path: persistent, warp-scheduled over all work items of all frames that share
// covariance order L. `counter` must be zero when the kernel starts.
struct BatchedArgs {
    int max_sweeps;
    int max_iters;
    int polish64;
    int exhaustive;                // 1: Jacobi sweeps and all roots for every pixel (no shortcuts)
    unsigned long long* counters;  // [0] Jacobi sweeps, [1] Aberth iterations, [2] items, [3] Aberth root
                                   // updates, [4] Aberth evaluations of Q and Q', [5] power steps,
                                   // [6] Jacobi fallbacks, [7] Newton steps, [8] Aberth fallbacks,
                                   // [9] polish steps
    int fb;                        // model-order solver: 1 = the forward-backward average of R
};
bool batched_supports(int L);
int batched_num_variants(int L);
int batched_default_variant(int L);
int batched_variant_ctas(int L, int v);  // resident CTAs per SM variant v is compiled for
cudaError_t init_batched(int device);
cudaError_t launch_batched(int L, int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                           unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                           uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream);
int batched_grid(int L, int v, int device);

// Batched FP32 path without the forward-backward average (the paper's forward estimate R = R_f):
// the same work items and arguments on the complex Hermitian R, any covariance order 2 .. kMaxL.
bool batched_fwd_supports(int L);
int batched_fwd_num_variants(int L);
int batched_fwd_default_variant(int L);
int batched_fwd_variant_ctas(int L, int v);
cudaError_t launch_batched_fwd(int L, int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                               unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                               uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream);
int batched_fwd_grid(int L, int v, int device);

// Batched FP32 path for model order p = 2 or 3 on raw real lines (batched_p_kernel.cuh): the same
// work items and arguments (a.fb selects the forward-backward average), L = p + 1 .. kMaxL, one
// register cap per L.
bool batched_p_supports(int p, int L);
int batched_p_ctas(int L);
cudaError_t launch_batched_p(int p, int L, const FrameDev* d_frames, int nframes, int64_t total_items,
                             unsigned long long* d_counter, const float2* d_gamma, float* d_out, uint8_t* d_status,
                             BatchedArgs a, int grid, cudaStream_t stream);
int batched_p_grid(int p, int L, int device);

// Square-block FP32 path (the paper's geometry): persistent, one warp per work item, over all
// frames that share the half-width Lp. The items: first every frame's 32 x kSqTY strips (the warp
// walks the rows in order, each row starting from the one above), then every frame's last rows
// (about an eighth) one 32-pixel row per item, so that the warps end together. `counter` must be
// zero when it starts.
constexpr int kMaxSquareLp = 8;
constexpr int kSqTX = 32;     // item width in pixels: one per lane
constexpr int kSqTY = 8;      // strip height: the rows one warp walks in order
constexpr int kSqWarps = 4;   // warps of the 128-thread CTA, each on its own items
constexpr int kSqTailDiv = 8; // about H / kSqTailDiv rows of each frame go one row per item
// Rows of an H-row frame that go in strips (a multiple of kSqTY).
__host__ __device__ constexpr int square_strip_rows(int H) { return kSqTY * ((H - H / kSqTailDiv) / kSqTY); }
struct SquareArgs {
    int max_power_iters;
    int max_iters;
    int polish64;
    int exhaustive;                // 1: all roots for every pixel (no Newton certificate)
    float tol2;                    // power iteration stops when |u_new - u|^2 <= tol2
    unsigned long long* counters;  // [0] power iterations, [1] Aberth iterations, [2] warps, [3] Aberth root
                                   // updates, [4] Aberth evaluations of Q and Q', [5] warm starts,
                                   // [7] Newton steps, [8] Aberth fallbacks, [9] polish steps (root
                                   // figures: both polynomials)
    const unsigned char* direct;   // non-null: every frame is complex64 and read in place, frame f's
                                   // row y at direct + F.in_off + 8 F.pitch y (d_gamma is not read)
};
bool square_supports(int Lp);
int square_num_variants(int Lp);
int square_default_variant(int Lp);
int square_variant_ctas(int Lp, int v);
cudaError_t launch_square(int Lp, int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                          unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                          uint8_t* d_status, SquareArgs a, int grid, cudaStream_t stream);
int square_grid(int Lp, int v, int device);

// Phase assembly (unwrap.cu): unwraps the wrapped map of every frame of the table (frame f's
// pixels are g = F.gam_off .. F.gam_off + H W - 1; its input map at in + F.out_off + in_maps H W,
// its output at out + F.out_off + out_maps H W; NaN = no value). max_frame_nodes is the largest
// unwrap_frame_nodes(H, W) over the frames (it bounds the rounds); any larger value is safe. work
// must hold unwrap_workspace_bytes(npx, max_frame_nodes) bytes; npx < 2^31. The global phase's
// first launched_rounds rounds (-1: half the rounds bound, rounded up; clamped to the bound) run as
// two launches each, the rest in one cooperative launch whose CTAs wait on one another at
// grid-wide barriers; a wait that gives up (after 0.5 s) stops that kernel and adds one to
// *timeouts (a device counter, may be null): the output of that call is then incomplete.
int64_t unwrap_frame_nodes(int H, int W);
size_t unwrap_workspace_bytes(int64_t npx, int64_t max_frame_nodes);
cudaError_t launch_unwrap(const FrameDev* d_frames, int nframes, int64_t npx, int64_t max_frame_nodes,
                          const float* in, int64_t in_maps, float* out, int64_t out_maps, void* work,
                          int launched_rounds, unsigned long long* timeouts, int* launches, cudaStream_t s);

}  // namespace rmusic
