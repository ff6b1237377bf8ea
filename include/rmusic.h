/*
 * rmusic.h -- C ABI of the GB300 (sm_103a) sliding-window root-MUSIC phase-derivative library.
 *
 * The library turns a stack of carrier-fringe frames into per-pixel local phase-derivative
 * maps with the root-MUSIC estimator of Ramaiah, Ajithaprasad, Rajshekhar and Ambrosini,
 * "Fast and robust method for flow analysis using GPU assisted diffractive optical element
 * based background oriented schlieren (BOS)", arXiv:1910.11872:
 *   - analytic signal of each line by band-pass filtering       (Sec. 2, Eq. 1)
 *   - moving window and local linear-phase model                  (Sec. 3, Eq. 2-3)
 *   - sample auto-correlation matrix R of the window               (Sec. 3, Eq. 4-5)
 *   - signal eigenvector u1 and noise subspace                     (Sec. 3, Eq. 6-11)
 *   - root-MUSIC polynomial of the noise projector                 (Sec. 3, Eq. 12-14)
 *   - the root nearest the unit circle with |z| <= 1               (Sec. 3; Algorithm 1)
 *   - its angle, minus the carrier, is the phase derivative        (Sec. 3, Eq. 15)
 * Two window geometries: a window of N samples along one axis with Hankel snapshots (the
 * workloads' row windows), and the paper's own square block of (2 Lp + 1) x (2 Lp + 1) samples
 * whose columns and conjugated rows are the snapshots, giving both derivatives and the local
 * phase alpha of Eq. 15 at once (Sec. 3, Eq. 4-15; Algorithm 1).
 *
 * Conventions shared by every entry point:
 *   - All functions are plain C, callable from any language; no C++ exceptions cross them.
 *   - Return codes: RMUSIC_OK (0) or a negative RMUSIC_E* value; rmusic_strerror() names it.
 *   - "Device pointer" means memory of the context's CUDA device (cudaMalloc, a PyTorch
 *     tensor's data_ptr(), ...). The caller owns every pointer it passes; the library only
 *     reads inputs and writes outputs during the call's stream-ordered execution.
 *   - The library owns its workspaces, graphs and tables, all released by rmusic_destroy.
 *   - Work is queued asynchronously on the caller's stream (cudaStream_t passed as void*;
 *     NULL = the legacy default stream); results are valid once that stream reaches the
 *     point after the call.
 *   - A context is not thread-safe: use one per host thread. Calls on one context share its
 *     workspace, so they must be ordered (one stream, or synchronised between streams).
 */
#ifndef RMUSIC_H
#define RMUSIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------------- */
#define RMUSIC_OK 0
#define RMUSIC_EINVAL (-1)       /* an argument is out of range or inconsistent             */
#define RMUSIC_ENOMEM (-2)       /* a workspace would exceed the HBM budget / cudaMalloc failed */
#define RMUSIC_EUNSUPPORTED (-3) /* a valid request this build does not implement           */
#define RMUSIC_ETIMEDOUT (-4)    /* a bounded device-side wait gave up                      */
#define RMUSIC_ECUDA (-5)        /* a CUDA runtime call failed (see rmusic_last_cuda_error)   */
#define RMUSIC_EAGAIN (-6)       /* serving: every frame slot of the stream is busy, retry later */

/* ---- execution paths (rmusic_params.precision) ----------------------------------------- */
#define RMUSIC_PLAIN_FP64 0   /* thread per pixel, FP64 throughout, one launch per frame     */
#define RMUSIC_PLAIN_FP32 1   /* thread per pixel, FP32 throughout, one launch per frame     */
#define RMUSIC_FP32_BATCHED 2 /* persistent warp-scheduled FP32 kernel over all frames       */

/* ---- input sample types (rmusic_frame_desc.dtype) -------------------------------------- */
#define RMUSIC_DTYPE_F32 0 /* float32 intensity                                             */
#define RMUSIC_DTYPE_U16 1 /* uint16 camera code (e.g. 12-bit); any scale gives the same map */
#define RMUSIC_DTYPE_C64 2 /* complex64 (re, im float32): already the analytic signal Gamma,  */
                           /* used as is without the band-pass (the paper's complex fringe)  */

/* ---- window geometries (rmusic_params.geometry) ---------------------------------------- */
#define RMUSIC_GEOM_ROW 0    /* N samples along deriv_axis, snapshots of length L           */
#define RMUSIC_GEOM_SQUARE 1 /* the paper's (2 Lp + 1)^2 block: d/dx, d/dy and alpha        */

/* ---- per-pixel status codes (optional uint8 map) --------------------------------------- */
#define RMUSIC_STATUS_OK 0
#define RMUSIC_STATUS_BORDER 1        /* the window leaves the line: derivative is NaN      */
#define RMUSIC_STATUS_DEGENERATE 2    /* R is zero or its top eigenvalue is not separated   */
#define RMUSIC_STATUS_NOT_CONVERGED 3 /* an iteration cap was hit; best estimate is stored  */

/* Parameters of the estimator (Sec. 3) and of the execution path.
 *   window_len       N, samples in the moving window along deriv_axis (2 <= N <= 64). The
 *                    window of the pixel at position n covers n - N/2 .. n - N/2 + N - 1
 *                    (integer N/2); pixels whose window leaves the line are border pixels.
 *   cov_order        L, length of the snapshots s_i = w[i .. i+L-1], i = 0 .. N-L, and order of
 *                    the L x L auto-correlation matrix (2 <= L <= 12, L <= N). The batched path
 *                    takes even L with forward_backward = 1 (a real symmetric transform of R) and
 *                    any L with forward_backward = 0 (the complex Hermitian R); odd L with the
 *                    forward-backward average needs a plain path.
 *   model_order      number of complex exponentials per window; the method uses 1 (Eq. 2). All
 *                    row-window paths also take 2 or 3 (a real fringe without the analytic step
 *                    holds exp(+-j omega), and a local offset one more at zero frequency): the noise
 *                    projector then removes the p largest eigenvalues' eigenvectors, and the
 *                    derivative comes from the one of the p roots nearest the unit circle whose
 *                    angle is nearest the expected one (2 pi f0). Needs cov_order > model_order.
 *                    RMUSIC_FP32_BATCHED takes it with raw_input = 1 on float32 or uint16 frames
 *                    (RMUSIC_EUNSUPPORTED otherwise); its FP32 roots lose accuracy (a few 1e-4 rad)
 *                    when cov_order <= model_order + 2, where the roots crowd in pairs.
 *   forward_backward 1: R = (R_f + J conj(R_f) J) / 2 (forward-backward average); 0: R = R_f,
 *                    the forward estimate of Eq. 4-5 alone (its signal root lies further inside
 *                    the circle on noisy windows; both give the same derivative on noise-free
 *                    constant-amplitude fringes).
 *   deriv_axis       0: windows run along x (rows); 1: along y (columns).
 *   carrier_axis     axis of the carrier and of the band-pass (0 = x, 1 = y).
 *   carrier_freq     f0 in cycles/pixel; the band keeps 1 <= k < len/2 with |k/len - f0| < B,
 *                    and 2 pi f0 is subtracted from the angle when deriv_axis == carrier_axis.
 *   band_halfwidth   B in cycles/pixel; <= 0 selects f0 / 2.
 *   precision        RMUSIC_PLAIN_FP64, RMUSIC_PLAIN_FP32 or RMUSIC_FP32_BATCHED.
 *   max_sweeps       cap on Jacobi sweeps (0 = default: 30 plain, 6 batched).
 *   max_root_iters   cap on root iterations (0 = default: 500 plain, 16 batched).
 *   polish_fp64      batched path only: 1 adds one FP64 Newton step on the selected root.
 *   use_graph        batched path only: 1 captures the whole call in a CUDA graph and replays
 *                    it when the same frames, tables and outputs are passed again.
 *   timing           1: record CUDA events around every kernel of a call on its stream, so that
 *                    rmusic_get_stats() can report the device time of each stage.
 *   autotune         batched path: 1 lets the first call that meets a covariance order with no
 *                    tuned solver variant on this device time all variants on its own work and
 *                    keep the fastest (that call synchronises its stream). See rmusic_autotune.
 *   geometry         RMUSIC_GEOM_ROW (0) or RMUSIC_GEOM_SQUARE (1). The square block needs
 *                    precision RMUSIC_FP32_BATCHED; window_len, cov_order, forward_backward and
 *                    deriv_axis are then ignored (the paper's estimate has no FB average).
 *   half_width       square geometry: Lp, the block is (2 Lp + 1) x (2 Lp + 1) (1 <= Lp <= 8).
 *                    A pixel whose block leaves the frame is a border pixel. max_sweeps then caps
 *                    the power-iteration steps of the block's singular vectors (0 = 100).
 *   unwrap           square geometry only: 1 also assembles the phase map (Sec. 3: the local
 *                    phases are unwrapped with the reliability-sorting method the paper cites) and
 *                    writes it as a fourth map per frame (see rmusic_unwrap_phase).
 *   band_cross       B_c in cycles/pixel, 0 <= B_c < 0.5: when > 0, the analytic signal is also
 *                    low-passed across the carrier lines to |k / len| < B_c (k the signed bin), so
 *                    the kept band is a rectangle of the 2-D spectrum (a 2-D band-pass variant, after
 *                    the 2-D Fourier methods the paper cites for its band-pass). At most 361 kept
 *                    bins per line (B_c len <= 181); applies to complex frames too. Not supported
 *                    by rmusic_demodulate_frames_noalloc.
 *   raw_input        1: no band-pass; the window holds the real samples of the carrier line minus
 *                    the line's mean (for model_order 2 or 3). Needs the row geometry with
 *                    deriv_axis == carrier_axis (the carrier decides which of +-omega is meant).
 *   exhaustive       batched path: 0 (default) finds the selected root by Newton's method and
 *                    certifies it with a root count -- in the row geometry with L <= 10 by Rouche's
 *                    theorem against the noise-free polynomial, with the Schur-Cohn count where that
 *                    test does not decide; otherwise by the Schur-Cohn count -- (every root is
 *                    computed only where the certificate fails), and the row geometry's eigenvector by power iteration
 *                    (Jacobi sweeps only where it does not settle); 1 computes every inner root by
 *                    Aberth-Ehrlich and, in the row geometry, runs the Jacobi sweeps for every
 *                    pixel. Both select the same root; 1 is slower.
 * carrier_freq may be 0 (no carrier) for complex frames; for real frames it must lie in (0, 0.5).
 */
typedef struct {
    int32_t window_len;
    int32_t cov_order;
    int32_t model_order;
    int32_t forward_backward;
    int32_t deriv_axis;
    int32_t carrier_axis;
    double carrier_freq;
    double band_halfwidth;
    int32_t precision;
    int32_t max_sweeps;
    int32_t max_root_iters;
    int32_t polish_fp64;
    int32_t use_graph;
    int32_t timing;
    int32_t autotune;
    int32_t geometry;
    int32_t half_width;
    int32_t unwrap;
    double band_cross;
    int32_t raw_input;
    int32_t exhaustive;
} rmusic_params;

/* One frame of a batch. Frames of one call may differ in size, type and window.
 *   offset_bytes  byte offset of the frame's first sample from the base input pointer.
 *   height/width  H, W in pixels (>= 1).
 *   pitch_elems   elements between the starts of consecutive rows (>= width; 0 = width).
 *   dtype         RMUSIC_DTYPE_F32, RMUSIC_DTYPE_U16 or RMUSIC_DTYPE_C64. offset_bytes and
 *                 pitch must keep every sample naturally aligned.
 *   out_offset    element offset of the frame's dense H x W float32 map (row-major) in the
 *                 output buffer, and of its H x W uint8 map in the status buffer. In the square
 *                 geometry a frame writes three maps: d/dx at out_offset, d/dy at
 *                 out_offset + H W and alpha at out_offset + 2 H W (3 H W floats; with
 *                 params.unwrap = 1 a fourth map, the unwrapped phase, at out_offset + 3 H W),
 *                 and its status map at out_offset of the status buffer.
 *   window_len, cov_order  per-frame N and L; 0 = the context's parameters.
 */
typedef struct {
    uint64_t offset_bytes;
    int32_t height;
    int32_t width;
    int32_t pitch_elems;
    int32_t dtype;
    uint64_t out_offset;
    int32_t window_len;
    int32_t cov_order;
} rmusic_frame_desc;

typedef struct rmusic_ctx rmusic_ctx;

/* Create a context on CUDA device `device` with the given parameters. hbm_budget_bytes caps
 * the device memory the library may allocate for its workspaces (0 = no cap); calls whose
 * workspace would exceed it are split into smaller batches, or fail with RMUSIC_ENOMEM if a
 * single frame does not fit. On success *out receives the context. Errors: RMUSIC_EINVAL
 * (bad parameters, out == NULL), RMUSIC_EUNSUPPORTED (model_order != 1), RMUSIC_ECUDA. */
int rmusic_create(const rmusic_params* params, int device, size_t hbm_budget_bytes,
                  rmusic_ctx** out);

/* Demodulate n_frames frames (Sec. 3, Eq. 2-15, all pixels of all frames).
 *   d_frames  device pointer; frame f starts at (const char*)d_frames + descs[f].offset_bytes.
 *   descs     HOST array of n_frames descriptors; copied by the library before return.
 *   d_out     device float32 buffer; frame f writes H*W values at d_out + descs[f].out_offset:
 *             the phase derivative in rad/pixel along deriv_axis, NaN where undefined. In the
 *             square geometry three maps of H*W values: d/dx and d/dy in rad/pixel and the
 *             local phase alpha in rad, wrapped to (-pi, pi], with the carrier's phase
 *             2 pi f0 X at the pixel removed (X the pixel's coordinate along carrier_axis).
 *   d_status  device uint8 buffer laid out like d_out, or NULL.
 *   cuda_stream  cudaStream_t (as void*) on which all work is queued.
 * Errors: RMUSIC_EINVAL (NULL pointers with n_frames > 0, a bad descriptor, unsupported
 * (N, L) for the path), RMUSIC_EUNSUPPORTED (a frame of 2^31 or more 512-pixel work items, about
 * 1.1e12 pixels: far beyond what fits a GPU), RMUSIC_ENOMEM, RMUSIC_ECUDA. n_frames == 0 is a
 * no-op. */
int rmusic_demodulate_frames(rmusic_ctx* ctx, const void* d_frames, const rmusic_frame_desc* descs,
                             int32_t n_frames, float* d_out, uint8_t* d_status, void* cuda_stream);

/* Batched path only: the FP32-batched solver is compiled in several variants per covariance order
 * that differ in how many CTAs they keep resident per SM (register cap vs latency hiding; the
 * best one depends on L and on the GPU). This call demodulates like rmusic_demodulate_frames but
 * first times every variant on the call's own frames for each covariance order they use, keeps
 * the fastest for this device (all contexts of the process share the choice) and, when the
 * environment variable RMUSIC_TUNE_CACHE names a file, appends the choice to it as a JSON line
 * that later processes read. Synchronises its stream. Without tuning a default variant is used.
 * The paper has no counterpart: this is a property of the GPU implementation. */
int rmusic_autotune(rmusic_ctx* ctx, const void* d_frames, const rmusic_frame_desc* descs, int32_t n_frames,
                    float* d_out, uint8_t* d_status, void* cuda_stream);

/* Same as rmusic_demodulate_frames_host, but asynchronous: the call queues the work on
 * cuda_stream and returns; the maps are complete once the stream's work is (cudaStreamSynchronize
 * or an event recorded after the call). The frames are always staged into the context's workspace
 * by the copy engine -- which needs no SM -- so a caller alternating two contexts on two streams
 * (double buffering) overlaps the frames' transfer of one call with the kernels of the other;
 * pinned output buffers are written in place by the solver where its stores are coalesced (plain
 * paths, square geometry without unwrap), others through the workspace and a copy queued at the
 * end. The host buffers must stay valid and the input unchanged until the
 * stream has completed the call (pageable input is copied before the call returns), and a context
 * serves one call at a time: the next call on it must follow on the same stream or after the
 * previous one completes. Errors: as rmusic_demodulate_frames_host; a CUDA error met while the
 * work runs surfaces at the caller's synchronisation. */
int rmusic_demodulate_frames_host_async(rmusic_ctx* ctx, const void* h_frames, size_t in_bytes,
                                        const rmusic_frame_desc* descs, int32_t n_frames, float* h_out,
                                        uint8_t* h_status, void* cuda_stream);

/* Pre-allocate the context's device workspace for calls of up to max_pixels pixels in total
 * (sum of height x width over the call's frames) and up to max_frames frames: the analytic-signal
 * buffer (8 bytes per pixel, 16 on the plain FP64 path), the frame tables (device and pinned
 * host) and, with unwrap = 1, the phase-assembly workspace. A later call within these limits
 * allocates nothing, so it never waits for the device as a buffer that grows does (freeing
 * device memory synchronises the device): what a serving loop or a real-time caller needs.
 * Without it the workspace grows on demand. The reservation counts against the context's HBM
 * budget and is kept until rmusic_destroy. It does not cover the host-buffer entries' staging
 * buffers (frames and maps in device memory, sized by the frames' element type), which a context
 * allocates on its first host-buffer call and reuses while the calls do not grow. Synchronises the device when it replaces a smaller
 * buffer. Errors: RMUSIC_EINVAL (NULL context, max_frames < 0, max_pixels >= 2^31 with
 * unwrap = 1), RMUSIC_ENOMEM (the reservation exceeds the budget: nothing changes; or the device
 * is out of memory: the buffer being replaced is gone and later calls allocate on demand).
 * max_pixels = 0 or max_frames = 0 reserves nothing of that kind.
 * The paper has no counterpart: this is a property of the GPU implementation. */
int rmusic_reserve(rmusic_ctx* ctx, uint64_t max_pixels, int32_t max_frames);

/* Same as rmusic_demodulate_frames, but every buffer is in HOST memory; the maps are complete when
 * the call returns (it synchronises its stream). in_bytes is the size of h_frames. Buffers the GPU
 * can address directly (pinned memory from cudaHostAlloc / cudaMallocHost, or registered with
 * cudaHostRegister) are used in place: the band-pass kernel reads the frames and the solver writes
 * the maps over the host link while it runs, instead of a copy before and after the kernels. The
 * maps are staged on the device instead (and copied back at the end) for the FP32-batched row
 * solver, whose lanes each write 16 consecutive pixels (one store instruction touches 32 pixels 64
 * bytes apart: one host-link transaction per pixel), and with phase assembly (square geometry with
 * unwrap = 1), which rereads its maps.
 * Pageable buffers are copied to and from the context's device workspace. The results are
 * identical either way. */
int rmusic_demodulate_frames_host(rmusic_ctx* ctx, const void* h_frames, size_t in_bytes,
                                  const rmusic_frame_desc* descs, int32_t n_frames, float* h_out,
                                  uint8_t* h_status, void* cuda_stream);

/* For callers that cannot allocate device memory (an application whose allocator belongs to a
 * host framework or pool, a real-time loop that forbids allocation after start-up, a plug-in
 * whose host accounts for every byte): the FP32-batched path (precision must be
 * RMUSIC_FP32_BATCHED, forward_backward 1, geometry RMUSIC_GEOM_ROW) without a context and without any cudaMalloc,
 * cudaFree or other allocating call. The paper has no counterpart; this is an interface
 * convenience of this library.
 *   - All device scratch (analytic signal, frame table, work counters) lives in one fixed array
 *     inside the library's device code, about 32 MiB per GPU, held from the moment that code is
 *     loaded on the GPU (with CUDA's default lazy loading: this entry point's first call there)
 *     until the process exits. With eager module loading (CUDA_MODULE_LOADING=EAGER) every
 *     process that loads the library pays the 32 MiB on each GPU it uses, whether or not it ever
 *     calls this entry point; a process that also loads the checked build of the library
 *     (RMUSIC_CHECKS) holds a second, separate array for it. The caller passes frames and output
 *     maps exactly as for rmusic_demodulate_frames; descs is a host array read before the call
 *     returns.
 *   - Parameters and descriptors are validated exactly as rmusic_create and
 *     rmusic_demodulate_frames validate them (same codes), then this entry point adds its own
 *     restrictions (RMUSIC_EUNSUPPORTED otherwise).
 *   - The solver always runs the default register-cap variant for each covariance order (no
 *     tuning run, which would need timing buffers); its maps equal those of a context pinned to
 *     that variant with rmusic_set_solver_variant.
 *   - Limits: at most 4,194,304 pixels (e.g. four 1024 x 1024 frames) and 256 frames per call;
 *     larger requests are rejected with RMUSIC_ENOMEM before any work is queued.
 *   - The first call on a device looks the array's address up (cudaGetSymbolAddress) and sets
 *     the kernels' attributes; make that first call before any stream capture.
 *   - Every call on a device reuses the same array, so calls whose work overlaps on the GPU
 *     (different streams without ordering, or several host threads) race and corrupt each
 *     other's results: order them on one stream or synchronise between them.
 *   - device is the CUDA device to run on; the calling thread's current device is restored.
 * Errors: RMUSIC_EINVAL, RMUSIC_EUNSUPPORTED, RMUSIC_ENOMEM (over the limits), RMUSIC_ECUDA. */
int rmusic_demodulate_frames_noalloc(const rmusic_params* params, int device, const void* d_frames,
                                     const rmusic_frame_desc* descs, int32_t n_frames, float* d_out,
                                     uint8_t* d_status, void* cuda_stream);

/* Phase assembly (Sec. 3: the local phases are followed by an unwrapping operation, the
 * reliability-sorting method of Herraez et al. 2002 that the paper cites). Unwraps n_frames wrapped
 * phase maps, e.g. the alpha maps of the square geometry:
 *   d_phase  device float32 buffer; frame f's H x W map (row-major) at d_phase + descs[f].out_offset,
 *            values in (-pi, pi], NaN where a pixel has no value (border pixels).
 *   d_out    device float32 buffer; frame f's unwrapped map at d_out + descs[f].out_offset, NaN
 *            where the input is NaN. d_out may equal d_phase (in place).
 *   descs    HOST array; only height, width and out_offset are read.
 * Pixels with values that touch horizontally or vertically form regions; each region is unwrapped
 * as the method does (edges taken by decreasing reliability, the reliability of a pixel being the
 * inverse of its wrapped second differences, 0 where a neighbour has no value) and then shifted so
 * that its first pixel in row-major order keeps its wrapped value. Reliabilities and 2 pi jumps
 * are decided in float32. The work is a fixed sequence of kernels queued on cuda_stream: three per
 * pixel or per 32 x 32 tile; for the global phase's R = ceil(log2(n)) + 1 rounds (n the border
 * pixels of the largest frame's 32 x 32 tiles) two per round of the first ceil(R / 2), then one
 * cooperative launch (every CTA resident) for the rest, whose CTAs wait on one another at
 * grid-wide barriers, each wait bounded (see rmusic_stats.wait_timeouts); two per pixel at the
 * end. Total pixels of a call: below 2^31.
 * Errors: RMUSIC_EINVAL, RMUSIC_ENOMEM (workspace of about 132 bytes per pixel over the budget),
 * RMUSIC_ECUDA. */
int rmusic_unwrap_phase(rmusic_ctx* ctx, const float* d_phase, const rmusic_frame_desc* descs, int32_t n_frames,
                        float* d_out, void* cuda_stream);

/* rmusic_unwrap_phase with the global phase's schedule given: its first launched_rounds rounds
 * (clamped to R) as two launches each, the rest in the cooperative launch; -1 is
 * rmusic_unwrap_phase's own split, ceil(R / 2); 0 runs every round cooperatively. Every split
 * computes the same maps bit for bit (for tests and measurement).
 * Errors: those of rmusic_unwrap_phase; RMUSIC_EINVAL for launched_rounds < -1. */
int rmusic_unwrap_phase_sched(rmusic_ctx* ctx, const float* d_phase, const rmusic_frame_desc* descs, int32_t n_frames,
                              float* d_out, int32_t launched_rounds, void* cuda_stream);

/* Batched path: pin the solver variant this context uses for covariance order `order` (row
 * geometry) or half-width `order` (square geometry), overriding the autotuner's choice; -1 returns
 * to it. Row geometry: variants 0, 1, 2 differ only in their register cap (2, 3 ... 16 resident
 * CTAs per SM depending on L; the same source, though the compiler may fuse multiply-adds
 * differently in each, so maps agree to FP32 rounding and statuses are identical); variant 3
 * (L <= 8) runs the eigenvalue sweeps with one warp per matrix instead of one thread per matrix
 * (the same stopping rule; results agree to FP32 rounding). Each variant is deterministic: a
 * pixel's result does not depend on the frames batched with it or on the schedule. Square geometry: variants 0 and 1, register caps. Useful to compare the
 * schedules on a given GPU. Errors: RMUSIC_EINVAL (bad order or variant), RMUSIC_EUNSUPPORTED
 * (not the batched path). */
int rmusic_set_solver_variant(rmusic_ctx* ctx, int32_t order, int32_t variant);

/* Destroy a context and free everything it owns. NULL is allowed. Waits for the context's
 * outstanding work on its device. */
void rmusic_destroy(rmusic_ctx* ctx);

/* Static, human-readable name of a return code. */
const char* rmusic_strerror(int code);

/* Text of the last CUDA error seen by this context (static storage inside ctx), or "". */
const char* rmusic_last_cuda_error(const rmusic_ctx* ctx);

/* 1 if this library was compiled with RMUSIC_CHECKS: the FP32-batched solvers then test their
 * work items' data-dependent indices (frame, window line, window length, covariance order) and
 * count failures in rmusic_stats.check_violations instead of touching memory out of range -- the
 * stand-in for a device memory checker. 0 for the ordinary build, which carries none of it. */
int rmusic_checked_build(void);

/* Counters of the last call on this context (for measurement and tests).
 *   kernel_launches  kernels the last call queued (graph replays count their kernels).
 *   graph_replayed   1 if the last call replayed a cached CUDA graph.
 *   workspace_bytes  device bytes the context currently holds.
 *   pixels           pixels of all frames of the last call.
 *   mean_sweeps      batched path: Jacobi sweeps per 32-pixel group (the 32 pixels a warp solves
 *                    together: one per lane), averaged (the eigen fallback's; 0 where the power
 *                    iteration sufficed).
 *   mean_root_iters  batched path: Aberth iterations per 32-pixel group, averaged (the root
 *                    fallback's; 0 where the Newton root was certified in every lane).
 *   mean_root_updates batched path: Aberth root updates a warp executed per 32-pixel group, averaged
 *                    (roots already converged in every lane of the warp are skipped).
 *   mean_root_evals  batched path: Aberth evaluations of Q and Q' a warp executed per 32-pixel group,
 *                    averaged (a root frozen in every lane of the warp is not evaluated).
 *   mean_power_steps row geometry: power-iteration steps per 32-pixel group, averaged.
 *   eig_fallback_frac row geometry: fraction of 32-pixel groups whose warp ran the Jacobi fallback.
 *   mean_newton_steps batched path: Newton steps of the signal root per 32-pixel group, averaged.
 *   root_fallback_frac batched path: fraction of 32-pixel groups whose warp ran the Aberth fallback.
 *   mean_polish_steps batched path: polish steps of the selected root per 32-pixel group, averaged.
 *   check_violations  batched path, checked builds only (rmusic_checked_build() == 1): index
 *                    tests of the solvers that failed in the last call (each skips its work item
 *                    instead of faulting; 0 is the only acceptable value). Always 0 otherwise.
 *   wait_timeouts    phase assembly (unwrap = 1, or the last rmusic_unwrap_phase call): grid-wide
 *                    waits of its cooperative kernel that gave up (0.5 s each; the kernel then
 *                    stops and that call's unwrapped maps are incomplete). 0 in every correct run.
 *   In the square geometry a 32-pixel group is one warp's 32 pixels of a strip row, mean_sweeps counts
 *   power-iteration steps, mean_power_steps the fraction of groups in which some pixel started from
 *   the row above's right singular vector (one extra block product), and the root figures add both
 *   polynomials (root_fallback_frac up to 2, mean_polish_steps counts both).
 *   bandpass_ms, solver_ms  with params.timing = 1: summed device time (CUDA events on the
 *                    call's stream) of the band-pass launches and of the solver launches.
 *   solver_ctas_per_sm  batched path: resident CTAs per SM of the solver variant last launched.
 *   solver_variant   batched path: index of that variant (see rmusic_set_solver_variant).
 * rmusic_get_stats waits until the last call's work has finished. */
typedef struct {
    int32_t kernel_launches;
    int32_t graph_replayed;
    uint64_t workspace_bytes;
    uint64_t pixels;
    double mean_sweeps;
    double mean_root_iters;
    double mean_root_updates;
    double mean_root_evals;
    float bandpass_ms;
    float solver_ms;
    int32_t solver_ctas_per_sm;
    int32_t solver_variant;
    double mean_power_steps;
    double eig_fallback_frac;
    double mean_newton_steps;
    double root_fallback_frac;
    double mean_polish_steps;
    uint64_t check_violations;
    uint64_t wait_timeouts;
} rmusic_stats;

int rmusic_get_stats(const rmusic_ctx* ctx, rmusic_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* RMUSIC_H */
