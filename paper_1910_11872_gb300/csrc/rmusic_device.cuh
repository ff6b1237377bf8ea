// rmusic_device.cuh -- device-side types and helpers shared by the library's CUDA sources.
//
// Data layout in HBM for one call (all frames of the call share one workspace):
//   frames   caller's buffer, frame f at byte offset in_off, row pitch `pitch` elements.
//   gamma    library workspace, complex64 analytic signal (Sec. 2, Eq. 1) of every frame,
//            stored "window-line major": the window runs along a contiguous line, so
//            gamma[gam_off + wline * wlen + pos] is the sample at position `pos` of window
//            line `wline` (wline = y, pos = x when windows run along x; wline = x, pos = y
//            when they run along y).
//   out      caller's float32 maps, frame f dense H x W row-major at element offset out_off
//            (square geometry: three maps, d/dx at out_off, d/dy at out_off + H W and the
//            local phase alpha at out_off + 2 H W).
//   status   caller's optional uint8 maps, one per frame at element offset out_off.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rmusic {

constexpr int kMaxL = 12;        // largest covariance order L
constexpr int kMaxN = 64;        // largest window length N
constexpr int kMaxLine = 8192;   // longest carrier line the band-pass kernel accepts
// Row geometry, FP32-batched path: one warp work item is a run of 32 P consecutive pixels of a
// window line, starting at a multiple of 32 P; lane l owns its pixels l P .. l P + P - 1. P is a
// property of the frame (FrameDev::rowp_shift, P = 1 << rowp_shift), kRowPMin <= P <= kRowP:
// row_pixels_per_lane_shift picks it from the window-line length.
constexpr int kRowP = 16;
constexpr int kRowPMin = 8;
constexpr int kRowRun = 32 * kRowP;

// log2 of the pixels per lane for window lines of wlen pixels: 16 (anchors amortised over more
// pixels), unless 8 leaves fewer idle lanes at the line's end by more than a sixteenth of the line
// (lines of 256 or 768 pixels take 8, of 512 or 1024 take 16).
__host__ __device__ constexpr int row_pixels_per_lane_shift(int wlen) {
    return ((wlen + 511) / 512) * 512 - wlen > ((wlen + 255) / 256) * 256 - wlen + wlen / 16 ? 3 : 4;
}

enum : uint8_t { kStOk = 0, kStBorder = 1, kStDegenerate = 2, kStNotConverged = 3 };

// Frame sample types (the values of RMUSIC_DTYPE_*) and solver geometries (RMUSIC_GEOM_*).
enum : int32_t { kDtF32 = 0, kDtU16 = 1, kDtC64 = 2 };
enum : int32_t { kGeomRow = 0, kGeomSquare = 1 };

// Per-frame entry of the device frame table (built on the host for each call).
struct FrameDev {
    uint64_t in_off;      // byte offset of the frame in the input buffer
    uint64_t out_off;     // element offset of the frame's map in out / status
    uint64_t gam_off;     // element offset of the frame's analytic signal in the workspace
    int64_t line_start;   // first carrier line of this frame in the band-pass grid
    int64_t item_start;   // first warp work item of this frame in the batched schedule
    int64_t item_start2;  // square geometry: first single-row item of this frame (they follow every
                          // frame's strips)
    int32_t H, W, pitch, dtype;
    int32_t N, L;
    int32_t carrier_axis, deriv_axis;
    int32_t nlines, len;  // carrier lines and their length
    int32_t k_lo, nb;     // kept DFT bins k_lo .. k_lo + nb - 1 of a carrier line
    int32_t wlines, wlen; // window lines and their length
    int32_t nchunks;      // row geometry: work items per window line (ceil(wlen / (32 << rowp_shift)));
                          // square geometry: tiles per tile row (ceil(W / 32))
    int32_t geom;         // kGeomRow or kGeomSquare (then L holds the half-width Lp, N = 2 Lp + 1)
    double omega_ref;     // carrier phase step removed from the angle (rad/pixel)
    double f0;            // carrier frequency (cycles/pixel)
    int64_t cross_start;  // first 32-line group of this frame in the cross-band grid
    int32_t cross_kc;     // cross band: signed bins -kc .. kc kept across the carrier (0: none)
    int32_t raw;          // 1: no band-pass; Gamma = the real line minus its mean
    int32_t band_r;       // band-pass schedule: 0 one CTA per carrier line; 8, 16 or 32: lines of
                          // 32 band_r samples in groups of 4 x 32 / band_r per CTA (warp FFTs)
    int32_t rowp_shift;   // row geometry, FP32-batched path: log2 of the pixels each lane owns
    int32_t sq_strip_rows; // square geometry: rows 0 .. sq_strip_rows - 1 go in strips of kSqTY rows,
                           // the rest one row per item
};

// Index of the frame that owns global index `g` given each frame's start (non-decreasing).
template <typename Get>
__device__ __forceinline__ int find_frame(const FrameDev* __restrict__ fr, int nframes, int64_t g,
                                          Get start) {
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (start(fr[mid]) <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Map a (window line, position) pair to the output element index of the frame.
__device__ __forceinline__ uint64_t out_index(const FrameDev& F, int wline, int pos) {
    int y = F.deriv_axis == 0 ? wline : pos;
    int x = F.deriv_axis == 0 ? pos : wline;
    return F.out_off + (uint64_t)y * (uint64_t)F.W + (uint64_t)x;
}

// Minimal complex arithmetic for float and double.
template <typename T>
struct cx {
    T r, i;
};

template <typename T>
__device__ __forceinline__ cx<T> mkc(T r, T i) {
    cx<T> z;
    z.r = r;
    z.i = i;
    return z;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mkc(a.r + b.r, a.i + b.i); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mkc(a.r - b.r, a.i - b.i); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mkc(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mkc(s * a.r, s * a.i); }
template <typename T>
__device__ __forceinline__ cx<T> conjg(cx<T> a) { return mkc(a.r, -a.i); }
template <typename T>
__device__ __forceinline__ T norm2(cx<T> a) { return a.r * a.r + a.i * a.i; }
// a * conj(b)
template <typename T>
__device__ __forceinline__ cx<T> mulc(cx<T> a, cx<T> b) {
    return mkc(a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i);
}
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
    T d = b.r * b.r + b.i * b.i;
    T inv = T(1) / d;
    return mkc((a.r * b.r + a.i * b.i) * inv, (a.i * b.r - a.r * b.i) * inv);
}
template <typename T>
__device__ __forceinline__ cx<T> crecip(cx<T> b) {
    T inv = T(1) / (b.r * b.r + b.i * b.i);
    return mkc(b.r * inv, -b.i * inv);
}

template <typename T>
__device__ __forceinline__ T wrap_pi(T a) {
    const T pi = T(3.14159265358979323846);
    const T two_pi = T(6.28318530717958647692);
    if (a > pi) a -= two_pi;
    if (a <= -pi) a += two_pi;
    return a;
}

}  // namespace rmusic
