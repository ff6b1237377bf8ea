// crossband.cu -- the 2-D band-pass variant's second pass (Sec. 2: the analytic signal from
// band-pass filtering; the 2-D Fourier methods the paper cites): after the one-sided carrier band
// of analytic.cu, every line ACROSS the carrier is low-passed to |k / len| < B_c (k the signed
// bin), which makes the kept band a rectangle of the 2-D spectrum.
//
// One CTA takes 32 adjacent cross lines of one frame. Positions along the lines are staged
// through shared memory in tiles of 64 with coalesced loads in either workspace layout (lines
// adjacent in memory, or positions contiguous), padded against bank conflicts. Forward: each warp
// owns a set of the 2 kc + 1 kept bins and adds every tile's contribution, X[k][line] +=
// sum_n G[n][line] exp(-2 pi j k n / len), the twiddles rotated within the tile from an exactly
// reduced anchor exp(-2 pi j (k n0 mod len) / len). Inverse, after all tiles: G[n][line] =
// (1/len) sum_k X[k][line] exp(2 pi j k n / len), the twiddles again from exactly reduced anchors.
// The lines are rewritten in place. Work per pixel: 2 (2 kc + 1) complex multiply-adds and as
// many twiddle rotations.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

namespace {

constexpr int kCbThreads = 256;   // 8 warps; lane = line within the CTA's group of 32
constexpr int kCbTile = 64;       // positions per staged tile
constexpr int kCbPad = 33;        // tile row length (float2 / double2 units), 32 lines + 1

template <typename T>
__device__ __forceinline__ void sincospi_t(T x, T* s, T* c);
template <>
__device__ __forceinline__ void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }

// exp(sign 2 pi j m / len) for an integer m reduced into [0, len)
template <typename T>
__device__ __forceinline__ cx<T> twiddle(int64_t m, int len, T sign) {
    m %= len;
    if (m < 0) m += len;
    T s, c;
    sincospi_t<T>((T)(2 * m) / (T)len, &s, &c);
    return mkc(c, sign * s);
}

// element (line, pos) of frame F's cross lines in the workspace
__device__ __forceinline__ uint64_t cb_index(const FrameDev& F, int line, int pos) {
    const int y = F.carrier_axis == 0 ? pos : line;
    const int x = F.carrier_axis == 0 ? line : pos;
    return F.gam_off + (F.deriv_axis == 0 ? (uint64_t)y * F.W + x : (uint64_t)x * F.H + y);
}

template <typename T>
__global__ void __launch_bounds__(kCbThreads) crossband_kernel(const FrameDev* __restrict__ fr, int nframes,
                                                               cx<T>* __restrict__ gam) {
    extern __shared__ __align__(16) double cb_smem_d[];
    cx<T>* tile = reinterpret_cast<cx<T>*>(cb_smem_d);  // [kCbTile][kCbPad]
    cx<T>* X = tile + kCbTile * kCbPad;                  // [nbins][32]
    const int64_t group = blockIdx.x;
    const int f = find_frame(fr, nframes, group, [](const FrameDev& F) { return F.cross_start; });
    const FrameDev& F = fr[f];
    const int nlines = F.carrier_axis == 0 ? F.W : F.H;
    const int len = F.carrier_axis == 0 ? F.H : F.W;
    const int li0 = (int)(group - F.cross_start) * 32;
    const int kc = F.cross_kc, nbins = 2 * kc + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool lines_adjacent = (F.carrier_axis == 0) == (F.deriv_axis == 0);

    for (int i = threadIdx.x; i < nbins * 32; i += kCbThreads) X[i] = mkc((T)0, (T)0);

    // ---- forward over the tiles ------------------------------------------------------------------
    for (int n0 = 0; n0 < len; n0 += kCbTile) {
        const int tn = min(kCbTile, len - n0);
        __syncthreads();  // the previous tile has been consumed (and X initialised)
        for (int i = threadIdx.x; i < kCbTile * 32; i += kCbThreads) {
            int pos, ln;
            if (lines_adjacent) {
                pos = i >> 5;
                ln = i & 31;
            } else {
                ln = i / kCbTile;
                pos = i % kCbTile;
            }
            cx<T> v = mkc((T)0, (T)0);
            if (pos < tn && li0 + ln < nlines) v = gam[cb_index(F, li0 + ln, n0 + pos)];
            tile[pos * kCbPad + ln] = v;
        }
        __syncthreads();
        for (int b = warp; b < nbins; b += kCbThreads / 32) {
            const int k = b - kc;
            cx<T> w = twiddle<T>((int64_t)k * n0, len, (T)-1);  // exp(-2 pi j k n0 / len)
            const cx<T> step = twiddle<T>(k, len, (T)-1);
            cx<T> acc = mkc((T)0, (T)0);
            for (int p = 0; p < tn; ++p) {
                acc = acc + tile[p * kCbPad + lane] * w;
                w = w * step;
            }
            X[b * 32 + lane] = X[b * 32 + lane] + acc;
        }
    }
    __syncthreads();

    // ---- inverse, tile by tile, written back in place -------------------------------------------
    const T inv_len = (T)1 / (T)len;
    for (int n0 = 0; n0 < len; n0 += kCbTile) {
        const int tn = min(kCbTile, len - n0);
        for (int p = warp; p < tn; p += kCbThreads / 32) {
            const int n = n0 + p;
            cx<T> w = twiddle<T>(-(int64_t)kc * n, len, (T)1);  // exp(2 pi j (-kc) n / len)
            const cx<T> step = twiddle<T>(n, len, (T)1);
            cx<T> acc = mkc((T)0, (T)0);
            for (int b = 0; b < nbins; ++b) {
                acc = acc + X[b * 32 + lane] * w;
                w = w * step;
            }
            tile[p * kCbPad + lane] = inv_len * acc;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kCbTile * 32; i += kCbThreads) {
            int pos, ln;
            if (lines_adjacent) {
                pos = i >> 5;
                ln = i & 31;
            } else {
                ln = i / kCbTile;
                pos = i % kCbTile;
            }
            if (pos < tn && li0 + ln < nlines) gam[cb_index(F, li0 + ln, n0 + pos)] = tile[pos * kCbPad + ln];
        }
        __syncthreads();  // the tile is reused by the next inverse tile
    }
}

template <typename T>
size_t cb_smem_bytes(int max_bins) {
    return sizeof(cx<T>) * ((size_t)kCbTile * kCbPad + (size_t)max_bins * 32);
}

}  // namespace

cudaError_t init_crossband() {
    cudaError_t e = cudaFuncSetAttribute(crossband_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cb_smem_bytes<float>(2 * kMaxCrossKc + 1));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(crossband_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cb_smem_bytes<double>(2 * kMaxCrossKc + 1));
}

cudaError_t launch_crossband(const FrameDev* d_frames, int nframes, int64_t total_groups, int max_kc,
                             void* d_gamma, bool fp64, cudaStream_t stream) {
    if (total_groups <= 0) return cudaSuccess;
    if (fp64)
        crossband_kernel<double><<<(unsigned)total_groups, kCbThreads, cb_smem_bytes<double>(2 * max_kc + 1), stream>>>(
            d_frames, nframes, static_cast<cx<double>*>(d_gamma));
    else
        crossband_kernel<float><<<(unsigned)total_groups, kCbThreads, cb_smem_bytes<float>(2 * max_kc + 1), stream>>>(
            d_frames, nframes, static_cast<cx<float>*>(d_gamma));
    return cudaGetLastError();
}

}  // namespace rmusic
