// analytic.cu -- analytic signal of every carrier line of every frame (Sec. 2, Eq. 1:
// "bandpass filtering and carrier removal" turn the real fringe a + b cos(2 pi f0 t + phi)
// into Gamma = A exp(j phi) + eta).
//
// One CTA per carrier line. The line is read once from HBM (float32 or uint16), its mean is
// removed (DC is outside the band anyway; removing it first keeps the FP32 sums small), and the
// kept one-sided band k_lo .. k_lo + nb - 1 (1 <= k < len/2, |k/len - f0| < B) is computed by a
// band-limited DFT. Only nb ~ f0 * len bins are needed, so the forward transform is nb Horner
// sums of length len and the inverse is one Horner sum of length nb per sample:
//   X[k]   = sum_n v[n] xi_k^n,                 xi_k = exp(-2 pi j k / len)
//   G[n]   = (1/len) exp(2 pi j k_lo n / len) sum_i X[k_lo + i] zeta_n^i,  zeta_n = exp(2 pi j n / len)
// The forward sums are re-anchored every 32 samples with an exactly reduced twiddle
// exp(-2 pi j (k * n0 mod len) / len), so rounding in xi_k never compounds over more than 32
// steps. All sincos values come from sincospi on arguments in [0, 2). Work per pixel is
// about 4 nb FMAs each way (nb ~ 100 at len = 1024, f0 = 0.1): a few percent of the solver.
// Lines whose length is a power of two take the same band through a radix-2 FFT in shared
// memory instead (forward transform of the mean-free line, the band kept, inverse transform):
// about 10 log2(len) flops per sample instead of ~8 nb, with twiddles exp(-2 pi j k / len) from
// sincospi of exact fractions, tabulated once per line.
// T = float feeds the FP32 paths (complex64 output); T = double feeds the plain FP64 path
// (complex128 output), so that path is double precision end to end. Complex64 frames are the
// analytic signal already and are only copied into the workspace layout.
#include <math.h>

#include <algorithm>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

constexpr int kA1Threads = 128;
constexpr int kA1Block = 32;  // forward Horner re-anchoring period

template <typename T>
__device__ __forceinline__ void sincospi_t(T x, T* s, T* c);
template <>
__device__ __forceinline__ void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }

// p <- sum_i v[n0 + i] xi^i over n0 <= n < n1 by Horner (xi = ck - j sk), highest index first.
template <typename T>
__device__ __forceinline__ void horner_fwd(const T* v, int n0, int n1, T ck, T sk, T& pr, T& pi) {
    for (int n = n1 - 1; n >= n0; --n) {
        T nr = fma_t<T>(pr, ck, fma_t<T>(pi, sk, v[n]));
        T ni = fma_t<T>(pi, ck, -pr * sk);
        pr = nr;
        pi = ni;
    }
}
// FP32: four samples per 16-byte shared-memory read (n0 is a multiple of 4).
template <>
__device__ __forceinline__ void horner_fwd<float>(const float* v, int n0, int n1, float ck, float sk, float& pr,
                                                  float& pi) {
    const int rem = (n1 - n0) & 3;
    for (int n = n1 - 1; n >= n1 - rem; --n) {
        float nr = fmaf(pr, ck, fmaf(pi, sk, v[n]));
        float ni = fmaf(pi, ck, -pr * sk);
        pr = nr;
        pi = ni;
    }
    for (int n = n1 - rem - 4; n >= n0; n -= 4) {
        const float4 q = *reinterpret_cast<const float4*>(v + n);
        const float vv[4] = {q.w, q.z, q.y, q.x};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float nr = fmaf(pr, ck, fmaf(pi, sk, vv[t]));
            float ni = fmaf(pi, ck, -pr * sk);
            pr = nr;
            pi = ni;
        }
    }
}

// a <- sum_b X[b] zeta^b by Horner (zeta = cn + j sn), highest bin first.
template <typename T>
__device__ __forceinline__ void horner_inv(const cx<T>* X, int nb, T cn, T sn, T& ar, T& ai) {
    for (int b = nb - 1; b >= 0; --b) {
        const cx<T> x = X[b];
        T nr = fma_t<T>(ar, cn, fma_t<T>(-ai, sn, x.r));
        T ni = fma_t<T>(ar, sn, fma_t<T>(ai, cn, x.i));
        ar = nr;
        ai = ni;
    }
}
// FP32: two bins per 16-byte shared-memory read (X is 16-byte aligned).
template <>
__device__ __forceinline__ void horner_inv<float>(const cx<float>* X, int nb, float cn, float sn, float& ar,
                                                  float& ai) {
    int b = nb - 1;
    if (nb & 1) {
        const cx<float> x = X[b];
        float nr = fmaf(ar, cn, fmaf(-ai, sn, x.r));
        float ni = fmaf(ar, sn, fmaf(ai, cn, x.i));
        ar = nr;
        ai = ni;
        --b;
    }
    for (; b >= 1; b -= 2) {
        const float4 q = *reinterpret_cast<const float4*>(X + (b - 1));  // X[b-1], X[b]
        float nr = fmaf(ar, cn, fmaf(-ai, sn, q.z));
        float ni = fmaf(ar, sn, fmaf(ai, cn, q.w));
        ar = fmaf(nr, cn, fmaf(-ni, sn, q.x));
        ai = fmaf(nr, sn, fmaf(ni, cn, q.y));
    }
}

template <typename T>
__device__ __forceinline__ T frame_sample(const FrameDev& F, const unsigned char* __restrict__ in, uint64_t idx) {
    if (F.dtype == kDtF32) return (T)reinterpret_cast<const float*>(in + F.in_off)[idx];
    return (T)reinterpret_cast<const uint16_t*>(in + F.in_off)[idx];
}

// In-place iterative radix-2 transform of a[0 .. len) (bit-reversed input, natural-order output)
// with the table tw[k] = exp(-2 pi j k / len), k < len / 2; conj_tw selects the inverse kernel.
template <typename T>
__device__ __forceinline__ void fft_stages(cx<T>* a, const cx<T>* tw, int len, int logn, bool conj_tw) {
    for (int st = 1; st <= logn; ++st) {
        const int half = 1 << (st - 1);
        const int shift = logn - st;  // twiddle index = pos << shift
        for (int b = threadIdx.x; b < (len >> 1); b += blockDim.x) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> (st - 1)) << st) + pos, i1 = i0 + half;
            cx<T> w = tw[pos << shift];
            if (conj_tw) w.i = -w.i;
            const cx<T> u = a[i0], v = a[i1] * w;
            a[i0] = u + v;
            a[i1] = u - v;
        }
        __syncthreads();
    }
}

// Band-pass of one power-of-two line through the FFT (see the file comment).
template <typename T>
__device__ void analytic_line_fft(const FrameDev& F, int li, const unsigned char* __restrict__ in,
                                  cx<T>* __restrict__ gam, cx<T>* a, T* red) {
    const int len = F.len;
    const int logn = __ffs(len) - 1;
    cx<T>* tw = a + len;
    T s = 0;
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
        const uint64_t idx = F.carrier_axis == 0 ? (uint64_t)li * F.pitch + n : (uint64_t)n * F.pitch + li;
        const T val = frame_sample<T>(F, in, idx);
        a[__brev((unsigned)n) >> (32 - logn)] = mkc(val, (T)0);
        s += val;
    }
    const T two_over_len = T(2) / (T)len;
    for (int k = threadIdx.x; k < (len >> 1); k += blockDim.x) {
        T sk, ck;
        sincospi_t<T>((T)k * two_over_len, &sk, &ck);
        tw[k] = mkc(ck, -sk);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    T tot = 0;
#pragma unroll
    for (int w = 0; w < kA1Threads / 32; ++w) tot += red[w];
    const T mean = tot / (T)len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) a[n].r -= mean;
    __syncthreads();
    fft_stages<T>(a, tw, len, logn, false);
    // keep the band k_lo .. k_lo + nb - 1, and put the spectrum back into bit-reversed order
    for (int k = threadIdx.x; k < len; k += blockDim.x)
        if (k < F.k_lo || k >= F.k_lo + F.nb) a[k] = mkc((T)0, (T)0);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int j = __brev((unsigned)i) >> (32 - logn);
        if (i < j) {
            const cx<T> t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    __syncthreads();
    fft_stages<T>(a, tw, len, logn, true);
    const T inv_len = T(1) / (T)len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
        const int y = F.carrier_axis == 0 ? li : n;
        const int x = F.carrier_axis == 0 ? n : li;
        const int wline = F.deriv_axis == 0 ? y : x;
        const int pos = F.deriv_axis == 0 ? x : y;
        gam[F.gam_off + (uint64_t)wline * F.wlen + pos] = inv_len * a[n];
    }
}

// ---- warp-FFT band-pass: lines of len = 32 R samples (R = 8, 16, 32) along rows ------------------
// A warp takes G = 32 / R adjacent carrier lines (rows; the windows may run along them or across
// them, in which case the samples are stored column-major). With
// n = 32 a + l and k = b + R m (a, b < R; l, m < 32) the forward transform factors as
//   X[b + R m] = sum_l W32^(l m) W_len^(l b) sum_a x[32 a + l] W_R^(a b),
// so lane l first takes the R-point DFTs over a of its column (registers), the result is twiddled by
// W_len^(l b) and transposed through shared memory, and lane t = g R + b takes the 32-point DFT over
// l of line g's column b. The band k_lo <= k < k_lo + nb is kept and the inverse runs the same
// factorisation backwards (32-point inverse over m per lane, twiddle W_len^(-b l), transpose, R-point
// inverse over b per lane), which leaves lane l with samples l + 32 a: the loads and stores are
// coalesced rows and no __syncthreads is needed. The forward transforms are decimation in frequency
// (natural order in, bit-reversed out), the inverse ones decimation in time (bit-reversed in), so no
// reordering pass is needed. Twiddles: W32^e from cos(pi e / 16) constants, W_len^j from a table of
// exp(-2 pi j k / 1024) computed in double on the host.
constexpr int kFastTile = 32 * 33;  // float2 per warp: a 32 x 32 transpose tile with a padded row
constexpr size_t kFastSmem = (kA1Threads / 32) * kFastTile * sizeof(float2);
__device__ float2 g_tw1024[1024];  // exp(-2 pi j k / 1024)

// cos(pi e / 16) for an integer e >= -16 (a constant when e is)
__device__ __forceinline__ float cos_pi16(int e) {
    e &= 31;
    if (e > 16) e = 32 - e;
    const float t[17] = {1.0f,
                         0.98078528040323044913f,
                         0.92387953251128675613f,
                         0.83146961230254523708f,
                         0.70710678118654752440f,
                         0.55557023301960222474f,
                         0.38268343236508977173f,
                         0.19509032201612826785f,
                         0.0f,
                         -0.19509032201612826785f,
                         -0.38268343236508977173f,
                         -0.55557023301960222474f,
                         -0.70710678118654752440f,
                         -0.83146961230254523708f,
                         -0.92387953251128675613f,
                         -0.98078528040323044913f,
                         -1.0f};
    return t[e];
}

// d W32^e (forward) or d W32^-e (INV), W32 = exp(-2 pi j / 32), 0 <= e < 16
template <bool INV>
__device__ __forceinline__ cx<float> tw32(cx<float> d, int e) {
    if (e == 0) return d;
    if (e == 8) return INV ? mkc(-d.i, d.r) : mkc(d.i, -d.r);
    const float c = cos_pi16(e), s = cos_pi16(8 - e);  // cos and sin of pi e / 16
    return INV ? mkc(d.r * c - d.i * s, d.r * s + d.i * c) : mkc(d.r * c + d.i * s, d.i * c - d.r * s);
}

__host__ __device__ constexpr int brev_bits(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}
__host__ __device__ constexpr int log2_int(int x) { return x <= 1 ? 0 : 1 + log2_int(x >> 1); }

// Radix-2 decimation in frequency on v[o .. o + R): natural order in, bin k at o + brev(k).
template <int R, bool INV>
__device__ __forceinline__ void dif_block(cx<float> (&v)[32], int o) {
#pragma unroll
    for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * half) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const cx<float> a = v[o + g + j], b = v[o + g + j + half];
                v[o + g + j] = a + b;
                v[o + g + j + half] = tw32<INV>(a - b, j * (16 / half));
            }
        }
    }
}

// Radix-2 decimation in time on v[o .. o + R): bin k at o + brev(k) in, natural order out.
template <int R, bool INV>
__device__ __forceinline__ void dit_block(cx<float> (&v)[32], int o) {
#pragma unroll
    for (int half = 1; half < R; half <<= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * half) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const cx<float> a = v[o + g + j], b = tw32<INV>(v[o + g + j + half], j * (16 / half));
                v[o + g + j] = a + b;
                v[o + g + j + half] = a - b;
            }
        }
    }
}

// One warp's group of G = 32 / R lines starting at line0 (nvalid of them inside the frame).
template <int R>
__device__ void analytic_group_fft(const FrameDev& F, int line0, int nvalid, const unsigned char* __restrict__ in,
                                   cx<float>* __restrict__ gam, float2* tile) {
    constexpr int G = 32 / R;
    constexpr int LR = log2_int(R);
    constexpr int len = 32 * R;
    const int lane = threadIdx.x & 31;
    cx<float> v[32];
    // load (coalesced rows) and remove each line's mean
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const bool ok = g < nvalid;
        const uint64_t row = (uint64_t)(line0 + g) * (uint64_t)F.pitch;
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const float x = ok ? frame_sample<float>(F, in, row + 32 * a + lane) : 0.f;
            v[g * R + a] = mkc(x, 0.f);
            s += x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float mean = s * (1.f / (float)len);
#pragma unroll
        for (int a = 0; a < R; ++a) v[g * R + a].r -= mean;
    }
    // R-point DFTs over a, twiddle W_len^(l b), transpose: row g R + b, column l
#pragma unroll
    for (int g = 0; g < G; ++g) {
        dif_block<R, false>(v, g * R);
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const float2 w = g_tw1024[lane * b * (1024 / len)];
            const cx<float> y = v[g * R + brev_bits(b, LR)] * mkc(w.x, w.y);
            tile[(g * R + b) * 33 + lane] = make_float2(y.r, y.i);
        }
    }
    __syncwarp();
    // lane t = g R + b: 32-point DFT over l, the band, 32-point inverse over m
    const int t = lane, b = t % R;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
        const float2 z = tile[t * 33 + l];
        v[l] = mkc(z.x, z.y);
    }
    dif_block<32, false>(v, 0);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int k = b + R * m;
        if (k < F.k_lo || k >= F.k_lo + F.nb) v[brev_bits(m, 5)] = mkc(0.f, 0.f);
    }
    dit_block<32, true>(v, 0);
    __syncwarp();  // every lane has read its tile row
#pragma unroll
    for (int l = 0; l < 32; ++l) {
        const float2 w = g_tw1024[b * l * (1024 / len)];
        const cx<float> y = v[l] * mkc(w.x, -w.y);
        tile[t * 33 + l] = make_float2(y.r, y.i);
    }
    __syncwarp();
    // lane l: R-point inverse over b for each line, samples l + 32 a
    const float inv_len = 1.f / (float)len;
#pragma unroll
    for (int g = 0; g < G; ++g) {
#pragma unroll
        for (int bb = 0; bb < R; ++bb) {
            const float2 z = tile[(g * R + bb) * 33 + lane];
            v[g * R + bb] = mkc(z.x, z.y);
        }
        dif_block<R, true>(v, g * R);
        if (g < nvalid) {
            if (F.deriv_axis == 0) {
                // windows along the line: the workspace row is the line (coalesced stores)
                cx<float>* out = gam + F.gam_off + (uint64_t)(line0 + g) * (uint64_t)F.wlen;
#pragma unroll
                for (int a = 0; a < R; ++a) out[32 * a + lane] = inv_len * v[g * R + brev_bits(a, LR)];
            } else {
                // windows across the lines (columns): sample x of line y goes to x wlen + y; the
                // CTA's 4 G consecutive lines fill each column's 32-byte sectors in L2
                cx<float>* out = gam + F.gam_off + (uint64_t)(line0 + g);
#pragma unroll
                for (int a = 0; a < R; ++a)
                    out[(uint64_t)(32 * a + lane) * (uint64_t)F.wlen] = inv_len * v[g * R + brev_bits(a, LR)];
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kA1Threads)
analytic_kernel(const FrameDev* __restrict__ fr, int nframes, const unsigned char* __restrict__ in,
                cx<T>* __restrict__ gam) {
    extern __shared__ __align__(16) double a1_smem_d[];
    T* a1_smem = reinterpret_cast<T*>(a1_smem_d);
    __shared__ T red[kA1Threads / 32];
    const int64_t line = blockIdx.x;
    const int f = find_frame(fr, nframes, line, [](const FrameDev& F) { return F.line_start; });
    const FrameDev& F = fr[f];
    const int li = (int)(line - F.line_start);
    if (F.band_r) return;  // taken by analytic_fast_kernel
    const int len = F.len;
    T* v = a1_smem;
    cx<T>* X = reinterpret_cast<cx<T>*>(a1_smem + ((len + 3) & ~3));

    if (F.dtype == kDtC64) {
        // a complex frame is the analytic signal already (the complex fringe the paper simulates
        // in Sec. 4): copied into the workspace layout without a band-pass
        const float2* src = reinterpret_cast<const float2*>(in + F.in_off);
        for (int n = threadIdx.x; n < len; n += blockDim.x) {
            const uint64_t idx = F.carrier_axis == 0 ? (uint64_t)li * F.pitch + n : (uint64_t)n * F.pitch + li;
            const float2 g = src[idx];
            const int y = F.carrier_axis == 0 ? li : n;
            const int x = F.carrier_axis == 0 ? n : li;
            const int wline = F.deriv_axis == 0 ? y : x;
            const int pos = F.deriv_axis == 0 ? x : y;
            gam[F.gam_off + (uint64_t)wline * F.wlen + pos] = mkc((T)g.x, (T)g.y);
        }
        return;
    }
    if (!F.raw && len >= 2 && (len & (len - 1)) == 0) {
        analytic_line_fft<T>(F, li, in, gam, reinterpret_cast<cx<T>*>(a1_smem_d), red);
        return;
    }

    // load the line and its sum
    T s = 0;
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
        uint64_t idx = F.carrier_axis == 0 ? (uint64_t)li * F.pitch + n : (uint64_t)n * F.pitch + li;
        T val;
        if (F.dtype == kDtF32)
            val = (T)reinterpret_cast<const float*>(in + F.in_off)[idx];
        else
            val = (T)reinterpret_cast<const uint16_t*>(in + F.in_off)[idx];
        v[n] = val;
        s += val;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    T tot = 0;
#pragma unroll
    for (int w = 0; w < kA1Threads / 32; ++w) tot += red[w];
    const T mean = tot / (T)len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) v[n] -= mean;
    __syncthreads();

    if (F.raw) {
        // no band-pass (model orders p > 1 on real fringes): the line minus its mean, as is
        for (int n = threadIdx.x; n < len; n += blockDim.x) {
            const int y = F.carrier_axis == 0 ? li : n;
            const int x = F.carrier_axis == 0 ? n : li;
            const int wline = F.deriv_axis == 0 ? y : x;
            const int pos = F.deriv_axis == 0 ? x : y;
            gam[F.gam_off + (uint64_t)wline * F.wlen + pos] = mkc(v[n], (T)0);
        }
        return;
    }

    // forward band-limited DFT, one thread per kept bin
    const T two_over_len = T(2) / (T)len;
    for (int b = threadIdx.x; b < F.nb; b += blockDim.x) {
        const int k = F.k_lo + b;
        T sk, ck;
        sincospi_t<T>((T)k * two_over_len, &sk, &ck);  // xi = ck - j sk
        T xr = 0, xi = 0;
        const int nblk = (len + kA1Block - 1) / kA1Block;
        for (int blk = nblk - 1; blk >= 0; --blk) {
            const int n0 = blk * kA1Block;
            const int n1 = min(len, n0 + kA1Block);
            T pr = 0, pi = 0;  // sum_{i} v[n0 + i] xi^i by Horner
            horner_fwd<T>(v, n0, n1, ck, sk, pr, pi);
            // X += xi^{n0} * partial, with xi^{n0} from the exactly reduced index k n0 mod len
            const int m = (int)(((int64_t)k * n0) % len);
            T sm, cm;
            sincospi_t<T>((T)m * two_over_len, &sm, &cm);  // xi^{n0} = cm - j sm
            xr += pr * cm + pi * sm;
            xi += pi * cm - pr * sm;
        }
        X[b] = mkc(xr, xi);
    }
    __syncthreads();

    // inverse over the band, one thread per sample, stored window-line major
    const T inv_len = T(1) / (T)len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
        T sn, cn;
        sincospi_t<T>((T)n * two_over_len, &sn, &cn);  // zeta = cn + j sn
        T ar = 0, ai = 0;
        horner_inv<T>(X, F.nb, cn, sn, ar, ai);
        const int m = (int)(((int64_t)F.k_lo * n) % len);
        T s2, c2;
        sincospi_t<T>((T)m * two_over_len, &s2, &c2);
        const T gr = (ar * c2 - ai * s2) * inv_len;
        const T gi = (ar * s2 + ai * c2) * inv_len;
        const int y = F.carrier_axis == 0 ? li : n;
        const int x = F.carrier_axis == 0 ? n : li;
        const int wline = F.deriv_axis == 0 ? y : x;
        const int pos = F.deriv_axis == 0 ? x : y;
        gam[F.gam_off + (uint64_t)wline * F.wlen + pos] = mkc(gr, gi);
    }
}

// The warp-FFT schedule (frames with band_r != 0): each CTA's 4 warps take 4 groups of 32 / R lines.
// A kernel of its own, so that its register budget (the 32-sample transforms in registers) does not
// lower the occupancy of the per-line schedule.
__global__ void __launch_bounds__(kA1Threads, 4)
analytic_fast_kernel(const FrameDev* __restrict__ fr, int nframes, const unsigned char* __restrict__ in,
                     cx<float>* __restrict__ gam) {
    extern __shared__ __align__(16) float2 a1_fast_smem[];
    const int64_t cta = blockIdx.x;
    const int f = find_frame(fr, nframes, cta, [](const FrameDev& F) { return F.line_start; });
    const FrameDev& F = fr[f];
    if (!F.band_r) return;  // taken by analytic_kernel
    const int G = 32 / F.band_r;
    const int line0 = ((int)(cta - F.line_start) * (kA1Threads / 32) + (int)(threadIdx.x >> 5)) * G;
    const int nvalid = min(G, F.nlines - line0);
    if (nvalid <= 0) return;
    float2* tile = a1_fast_smem + (threadIdx.x >> 5) * kFastTile;
    if (F.band_r == 32)
        analytic_group_fft<32>(F, line0, nvalid, in, gam, tile);
    else if (F.band_r == 16)
        analytic_group_fft<16>(F, line0, nvalid, in, gam, tile);
    else
        analytic_group_fft<8>(F, line0, nvalid, in, gam, tile);
}

template <typename T>
static size_t a1_smem_bytes(int len) {
    // the band-limited DFT: v[len] (padded to 4 elements) + X[nb <= len/2];
    // the FFT: a[len] + the twiddle table tw[len/2] (complex)
    const size_t dft = sizeof(T) * (size_t)((len + 3) & ~3) + 2 * sizeof(T) * (size_t)(len / 2 + 1);
    const size_t fft = 2 * sizeof(T) * ((size_t)len + (size_t)(len / 2));
    return dft > fft ? dft : fft;
}

int64_t band_assign(FrameDev* F, bool fp64) {
    F->band_r = 0;
    // carrier lines are rows (coalesced loads); the windows run along them or across them
    const bool rows = F->carrier_axis == 0;
    if (!fp64 && !F->raw && F->dtype != kDtC64 && rows && (F->len == 256 || F->len == 512 || F->len == 1024))
        F->band_r = F->len / 32;
    if (!F->band_r) return F->nlines;
    const int per_cta = (kA1Threads / 32) * (32 / F->band_r);
    return (F->nlines + per_cta - 1) / per_cta;
}

cudaError_t init_analytic() {
    // exp(-2 pi j k / 1024) in double, rounded once
    float2 tw[1024];
    for (int k = 0; k < 1024; ++k) {
        const double a = 6.283185307179586476925 * (double)k / 1024.0;
        tw[k] = make_float2((float)cos(a), (float)-sin(a));
    }
    cudaError_t e = cudaMemcpyToSymbol(g_tw1024, tw, sizeof(tw));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(analytic_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFastSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(analytic_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)a1_smem_bytes<float>(kMaxLine));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(analytic_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)a1_smem_bytes<double>(kMaxLine));
}

cudaError_t launch_analytic(const FrameDev* d_frames, int nframes, int64_t total_lines, int max_len, int schedules,
                            const void* d_in, void* d_gamma, bool fp64, cudaStream_t stream) {
    if (total_lines <= 0) return cudaSuccess;
    const unsigned char* in = static_cast<const unsigned char*>(d_in);
    if (fp64)
        analytic_kernel<double><<<(unsigned)total_lines, kA1Threads, a1_smem_bytes<double>(max_len), stream>>>(
            d_frames, nframes, in, static_cast<cx<double>*>(d_gamma));
    else {
        if (schedules & kBandPerLine)
            analytic_kernel<float><<<(unsigned)total_lines, kA1Threads, a1_smem_bytes<float>(max_len), stream>>>(
                d_frames, nframes, in, static_cast<cx<float>*>(d_gamma));
        if ((schedules & kBandWarpFft) && cudaPeekAtLastError() == cudaSuccess)
            analytic_fast_kernel<<<(unsigned)total_lines, kA1Threads, kFastSmem, stream>>>(
                d_frames, nframes, in, static_cast<cx<float>*>(d_gamma));
    }
    return cudaGetLastError();
}

}  // namespace rmusic
