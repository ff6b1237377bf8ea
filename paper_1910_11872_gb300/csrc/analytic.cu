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

template <typename T>
static size_t a1_smem_bytes(int len) {
    // the band-limited DFT: v[len] (padded to 4 elements) + X[nb <= len/2];
    // the FFT: a[len] + the twiddle table tw[len/2] (complex)
    const size_t dft = sizeof(T) * (size_t)((len + 3) & ~3) + 2 * sizeof(T) * (size_t)(len / 2 + 1);
    const size_t fft = 2 * sizeof(T) * ((size_t)len + (size_t)(len / 2));
    return dft > fft ? dft : fft;
}

cudaError_t init_analytic() {
    cudaError_t e = cudaFuncSetAttribute(analytic_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)a1_smem_bytes<float>(kMaxLine));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(analytic_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)a1_smem_bytes<double>(kMaxLine));
}

cudaError_t launch_analytic(const FrameDev* d_frames, int nframes, int64_t total_lines, int max_len,
                            const void* d_in, void* d_gamma, bool fp64, cudaStream_t stream) {
    if (total_lines <= 0) return cudaSuccess;
    const unsigned char* in = static_cast<const unsigned char*>(d_in);
    if (fp64)
        analytic_kernel<double><<<(unsigned)total_lines, kA1Threads, a1_smem_bytes<double>(max_len), stream>>>(
            d_frames, nframes, in, static_cast<cx<double>*>(d_gamma));
    else
        analytic_kernel<float><<<(unsigned)total_lines, kA1Threads, a1_smem_bytes<float>(max_len), stream>>>(
            d_frames, nframes, in, static_cast<cx<float>*>(d_gamma));
    return cudaGetLastError();
}

}  // namespace rmusic
