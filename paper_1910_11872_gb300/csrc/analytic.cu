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
// steps. All sincos values come from sincospif on arguments in [0, 2). Work per pixel is
// about 4 nb FMAs each way (nb ~ 100 at len = 1024, f0 = 0.1): a few percent of the solver.
#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

constexpr int kA1Threads = 256;
constexpr int kA1Block = 32;  // forward Horner re-anchoring period

__global__ void __launch_bounds__(kA1Threads)
analytic_kernel(const FrameDev* __restrict__ fr, int nframes, const unsigned char* __restrict__ in,
                float2* __restrict__ gam) {
    extern __shared__ float a1_smem[];
    __shared__ float red[kA1Threads / 32];
    const int64_t line = blockIdx.x;
    const int f = find_frame(fr, nframes, line, [](const FrameDev& F) { return F.line_start; });
    const FrameDev& F = fr[f];
    const int li = (int)(line - F.line_start);
    const int len = F.len;
    float* v = a1_smem;
    float2* X = reinterpret_cast<float2*>(a1_smem + ((len + 1) & ~1));

    // load the line and its sum
    float s = 0.f;
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
        uint64_t idx = F.carrier_axis == 0 ? (uint64_t)li * F.pitch + n : (uint64_t)n * F.pitch + li;
        float val;
        if (F.dtype == 0)
            val = reinterpret_cast<const float*>(in + F.in_off)[idx];
        else
            val = (float)reinterpret_cast<const uint16_t*>(in + F.in_off)[idx];
        v[n] = val;
        s += val;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    float tot = 0.f;
#pragma unroll
    for (int w = 0; w < kA1Threads / 32; ++w) tot += red[w];
    const float mean = tot / (float)len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) v[n] -= mean;
    __syncthreads();

    // forward band-limited DFT, one thread per kept bin
    const float two_over_len = 2.f / (float)len;
    for (int b = threadIdx.x; b < F.nb; b += blockDim.x) {
        const int k = F.k_lo + b;
        float sk, ck;
        sincospif((float)k * two_over_len, &sk, &ck);  // xi = ck - j sk
        float xr = 0.f, xi = 0.f;
        const int nblk = (len + kA1Block - 1) / kA1Block;
        for (int blk = nblk - 1; blk >= 0; --blk) {
            const int n0 = blk * kA1Block;
            const int n1 = min(len, n0 + kA1Block);
            float pr = 0.f, pi = 0.f;  // sum_{i} v[n0 + i] xi^i by Horner
            for (int n = n1 - 1; n >= n0; --n) {
                float nr = fmaf(pr, ck, fmaf(pi, sk, v[n]));
                float ni = fmaf(pi, ck, -pr * sk);
                pr = nr;
                pi = ni;
            }
            // X += xi^{n0} * partial, with xi^{n0} from the exactly reduced index k n0 mod len
            const int m = (int)(((int64_t)k * n0) % len);
            float sm, cm;
            sincospif((float)m * two_over_len, &sm, &cm);  // xi^{n0} = cm - j sm
            xr += pr * cm + pi * sm;
            xi += pi * cm - pr * sm;
        }
        X[b] = make_float2(xr, xi);
    }
    __syncthreads();

    // inverse over the band, one thread per sample, stored window-line major
    const float inv_len = 1.f / (float)len;
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
        float sn, cn;
        sincospif((float)n * two_over_len, &sn, &cn);  // zeta = cn + j sn
        float ar = 0.f, ai = 0.f;
        for (int b = F.nb - 1; b >= 0; --b) {
            const float2 x = X[b];
            float nr = fmaf(ar, cn, fmaf(-ai, sn, x.x));
            float ni = fmaf(ar, sn, fmaf(ai, cn, x.y));
            ar = nr;
            ai = ni;
        }
        const int m = (int)(((int64_t)F.k_lo * n) % len);
        float s2, c2;
        sincospif((float)m * two_over_len, &s2, &c2);
        const float gr = (ar * c2 - ai * s2) * inv_len;
        const float gi = (ar * s2 + ai * c2) * inv_len;
        const int y = F.carrier_axis == 0 ? li : n;
        const int x = F.carrier_axis == 0 ? n : li;
        const int wline = F.deriv_axis == 0 ? y : x;
        const int pos = F.deriv_axis == 0 ? x : y;
        gam[F.gam_off + (uint64_t)wline * F.wlen + pos] = make_float2(gr, gi);
    }
}

cudaError_t init_analytic() {
    return cudaFuncSetAttribute(analytic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * kMaxLine + sizeof(float2) * (kMaxLine / 2 + 1)));
}

cudaError_t launch_analytic(const FrameDev* d_frames, int nframes, int64_t total_lines, int max_len,
                            const void* d_in, float2* d_gamma, cudaStream_t stream) {
    if (total_lines <= 0) return cudaSuccess;
    // v[len] floats + X[nb <= len/2] float2
    size_t smem = sizeof(float) * (size_t)((max_len + 1) & ~1) + sizeof(float2) * (size_t)(max_len / 2 + 1);
    analytic_kernel<<<(unsigned)total_lines, kA1Threads, smem, stream>>>(
        d_frames, nframes, static_cast<const unsigned char*>(d_in), d_gamma);
    return cudaGetLastError();
}

}  // namespace rmusic
