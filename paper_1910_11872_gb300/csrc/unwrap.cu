// unwrap.cu -- phase assembly (Sec. 3: the local phases alpha are followed by an unwrapping
// operation, the reliability-sorting method of Herraez et al. 2002 that the paper cites).
//
// The method takes the edges between neighbouring pixels from the most reliable down and joins
// the two groups an edge connects, shifting one by the multiple of 2 pi that makes its endpoints
// differ by their wrapped difference. That order is Kruskal's algorithm for the maximum spanning
// forest of the pixel grid weighted by edge reliability, and the result is the 2 pi jumps
// integrated along that forest: it depends on the forest only, not on the order in which its
// edges are found. The GPU builds the same forest with Boruvka's algorithm, whose rounds are
// data parallel:
//   reliability  per pixel, R = 1 / D from the wrapped second differences (0 where a neighbour
//                is missing), computed with explicitly rounded float32 operations so that every
//                comparison below sees exactly the values of the sequential method;
//   per round    every component finds its most reliable outgoing edge (64-bit atomicMax on
//                (reliability bits, ~edge index): reliability first, then the smaller index),
//                hooks onto the component across it (of two components that chose the same edge
//                the smaller label stays the root) with the integer shift that makes the edge's
//                endpoints differ by their wrapped difference, the hooks are resolved to roots
//                by pointer jumping in place (shifts summed along the way; parent and shift share
//                one 64-bit word, so a jump always reads a consistent pair), and every pixel is
//                relabelled. Four launches per round; a round with nothing left to join makes
//                the later rounds return at once.
//                Each round at least halves the components, so ceil(log2(pixels)) rounds finish.
//   anchor       each connected region keeps its first pixel (row-major) at its wrapped value;
//                every component carries its smallest pixel index through the merges.
// All integer bookkeeping is exact; the output is phi + 2 pi k in float32.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

namespace {

constexpr int kUwThreads = 256;
constexpr float kPiF = 3.14159265358979f;
constexpr float kTwoPiF = 6.28318530717959f;

__device__ __forceinline__ float gam_f(float x) {
    if (x > kPiF) return __fsub_rn(x, kTwoPiF);
    if (x <= -kPiF) return __fadd_rn(x, kTwoPiF);
    return x;
}

// integer jump k_q - k_p across the edge p -> q of a wrapped map
__device__ __forceinline__ int jump(float pp, float pq) {
    const float d = __fsub_rn(pq, pp);
    return d > kPiF ? -1 : (d <= -kPiF ? 1 : 0);
}

struct UwArgs {
    const FrameDev* fr;
    int nframes;
    int64_t npx;
    const float* in;    // map of frame f at in + F.out_off + in_maps * H * W
    int64_t in_maps;
    float* out;         // map of frame f at out + F.out_off + out_maps * H * W
    int64_t out_maps;
};

__device__ __forceinline__ const FrameDev& frame_of(const UwArgs& a, int64_t g, int* fidx) {
    const int f = find_frame(a.fr, a.nframes, g, [](const FrameDev& F) { return (int64_t)F.gam_off; });
    *fidx = f;
    return a.fr[f];
}

// wph[g] = wrapped phase, fid[g] = frame, comp[g] = g, kk[g] = 0, minpix[g] = g
__global__ void __launch_bounds__(kUwThreads) uw_init(UwArgs a, float* __restrict__ wph, int32_t* __restrict__ fid,
                                                     int32_t* __restrict__ comp, int32_t* __restrict__ kk,
                                                     int32_t* __restrict__ minpix) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.npx; g += (int64_t)gridDim.x * blockDim.x) {
        int f;
        const FrameDev& F = frame_of(a, g, &f);
        const int64_t local = g - (int64_t)F.gam_off;
        wph[g] = a.in[F.out_off + a.in_maps * (int64_t)F.H * F.W + local];
        fid[g] = f;
        comp[g] = (int32_t)g;
        kk[g] = 0;
        minpix[g] = (int32_t)g;
    }
}

__global__ void __launch_bounds__(kUwThreads) uw_reliability(UwArgs a, const float* __restrict__ wph,
                                                            const int32_t* __restrict__ fid, float* __restrict__ rel) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.npx; g += (int64_t)gridDim.x * blockDim.x) {
        const FrameDev& F = a.fr[fid[g]];
        const int64_t local = g - (int64_t)F.gam_off;
        const int i = (int)(local / F.W), j = (int)(local % F.W), W = F.W;
        const float c = wph[g];
        if (isnan(c)) {
            rel[g] = c;
            continue;
        }
        bool inner = i >= 1 && i + 1 < F.H && j >= 1 && j + 1 < W;
        if (inner) {
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj)
                    if (isnan(wph[g + (int64_t)di * W + dj])) inner = false;
        }
        if (!inner) {
            rel[g] = 0.f;
            continue;
        }
        auto ph = [&](int di, int dj) { return wph[g + (int64_t)di * W + dj]; };
        const float h = __fsub_rn(gam_f(__fsub_rn(ph(0, -1), c)), gam_f(__fsub_rn(c, ph(0, 1))));
        const float v = __fsub_rn(gam_f(__fsub_rn(ph(-1, 0), c)), gam_f(__fsub_rn(c, ph(1, 0))));
        const float d1 = __fsub_rn(gam_f(__fsub_rn(ph(-1, -1), c)), gam_f(__fsub_rn(c, ph(1, 1))));
        const float d2 = __fsub_rn(gam_f(__fsub_rn(ph(-1, 1), c)), gam_f(__fsub_rn(c, ph(1, -1))));
        const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(h, h), __fmul_rn(v, v)), __fmul_rn(d1, d1)),
                                  __fmul_rn(d2, d2));
        rel[g] = __fdiv_rn(1.f, __fsqrt_rn(s));
    }
}

// best[c] = max over the edges leaving component c of (reliability bits << 32 | ~edge index)
__global__ void __launch_bounds__(kUwThreads) uw_best_edges(UwArgs a, const float* __restrict__ wph,
                                                           const int32_t* __restrict__ fid,
                                                           const float* __restrict__ rel,
                                                           const int32_t* __restrict__ comp,
                                                           unsigned long long* __restrict__ best,
                                                           const int32_t* __restrict__ live) {
    if (!*live) return;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.npx; g += (int64_t)gridDim.x * blockDim.x) {
        if (isnan(wph[g])) continue;
        const FrameDev& F = a.fr[fid[g]];
        const int64_t local = g - (int64_t)F.gam_off;
        const int i = (int)(local / F.W), j = (int)(local % F.W);
        const int32_t cp = comp[g];
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            if (dir == 0 ? j + 1 >= F.W : i + 1 >= F.H) continue;
            const int64_t q = g + (dir == 0 ? 1 : (int64_t)F.W);
            if (isnan(wph[q])) continue;
            const int32_t cq = comp[q];
            if (cp == cq) continue;
            const float w = __fadd_rn(rel[g], rel[q]);
            const unsigned long long e = 2ull * (unsigned long long)g + (unsigned long long)dir;
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(w) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)e);
            atomicMax(best + cp, key);
            atomicMax(best + cq, key);
        }
    }
}

// (parent, shift) of a component in one word: the shift is added to the component's k values
__device__ __forceinline__ unsigned long long pack_hook(int32_t par, int32_t sh) {
    return ((unsigned long long)(uint32_t)par << 32) | (unsigned long long)(uint32_t)sh;
}
__device__ __forceinline__ int32_t hook_par(unsigned long long w) { return (int32_t)(uint32_t)(w >> 32); }
__device__ __forceinline__ int32_t hook_sh(unsigned long long w) { return (int32_t)(uint32_t)(w & 0xffffffffull); }

// every root c hooks onto the component across its best edge: hook[c] = (parent, shift)
__global__ void __launch_bounds__(kUwThreads) uw_hook(UwArgs a, const float* __restrict__ wph,
                                                     const int32_t* __restrict__ fid, const int32_t* __restrict__ comp,
                                                     const int32_t* __restrict__ kk,
                                                     const unsigned long long* __restrict__ best,
                                                     unsigned long long* __restrict__ hook,
                                                     const int32_t* __restrict__ live_in, int32_t* __restrict__ live_out) {
    if (!*live_in) return;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.npx; c += (int64_t)gridDim.x * blockDim.x) {
        if (comp[c] != (int32_t)c) continue;  // not a root
        const unsigned long long key = best[c];
        hook[c] = pack_hook((int32_t)c, 0);
        if (key == 0ull) continue;
        const uint32_t e = 0xffffffffu - (uint32_t)(key & 0xffffffffull);
        const int64_t p = (int64_t)(e >> 1);
        const FrameDev& F = a.fr[fid[p]];
        const int64_t q = p + ((e & 1u) ? (int64_t)F.W : 1);
        const int32_t cp = comp[p], cq = comp[q];
        const int32_t other = cp == (int32_t)c ? cq : cp;
        if (best[other] == key && (int32_t)c < other) continue;  // both chose this edge: c stays the root
        const int s = jump(wph[p], wph[q]);                       // k_q - k_p must equal s
        hook[c] = pack_hook(other, cq == (int32_t)c ? kk[p] + s - kk[q] : kk[q] - s - kk[p]);
        *live_out = 1;
    }
}

// Resolves every hook chain to its root in place and clears the roots' best edges for the next
// round. Each root component jumps over its parent until the parent is a root; many components do
// so at once and help each other (every word read is a consistent (parent, shift) pair, so a
// component may jump over a parent that has itself jumped already). Every jump moves strictly up
// a chain of fewer than npx components, which bounds the loop.
__global__ void __launch_bounds__(kUwThreads) uw_compress(int64_t npx, const int32_t* __restrict__ comp,
                                                         unsigned long long* hook,
                                                         unsigned long long* __restrict__ best,
                                                         int32_t* __restrict__ minpix,
                                                         const int32_t* __restrict__ hooked) {
    if (!*hooked) return;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < npx; c += (int64_t)gridDim.x * blockDim.x) {
        if (comp[c] != (int32_t)c) continue;
        best[c] = 0ull;
        unsigned long long w = *(volatile unsigned long long*)(hook + c);
        for (int64_t it = 0; it < npx; ++it) {
            const int32_t p = hook_par(w);
            if (p == (int32_t)c) break;  // c did not hook: a root of this round
            const unsigned long long wp = *(volatile unsigned long long*)(hook + p);
            const int32_t pp = hook_par(wp);
            if (pp == p) break;  // the parent is a root
            w = pack_hook(pp, hook_sh(w) + hook_sh(wp));
            *(volatile unsigned long long*)(hook + c) = w;
        }
        // the root this component joins inherits its smallest pixel (roots of the round only
        // receive, so minpix[c] is final here)
        const int32_t r = hook_par(w);
        if (r != (int32_t)c) atomicMin(minpix + r, minpix[c]);
    }
}

__global__ void __launch_bounds__(kUwThreads) uw_relabel(int64_t npx, int32_t* __restrict__ comp,
                                                        int32_t* __restrict__ kk,
                                                        const unsigned long long* __restrict__ hook,
                                                        const int32_t* __restrict__ live) {
    if (!*live) return;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < npx; g += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long w = hook[comp[g]];
        kk[g] += hook_sh(w);
        comp[g] = hook_par(w);
    }
}

__global__ void __launch_bounds__(kUwThreads) uw_write(UwArgs a, const float* __restrict__ wph,
                                                      const int32_t* __restrict__ fid, const int32_t* __restrict__ comp,
                                                      const int32_t* __restrict__ kk, const int32_t* __restrict__ minpix) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.npx; g += (int64_t)gridDim.x * blockDim.x) {
        const FrameDev& F = a.fr[fid[g]];
        const int64_t local = g - (int64_t)F.gam_off;
        const float p = wph[g];
        float v = p;
        if (!isnan(p)) {
            const int32_t k = kk[g] - kk[minpix[comp[g]]];
            v = __fadd_rn(p, __fmul_rn(kTwoPiF, (float)k));
        }
        a.out[F.out_off + a.out_maps * (int64_t)F.H * F.W + local] = v;
    }
}

// Workspace carved from one buffer; every array has npx entries.
struct UwWork {
    float* wph;
    float* rel;
    int32_t* minpix;  // smallest pixel index of each component (at its root)
    int32_t* fid;
    int32_t* comp;
    int32_t* kk;
    unsigned long long* hook;
    unsigned long long* best;
    int32_t* flags;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

UwWork carve(void* base, int64_t npx, int rounds) {
    UwWork w;
    char* p = static_cast<char*>(base);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += align256(bytes);
        return r;
    };
    w.best = reinterpret_cast<unsigned long long*>(take(8 * (size_t)npx));
    w.wph = reinterpret_cast<float*>(take(4 * (size_t)npx));
    w.rel = reinterpret_cast<float*>(take(4 * (size_t)npx));
    w.fid = reinterpret_cast<int32_t*>(take(4 * (size_t)npx));
    w.comp = reinterpret_cast<int32_t*>(take(4 * (size_t)npx));
    w.kk = reinterpret_cast<int32_t*>(take(4 * (size_t)npx));
    w.minpix = reinterpret_cast<int32_t*>(take(4 * (size_t)npx));
    w.hook = reinterpret_cast<unsigned long long*>(take(8 * (size_t)npx));
    w.flags = reinterpret_cast<int32_t*>(take(4 * (size_t)(rounds + 1)));
    return w;
}

int ceil_log2(int64_t n) {
    int r = 0;
    while (((int64_t)1 << r) < n) ++r;
    return r;
}

}  // namespace

int unwrap_rounds(int64_t max_frame_px) { return ceil_log2(max_frame_px < 2 ? 2 : max_frame_px) + 1; }

size_t unwrap_workspace_bytes(int64_t npx, int64_t max_frame_px) {
    const int R = unwrap_rounds(max_frame_px);
    return 2 * align256(8 * (size_t)npx) + 6 * align256(4 * (size_t)npx) + align256(4 * (size_t)(R + 1));
}

cudaError_t launch_unwrap(const FrameDev* d_frames, int nframes, int64_t npx, int64_t max_frame_px,
                          const float* in, int64_t in_maps, float* out, int64_t out_maps, void* work,
                          int* launches, cudaStream_t s) {
    if (npx <= 0) return cudaSuccess;
    const int R = unwrap_rounds(max_frame_px);
    UwWork w = carve(work, npx, R);
    UwArgs a{d_frames, nframes, npx, in, in_maps, out, out_maps};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (npx + kUwThreads - 1) / kUwThreads;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    cudaError_t e;
    // flags[r]: round r is live (round 0 always; round r + 1 if round r joined anything)
    e = cudaMemsetAsync(w.flags, 0, 4 * (size_t)(R + 1), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.flags, 0xff, 4, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.best, 0, 8 * (size_t)npx, s);
    if (e != cudaSuccess) return e;
    uw_init<<<grid, kUwThreads, 0, s>>>(a, w.wph, w.fid, w.comp, w.kk, w.minpix);
    uw_reliability<<<grid, kUwThreads, 0, s>>>(a, w.wph, w.fid, w.rel);
    *launches += 2;
    for (int r = 0; r < R; ++r) {
        const int32_t* live = w.flags + r;
        int32_t* hooked = w.flags + r + 1;
        uw_best_edges<<<grid, kUwThreads, 0, s>>>(a, w.wph, w.fid, w.rel, w.comp, w.best, live);
        uw_hook<<<grid, kUwThreads, 0, s>>>(a, w.wph, w.fid, w.comp, w.kk, w.best, w.hook, live, hooked);
        uw_compress<<<grid, kUwThreads, 0, s>>>(npx, w.comp, w.hook, w.best, w.minpix, hooked);
        uw_relabel<<<grid, kUwThreads, 0, s>>>(npx, w.comp, w.kk, w.hook, hooked);
        *launches += 4;
    }
    uw_write<<<grid, kUwThreads, 0, s>>>(a, w.wph, w.fid, w.comp, w.kk, w.minpix);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace rmusic
