// unwrap.cu -- phase assembly (Sec. 3: the local phases alpha are followed by an unwrapping
// operation, the reliability-sorting method of Herraez et al. 2002 that the paper cites).
//
// The method takes the edges between neighbouring pixels from the most reliable down and joins
// the two groups an edge connects, shifting one by the multiple of 2 pi that makes its endpoints
// differ by their wrapped difference. That order is Kruskal's algorithm for the maximum spanning
// forest of the pixel grid weighted by edge reliability, and the result is the 2 pi jumps
// integrated along that forest: it depends on the forest only, not on the order in which its
// edges are found. Edge weights are made unique by the edge index (reliability first, then the
// smaller index), so the forest is unique, and any algorithm that only ever adds forest edges
// reproduces the sequential result bit for bit. The GPU builds it in two phases:
//   reliability  per pixel, R = 1 / D from the wrapped second differences (0 where a neighbour
//                is missing), computed with explicitly rounded float32 operations so that every
//                comparison below sees exactly the values of the sequential method;
//   tiles        one CTA per 32 x 32 tile runs Boruvka's rounds in shared memory: every local
//                component finds its most reliable edge over ALL its edges, those that leave the
//                tile included; where that edge stays inside the tile the component hooks across
//                it (the most reliable edge leaving a set of pixels belongs to the forest: the cut
//                property), where it leaves the tile the component waits (others may still hook
//                onto it). Rounds repeat until no component hooks. What is left of the tile's
//                edges to the global phase: every edge that leaves the tile, and the edges inside
//                it between different local components;
//   global       Boruvka's rounds over that edge list and the local components that touch it
//                (a few per cent of the pixels and edges), two launches per round: the first
//                relabels every component to the root its hook chain leads to (in-place pointer
//                jumping; parent and shift share one 64-bit word, so a jump always reads a
//                consistent pair) and offers every edge between different components to both
//                (64-bit atomicMax on (reliability bits, ~edge index), issued only when it can
//                win); the second lets every root hook onto the component across its best edge
//                (of two roots that chose the same edge the smaller label stays the root) with the
//                integer shift that makes the edge's endpoints differ by their wrapped difference.
//                The edge list is compacted as it is scanned (an edge inside a component stays
//                inside). A round after one that joined nothing returns at once. Each round at
//                least halves the components that still have edges, and they are at most the
//                tiles' border pixels: ceil(log2) of that many rounds, plus one to relabel.
//   anchor ka    after the rounds, per local root: its shift to its final root minus the shift of
//                that root's anchor pixel; a pixel's output needs only its own k and its root's ka.
//   anchor       each connected region keeps its first pixel (row-major) at its wrapped value;
//                every component carries its smallest pixel index through the merges.
// A pixel's k is its shift within its local component plus that component's shift within its
// global component. All integer bookkeeping is exact; the output is phi + 2 pi k in float32.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

namespace {

constexpr int kUwThreads = 256;
constexpr int kTile = 32;                          // tile side (pixels)
constexpr int kTilePx = kTile * kTile;             // pixels per tile
constexpr int kPxPerThread = kTilePx / kUwThreads; // 4: rows w, w + 8, w + 16, w + 24 of warp w
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

// Edge e = 2 p + dir (dir 0: p -> p + 1, dir 1: p -> p + W) of weight w = rel[p] + rel[q]: the
// larger key is the more reliable edge, ties going to the smaller index.
__device__ __forceinline__ unsigned long long edge_key(float w, uint32_t e) {
    return ((unsigned long long)__float_as_uint(w) << 32) | (unsigned long long)(0xffffffffu - e);
}
__device__ __forceinline__ uint32_t key_edge(unsigned long long key) {
    return 0xffffffffu - (uint32_t)(key & 0xffffffffull);
}

// (parent, shift) of a component in one word: the shift is added to the component's k values
__device__ __forceinline__ unsigned long long pack_hook(int32_t par, int32_t sh) {
    return ((unsigned long long)(uint32_t)par << 32) | (unsigned long long)(uint32_t)sh;
}
__device__ __forceinline__ int32_t hook_par(unsigned long long w) { return (int32_t)(uint32_t)(w >> 32); }
__device__ __forceinline__ int32_t hook_sh(unsigned long long w) { return (int32_t)(uint32_t)(w & 0xffffffffull); }

struct UwArgs {
    const FrameDev* fr;
    int nframes;
    int64_t npx;
    const float* in;    // map of frame f at in + F.out_off + in_maps * H * W
    int64_t in_maps;
    float* out;         // map of frame f at out + F.out_off + out_maps * H * W
    int64_t out_maps;
    unsigned long long* timeouts;  // grid-wide waits of uw_gtail that gave up (device counter, may be null)
};

// Workspace carved from one buffer. Per pixel g: wph (wrapped phase), rel, fid (frame), comp (root
// of g's local component), kk (g's shift within it); per local root r: minpix, comp2 (r's root as
// of the last relabelling), kk2 (r's shift to it), ka, hook, best (two copies: even and odd
// rounds). Each edge list holds at most the grid's two edges per pixel, the node list at most one
// local root per pixel.
struct UwWork {
    float* wph;
    float* rel;
    int32_t* fid;
    int32_t* comp;
    int32_t* kk;
    int32_t* minpix;
    int32_t* comp2;
    int32_t* kk2;
    int32_t* ka;        // per local root: its shift to its final root minus the anchor pixel's k
    unsigned long long* hook;
    unsigned long long* best;   // two arrays of npx: best of even rounds, then of odd rounds
    uint4* edges;       // (e, weight bits, local root of p, local root of q) per listed edge
    uint4* edges2;      // the edges still between different components, round by round (ping-pong)
    int32_t* ecount;    // rounds + 1: edges entering each round after the first
    int32_t* nodes;     // local roots with at least one edge in the list
    int32_t* tile_start;  // nframes + 1 entries: first tile of each frame, then the total
    unsigned long long* counts;  // listed edges (low word) and nodes (high word)
    int32_t* flags;     // rounds + 1 live flags
    unsigned int* sync; // uw_gtail's grid barriers: [0] arrivals, [32] the last barrier passed
    int32_t* stop;      // set when one of uw_gtail's grid barriers gave up
    int64_t npx;
};

__device__ __forceinline__ int32_t n_edges(const UwWork& w) { return (int32_t)(uint32_t)(*w.counts & 0xffffffffull); }
__device__ __forceinline__ int32_t n_nodes(const UwWork& w) { return (int32_t)(uint32_t)(*w.counts >> 32); }

// Tiles of a frame: ceil(H / 32) x ceil(W / 32), row-major.
__device__ __forceinline__ int32_t frame_tiles(const FrameDev& F) {
    return ((F.H + kTile - 1) / kTile) * ((F.W + kTile - 1) / kTile);
}

// tile_start[f] = tiles of frames 0 .. f - 1 (one block; frames in chunks of its width), counters
// cleared, round 0 live.
__global__ void __launch_bounds__(kUwThreads) uw_prepare(UwArgs a, UwWork w, int rounds) {
    __shared__ int32_t wsum[kUwThreads / 32];
    __shared__ int32_t carry;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) carry = 0;
    for (int i = t; i < rounds + 1; i += blockDim.x) {
        w.flags[i] = i == 0 ? 1 : 0;
        w.ecount[i] = 0;
    }
    if (t == 0) {
        *w.counts = 0ull;
        w.sync[0] = 0u;
        w.sync[32] = 0u;
        *w.stop = 0;
    }
    __syncthreads();
    for (int base = 0; base < a.nframes; base += kUwThreads) {
        const int f = base + t;
        const int32_t n = f < a.nframes ? frame_tiles(a.fr[f]) : 0;
        int32_t x = n;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        int32_t before = carry;
        for (int k = 0; k < wid; ++k) before += wsum[k];
        if (f < a.nframes) w.tile_start[f] = before + x - n;
        __syncthreads();
        if (t == kUwThreads - 1) carry = before + x;
        __syncthreads();
    }
    if (t == 0) w.tile_start[a.nframes] = carry;
}

// wph[g] = wrapped phase, fid[g] = frame, rel[g] = reliability R = 1 / D from the wrapped second
// differences of the 3 x 3 neighbourhood (0 where a neighbour is missing or NaN; NaN at NaN pixels),
// read from the input map directly (a frame's map is contiguous, row-major).
__global__ void __launch_bounds__(kUwThreads) uw_init(UwArgs a, float* __restrict__ wph, int32_t* __restrict__ fid,
                                                     float* __restrict__ rel) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.npx; g += (int64_t)gridDim.x * blockDim.x) {
        const int f = find_frame(a.fr, a.nframes, g, [](const FrameDev& F) { return (int64_t)F.gam_off; });
        const FrameDev& F = a.fr[f];
        const int64_t local = g - (int64_t)F.gam_off;
        const float* m = a.in + F.out_off + a.in_maps * (int64_t)F.H * F.W;
        const float c = m[local];
        wph[g] = c;
        fid[g] = f;
        if (isnan(c)) {
            rel[g] = c;
            continue;
        }
        // a frame has fewer than 2^31 pixels: 32-bit division (a 64-bit one is a long routine)
        const int W = F.W;
        const int i = (int)((uint32_t)local / (uint32_t)W), j = (int)((uint32_t)local - (uint32_t)i * (uint32_t)W);
        bool inner = i >= 1 && i + 1 < F.H && j >= 1 && j + 1 < W;
        if (inner) {
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj)
                    if (isnan(m[local + (int64_t)di * W + dj])) inner = false;
        }
        if (!inner) {
            rel[g] = 0.f;
            continue;
        }
        auto ph = [&](int di, int dj) { return m[local + (int64_t)di * W + dj]; };
        const float h = __fsub_rn(gam_f(__fsub_rn(ph(0, -1), c)), gam_f(__fsub_rn(c, ph(0, 1))));
        const float v = __fsub_rn(gam_f(__fsub_rn(ph(-1, 0), c)), gam_f(__fsub_rn(c, ph(1, 0))));
        const float d1 = __fsub_rn(gam_f(__fsub_rn(ph(-1, -1), c)), gam_f(__fsub_rn(c, ph(1, 1))));
        const float d2 = __fsub_rn(gam_f(__fsub_rn(ph(-1, 1), c)), gam_f(__fsub_rn(c, ph(1, -1))));
        const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(h, h), __fmul_rn(v, v)), __fmul_rn(d1, d1)),
                                  __fmul_rn(d2, d2));
        rel[g] = __fdiv_rn(1.f, __fsqrt_rn(s));
    }
}

// Every thread of the block asks for ne slots of the edge list and nn of the node list; one 64-bit
// atomicAdd per block on the packed lengths (edges in the low word: at most two per pixel, below
// 2^32). Returns the thread's first slots. Called by all threads.
__device__ __forceinline__ void block_reserve(int32_t ne, int32_t nn, unsigned long long* counter, int32_t* s_wsum,
                                              unsigned long long* s_base, int32_t* e0, int32_t* n0) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int32_t xe = ne, xn = nn;  // inclusive scans within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t ye = __shfl_up_sync(0xffffffffu, xe, o), yn = __shfl_up_sync(0xffffffffu, xn, o);
        if (lane >= o) {
            xe += ye;
            xn += yn;
        }
    }
    if (lane == 31) {
        s_wsum[wid] = xe;
        s_wsum[kUwThreads / 32 + wid] = xn;
    }
    __syncthreads();
    if (t == 0) {
        int32_t te = 0, tn = 0;
        for (int k = 0; k < kUwThreads / 32; ++k) {
            const int32_t ve = s_wsum[k], vn = s_wsum[kUwThreads / 32 + k];
            s_wsum[k] = te;
            s_wsum[kUwThreads / 32 + k] = tn;
            te += ve;
            tn += vn;
        }
        const unsigned long long add = ((unsigned long long)(uint32_t)tn << 32) | (unsigned long long)(uint32_t)te;
        *s_base = add ? atomicAdd(counter, add) : 0ull;
    }
    __syncthreads();
    const unsigned long long base = *s_base;
    *e0 = (int32_t)(uint32_t)(base & 0xffffffffull) + s_wsum[wid] + xe - ne;
    *n0 = (int32_t)(uint32_t)(base >> 32) + s_wsum[kUwThreads / 32 + wid] + xn - nn;
    __syncthreads();
}

// The most reliable edge seen so far into *slot: a plain read first, so that the atomic is issued
// only by edges that can still win (best values only grow while edges are scanned).
__device__ __forceinline__ void offer(unsigned long long* slot, unsigned long long key) {
    if (key > *(volatile unsigned long long*)slot) atomicMax(slot, key);
}

// Shared-memory layout of uw_tiles (dynamic shared memory, kTileSmem bytes): per pixel l of the
// tile the phase, reliability, best edge of the edges leaving the tile at l, ownership bits of the
// edges to the right and lower tiles, the round-0 component and the shift within it; per component
// (indexed by its root's pixel) the best edge, the hook and whether it is a root of the current
// round; the lists the rounds after the first iterate over (edges between different components,
// ping-pong; roots, ping-pong; pixels with an edge out of the tile).
struct TileSmem {
    unsigned long long* best;   // kTilePx
    unsigned long long* hook;   // kTilePx
    unsigned long long* cross;  // kTilePx
    float* ph;                  // kTilePx
    float* rel;                 // kTilePx
    int32_t* kk;                // kTilePx
    int16_t* comp0;             // kTilePx
    uint16_t* elist0;           // 2 kTilePx each: (pixel << 1) | dir of an edge inside the tile
    uint16_t* elist1;
    uint16_t* rlist0;           // kTilePx each
    uint16_t* rlist1;
    uint16_t* blist;            // 4 kTile
    uint8_t* own;               // kTilePx
    uint8_t* cur;               // kTilePx: 1 for a root of the current round
    int32_t* misc;              // [0..2] edge counts, [3..5] root counts (by round modulo 3), [6] border count
};
constexpr size_t kTileSmem = 3 * 8 * kTilePx + 3 * 4 * kTilePx + 2 * kTilePx + 2 * (2 * 2 * kTilePx) +
                             2 * (2 * kTilePx) + 2 * 4 * kTile + 2 * kTilePx + 32 * 4;

__device__ __forceinline__ TileSmem tile_smem(unsigned char* base) {
    TileSmem t;
    unsigned char* p = base;
    t.best = reinterpret_cast<unsigned long long*>(p);
    p += 8 * kTilePx;
    t.hook = reinterpret_cast<unsigned long long*>(p);
    p += 8 * kTilePx;
    t.cross = reinterpret_cast<unsigned long long*>(p);
    p += 8 * kTilePx;
    t.ph = reinterpret_cast<float*>(p);
    p += 4 * kTilePx;
    t.rel = reinterpret_cast<float*>(p);
    p += 4 * kTilePx;
    t.kk = reinterpret_cast<int32_t*>(p);
    p += 4 * kTilePx;
    t.comp0 = reinterpret_cast<int16_t*>(p);
    p += 2 * kTilePx;
    // (named buffers, picked by ternaries below: a pointer array indexed at run time would put the
    // whole struct in local memory)
    t.elist0 = reinterpret_cast<uint16_t*>(p);
    p += 2 * 2 * kTilePx;
    t.elist1 = reinterpret_cast<uint16_t*>(p);
    p += 2 * 2 * kTilePx;
    t.rlist0 = reinterpret_cast<uint16_t*>(p);
    p += 2 * kTilePx;
    t.rlist1 = reinterpret_cast<uint16_t*>(p);
    p += 2 * kTilePx;
    t.blist = reinterpret_cast<uint16_t*>(p);
    p += 2 * 4 * kTile;
    t.own = p;
    p += kTilePx;
    t.cur = p;
    p += kTilePx;
    t.misc = reinterpret_cast<int32_t*>(p);
    return t;
}

// Root of the component whose former root is x (a component of round 0), and x's shift to it:
// chases the hooks, stopping at a root of the current round (cur), jumping in place (every word
// written is a valid (ancestor, summed shift) pair). A chain has fewer than kTilePx links.
__device__ __forceinline__ unsigned long long tile_find(const TileSmem& S, int32_t x) {
    volatile unsigned long long* vh = S.hook;
    unsigned long long hw = S.cur[x] ? pack_hook(x, 0) : vh[x];
    for (int it = 0; it < kTilePx && !S.cur[hook_par(hw)]; ++it) {
        const int32_t p = hook_par(hw);
        const unsigned long long wp = vh[p];
        hw = pack_hook(hook_par(wp), hook_sh(hw) + hook_sh(wp));
        vh[x] = hw;
    }
    return hw;
}

// Appends the flagged items of the block's threads to a shared list: one shared atomic per warp.
// Called by all threads; returns the item's slot (or -1 when not flagged).
__device__ __forceinline__ int32_t block_append(bool flag, int32_t* count) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    int32_t base = 0;
    if (lane == 0 && m) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    return flag ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

// One CTA per 32 x 32 tile (persistent over the tiles of all frames). Pixel l = 32 i + j of the
// tile is handled by thread l % 256 where the work is per pixel. Round 0 treats every pixel as a
// component: its best edge is the largest of its own (at most four, and the best of those leaving
// the tile), with no atomics. The rounds after it iterate only over the lists: the edges inside the
// tile between different components (compacted as components merge), the pixels with an edge out
// of the tile, and the roots; labels are looked up through the hook chains (tile_find) and written
// back per pixel once, after the last round.
__global__ void __launch_bounds__(kUwThreads) uw_tiles(UwArgs a, UwWork w) {
    extern __shared__ __align__(16) unsigned char tile_smem_raw[];
    const TileSmem S = tile_smem(tile_smem_raw);
    __shared__ int32_t s_wsum[2 * (kUwThreads / 32)];
    __shared__ unsigned long long s_base;
    __shared__ int s_any[2];
    const int t = threadIdx.x;
    const int32_t ntiles = w.tile_start[a.nframes];
    for (int32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int lo = 0, hi = a.nframes - 1;  // frame of the tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (w.tile_start[mid] <= tile)
                lo = mid;
            else
                hi = mid - 1;
        }
        const FrameDev& F = a.fr[lo];
        const int H = F.H, W = F.W;
        const int ntx = (W + kTile - 1) / kTile;
        const int lt = tile - w.tile_start[lo];
        const int y0 = (lt / ntx) * kTile, x0 = (lt % ntx) * kTile;
        const int64_t g0 = (int64_t)F.gam_off;
        const int64_t tg = g0 + (int64_t)y0 * W + x0;  // pixel (0, 0) of the tile
        auto gl = [&](int32_t m) { return (uint32_t)(tg + (int64_t)(m >> 5) * W + (m & 31)); };
        bool in[kPxPerThread];
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads, i = l >> 5, j = l & 31;
            const int y = y0 + i, x = x0 + j;
            in[k] = y < H && x < W;
            const int64_t g = tg + (int64_t)i * W + j;
            // the pixel and its neighbours across the tile's sides (at most one horizontal and one
            // vertical), all loads issued before any is used
            const bool hr = in[k] && j == kTile - 1 && x + 1 < W, hl = in[k] && j == 0 && x >= 1;
            const bool vd = in[k] && i == kTile - 1 && y + 1 < H, vu = in[k] && i == 0 && y >= 1;
            const int64_t gh = hr ? g + 1 : g - 1, gv = vd ? g + W : g - W;
            const float nan = __int_as_float(0x7fffffff);
            float ph = nan, r = 0.f, phh = nan, rh = 0.f, phv = nan, rv = 0.f;
            if (in[k]) {
                ph = w.wph[g];
                r = w.rel[g];
            }
            if (hr || hl) {
                phh = w.wph[gh];
                rh = w.rel[gh];
            }
            if (vd || vu) {
                phv = w.wph[gv];
                rv = w.rel[gv];
            }
            unsigned long long cross = 0ull;
            uint8_t own = 0;
            if (isnan(ph)) {
                r = 0.f;
            } else {
                if (!isnan(phh)) {
                    cross = max(cross, hr ? edge_key(__fadd_rn(r, rh), (uint32_t)(2 * g))
                                          : edge_key(__fadd_rn(rh, r), (uint32_t)(2 * gh)));
                    own |= hr ? 1 : 0;
                }
                if (!isnan(phv)) {
                    cross = max(cross, vd ? edge_key(__fadd_rn(r, rv), (uint32_t)(2 * g + 1))
                                          : edge_key(__fadd_rn(rv, r), (uint32_t)(2 * gv + 1)));
                    own |= vd ? 2 : 0;
                }
            }
            S.ph[l] = ph;
            S.rel[l] = r;
            S.cross[l] = cross;
            S.own[l] = own;
        }
        if (t < 8) S.misc[t] = 0;  // list counts
        if (t == 0) s_any[0] = s_any[1] = 0;
        __syncthreads();

        // ---- round 0: each pixel's most reliable edge among its own -----------------------------
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads, i = l >> 5, j = l & 31;
            unsigned long long b = 0ull;
            if (!isnan(S.ph[l])) {
                const int64_t g = tg + (int64_t)i * W + j;
                b = S.cross[l];
                if (j + 1 < kTile && !isnan(S.ph[l + 1]))
                    b = max(b, edge_key(__fadd_rn(S.rel[l], S.rel[l + 1]), (uint32_t)(2 * g)));
                if (i + 1 < kTile && !isnan(S.ph[l + kTile]))
                    b = max(b, edge_key(__fadd_rn(S.rel[l], S.rel[l + kTile]), (uint32_t)(2 * g + 1)));
                if (j > 0 && !isnan(S.ph[l - 1]))
                    b = max(b, edge_key(__fadd_rn(S.rel[l - 1], S.rel[l]), (uint32_t)(2 * (g - 1))));
                if (i > 0 && !isnan(S.ph[l - kTile]))
                    b = max(b, edge_key(__fadd_rn(S.rel[l - kTile], S.rel[l]), (uint32_t)(2 * (g - W) + 1)));
            }
            S.best[l] = b;
        }
        __syncthreads();
        // hooks across round 0's best edges that stay in the tile (shifts: every k is 0 here)
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            unsigned long long hk = pack_hook(l, 0);
            const unsigned long long key = S.best[l];
            if (key) {
                const uint32_t e = key_edge(key);
                const int64_t d = (int64_t)(e >> 1) - tg;
                if (d >= 0) {
                    const uint32_t pi = (uint32_t)d / (uint32_t)W, pj = (uint32_t)d - pi * (uint32_t)W;
                    const uint32_t qi = pi + (e & 1u), qj = pj + 1u - (e & 1u);
                    if (qi < kTile && qj < kTile) {
                        const int pl = (int)(pi * kTile + pj), ql = (int)(qi * kTile + qj);
                        const int32_t other = pl == l ? ql : pl;
                        if (!(S.best[other] == key && l < other)) {
                            const int s = jump(S.ph[pl], S.ph[ql]);
                            hk = pack_hook(other, ql == l ? s : -s);
                        }
                    }
                }
            }
            S.hook[l] = hk;
        }
        __syncthreads();
        // every pixel's round-0 root and shift (the hook chains, jumped in place); the roots are the
        // current ones of round 1 and start with no best edge
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            volatile unsigned long long* vh = S.hook;
            unsigned long long hw = vh[l];
            for (int it = 0; it < kTilePx; ++it) {
                const int32_t p = hook_par(hw);
                if (p == l) break;
                const unsigned long long wp = vh[p];
                const int32_t pp = hook_par(wp);
                if (pp == p) break;
                hw = pack_hook(pp, hook_sh(hw) + hook_sh(wp));
                vh[l] = hw;
            }
            S.comp0[l] = (int16_t)hook_par(hw);
            S.kk[l] = hook_sh(hw);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            const bool root = !isnan(S.ph[l]) && S.comp0[l] == l;
            S.cur[l] = root ? 1 : 0;
            S.best[l] = 0ull;
        }
        // the lists: edges inside the tile between different round-0 components, roots, pixels with
        // an edge out of the tile
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            const bool v = !isnan(S.ph[l]);
            const int c = S.comp0[l];
            const bool er = v && (l & 31) + 1 < kTile && !isnan(S.ph[l + 1]) && S.comp0[l + 1] != c;
            const bool ed = v && (l >> 5) + 1 < kTile && !isnan(S.ph[l + kTile]) && S.comp0[l + kTile] != c;
            int32_t slot = block_append(er, &S.misc[0]);
            if (er) S.elist0[slot] = (uint16_t)(l << 1);
            slot = block_append(ed, &S.misc[0]);
            if (ed) S.elist0[slot] = (uint16_t)((l << 1) | 1);
            slot = block_append(v && c == l, &S.misc[3]);
            if (slot >= 0) S.rlist0[slot] = (uint16_t)l;
            slot = block_append(v && S.cross[l] != 0ull, &S.misc[6]);
            if (slot >= 0) S.blist[slot] = (uint16_t)l;
        }
        __syncthreads();

        // ---- rounds 1, 2, ...: over the lists; round r reads the lists of round r - 1 (buffers by
        // parity) and their counts (misc[(r - 1) % 3] edges, misc[3 + (r - 1) % 3] roots), writes its
        // own; the counts of round r + 1 are cleared at the start of round r (their previous
        // contents were last read in round r - 1, before its last barrier). Each round that hooks
        // merges at least two components.
        for (int round = 1;; ++round) {
            int* any = &s_any[round & 1];
            if (t == 0) {
                s_any[(round + 1) & 1] = 0;
                S.misc[(round + 1) % 3] = 0;
                S.misc[3 + (round + 1) % 3] = 0;
            }
            const bool odd = round & 1;
            const uint16_t* ecur = odd ? S.elist0 : S.elist1;
            uint16_t* enext = odd ? S.elist1 : S.elist0;
            const uint16_t* rcur = odd ? S.rlist0 : S.rlist1;
            uint16_t* rnext = odd ? S.rlist1 : S.rlist0;
            const int32_t ne = S.misc[(round - 1) % 3];
            const int32_t nr = S.misc[3 + (round - 1) % 3];
            // every edge still between different components offered to both; kept for the next round
            for (int32_t b0 = 0; b0 < ne; b0 += kUwThreads) {
                const int32_t i = b0 + t;
                bool keep = false;
                uint16_t code = 0;
                if (i < ne) {
                    code = ecur[i];
                    const int pl = code >> 1, ql = pl + ((code & 1) ? kTile : 1);
                    const int32_t cp = hook_par(tile_find(S, S.comp0[pl]));
                    const int32_t cq = hook_par(tile_find(S, S.comp0[ql]));
                    if (cp != cq) {
                        keep = true;
                        const unsigned long long key =
                            edge_key(__fadd_rn(S.rel[pl], S.rel[ql]), 2u * gl(pl) + (uint32_t)(code & 1));
                        offer(&S.best[cp], key);
                        offer(&S.best[cq], key);
                    }
                }
                const int32_t slot = block_append(keep, &S.misc[round % 3]);
                if (keep) enext[slot] = code;
            }
            const int32_t nb = S.misc[6];
            for (int32_t i = t; i < nb; i += kUwThreads) {
                const int b = S.blist[i];
                offer(&S.best[hook_par(tile_find(S, S.comp0[b]))], S.cross[b]);
            }
            __syncthreads();
            // roots whose best edge stays in the tile hook across it (tile_find stops at the roots of
            // this round, so the hooks written meanwhile do not move the endpoints' roots)
            for (int32_t i = t; i < nr; i += kUwThreads) {
                const int32_t r = rcur[i];
                const unsigned long long key = S.best[r];
                if (!key) continue;
                const uint32_t e = key_edge(key);
                const int64_t d = (int64_t)(e >> 1) - tg;
                if (d < 0) continue;
                const uint32_t pi = (uint32_t)d / (uint32_t)W, pj = (uint32_t)d - pi * (uint32_t)W;
                const uint32_t qi = pi + (e & 1u), qj = pj + 1u - (e & 1u);
                if (qi >= kTile || qj >= kTile) continue;  // the edge leaves the tile: the root waits
                const int pl = (int)(pi * kTile + pj), ql = (int)(qi * kTile + qj);
                const unsigned long long hp = tile_find(S, S.comp0[pl]), hq = tile_find(S, S.comp0[ql]);
                const int32_t cp = hook_par(hp), cq = hook_par(hq);
                const int32_t other = cp == r ? cq : cp;
                if (S.best[other] == key && r < other) continue;  // both chose this edge: r stays the root
                const int s = jump(S.ph[pl], S.ph[ql]);
                const int32_t kp = S.kk[pl] + hook_sh(hp), kq = S.kk[ql] + hook_sh(hq);
                S.hook[r] = pack_hook(other, cq == r ? kp + s - kq : kq - s - kp);
                *any = 1;
            }
            __syncthreads();
            if (!*any || round >= kTilePx) break;  // (a productive round merges: < 1024 of them)
            // this round's hooks resolved to roots in place; the roots that stay form the next list
            for (int32_t b0 = 0; b0 < nr; b0 += kUwThreads) {
                const int32_t i = b0 + t;
                bool stay = false;
                int32_t r = 0;
                if (i < nr) {
                    r = rcur[i];
                    S.best[r] = 0ull;
                    volatile unsigned long long* vh = S.hook;
                    unsigned long long hw = vh[r];
                    for (int it = 0; it < kTilePx; ++it) {
                        const int32_t p = hook_par(hw);
                        if (p == r) break;
                        const unsigned long long wp = vh[p];
                        const int32_t pp = hook_par(wp);
                        if (pp == p) break;
                        hw = pack_hook(pp, hook_sh(hw) + hook_sh(wp));
                        vh[r] = hw;
                    }
                    stay = hook_par(hw) == r;
                    S.cur[r] = stay ? 1 : 0;
                }
                const int32_t slot = block_append(stay, &S.misc[3 + round % 3]);
                if (stay) rnext[slot] = (uint16_t)r;
            }
            __syncthreads();
        }

        // ---- every pixel's final component and shift; the smallest member of each component -----
        int16_t finv[kPxPerThread];
        int32_t kkv[kPxPerThread];
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            finv[k] = (int16_t)l;
            kkv[k] = 0;
            if (!isnan(S.ph[l])) {
                const unsigned long long hw = tile_find(S, S.comp0[l]);
                finv[k] = (int16_t)hook_par(hw);
                kkv[k] = S.kk[l] + hook_sh(hw);
            }
        }
        __syncthreads();
        int32_t* s_minm = reinterpret_cast<int32_t*>(S.best);  // free now
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            S.comp0[l] = finv[k];
            S.kk[l] = kkv[k];
            s_minm[l] = l;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            if (!isnan(S.ph[l])) atomicMin(&s_minm[finv[k]], l);
        }
        __syncthreads();

        // local components out: comp (as a pixel index), kk; per local root its smallest pixel and
        // the identity as its global state
        const int16_t* fin = S.comp0;
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            if (!in[k]) continue;
            const int64_t g = tg + (int64_t)(l >> 5) * W + (l & 31);
            const int32_t c = fin[l];
            w.comp[g] = (int32_t)gl(c);
            w.kk[g] = S.kk[l];
            if (c == l) {
                const int32_t m = s_minm[l];
                w.minpix[g] = (int32_t)gl(m);
                w.comp2[g] = (int32_t)g;
                w.kk2[g] = 0;
                w.ka[g] = -S.kk[m];  // a local root outside the global phase is its own final root
                w.best[g] = 0ull;    // best of round 0
                w.hook[g] = pack_hook((int32_t)g, 0);
            }
        }
        __syncthreads();
        int32_t* s_mark = S.kk;  // free now: marks the local roots that the global edges touch
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) s_mark[t + k * kUwThreads] = 0;
        __syncthreads();

        // the global phase's edges: every edge this tile owns across its right and lower sides,
        // and the edges inside the tile between different local components; and the local roots
        // that they touch (those with an edge out of the tile on any side, or such an edge inside)
        int32_t ne = 0;
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            if (isnan(S.ph[l])) continue;
            const int32_t c = fin[l];
            if (S.cross[l]) s_mark[c] = 1;
            ne += (S.own[l] & 1) + ((S.own[l] >> 1) & 1);
            if ((l & 31) + 1 < kTile && !isnan(S.ph[l + 1]) && fin[l + 1] != c) {
                ++ne;
                s_mark[c] = 1;
                s_mark[fin[l + 1]] = 1;
            }
            if ((l >> 5) + 1 < kTile && !isnan(S.ph[l + kTile]) && fin[l + kTile] != c) {
                ++ne;
                s_mark[c] = 1;
                s_mark[fin[l + kTile]] = 1;
            }
        }
        __syncthreads();
        int32_t nn = 0;
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) nn += s_mark[t + k * kUwThreads];
        int32_t eslot, nslot;
        block_reserve(ne, nn, w.counts, s_wsum, &s_base, &eslot, &nslot);
        // edge records (e, weight bits, local root of p, local root of q); an edge out of the tile
        // carries q | 2^31 instead, its weight and q's local root are filled in by the first round
#pragma unroll
        for (int k = 0; k < kPxPerThread; ++k) {
            const int l = t + k * kUwThreads;
            if (s_mark[l]) w.nodes[nslot++] = (int32_t)gl(l);
            if (isnan(S.ph[l])) continue;
            const int32_t c = fin[l];
            const uint32_t g = gl(l);
            if (S.own[l] & 1) {
                w.edges[eslot++] = make_uint4(2u * g, 0u, gl(c), (g + 1u) | 0x80000000u);
            } else if ((l & 31) + 1 < kTile && !isnan(S.ph[l + 1]) && fin[l + 1] != c) {
                w.edges[eslot++] = make_uint4(2u * g, __float_as_uint(__fadd_rn(S.rel[l], S.rel[l + 1])), gl(c),
                                              gl(fin[l + 1]));
            }
            if (S.own[l] & 2) {
                w.edges[eslot++] = make_uint4(2u * g + 1u, 0u, gl(c), (g + (uint32_t)W) | 0x80000000u);
            } else if ((l >> 5) + 1 < kTile && !isnan(S.ph[l + kTile]) && fin[l + kTile] != c) {
                w.edges[eslot++] = make_uint4(2u * g + 1u, __float_as_uint(__fadd_rn(S.rel[l], S.rel[l + kTile])),
                                              gl(c), gl(fin[l + kTile]));
            }
        }
        __syncthreads();
    }
}

// Root of the component of x and x's shift to it, through the hook chain (hooks of earlier rounds
// point up the chain; a root's hook is itself). Jumps are written back in place: every word written
// is a valid (ancestor, summed shift) pair, so threads that chase the same chain help each other.
// Each jump moves strictly up a chain of fewer than n components, which bounds the loop.
__device__ __forceinline__ unsigned long long find_root(unsigned long long* hook, int32_t x, int32_t n) {
    volatile unsigned long long* vh = hook;
    unsigned long long hw = vh[x];
    if (hook_par(hw) == x) return hw;
    for (int32_t it = 0; it < n; ++it) {
        const int32_t p = hook_par(hw);
        const unsigned long long wp = vh[p];
        const int32_t pp = hook_par(wp);
        if (pp == p) break;  // p is a root
        hw = pack_hook(pp, hook_sh(hw) + hook_sh(wp));
        vh[x] = hw;
    }
    return hw;
}

// Loads of words that other CTAs may have written earlier in the same launch (the cooperative
// kernel below): from L2 (ld.global.cg), never a stale L1 line. Between launches a plain load.
template <bool kL2>
__device__ __forceinline__ int32_t ldx(const int32_t* p) {
    if constexpr (kL2) return __ldcg(p);
    else return *p;
}
template <bool kL2>
__device__ __forceinline__ unsigned long long ldx(const unsigned long long* p) {
    if constexpr (kL2) return __ldcg(p);
    else return *p;
}
template <bool kL2>
__device__ __forceinline__ uint4 ldx(const uint4* p) {
    if constexpr (kL2) return __ldcg(p);
    else return *p;
}

// Round r, scan: every listed component takes the hooks of round r - 1 (comp2 = its root, kk2 +=
// its shift to it; a root of round r - 1 that hooked hands its smallest pixel to its new root),
// and every edge still between different components is offered to both components' best[r & 1]
// and kept for round r + 1 (the list shrinks as components merge: an edge inside a component
// stays inside). Called by every thread of the grid (tid, stride: its index and the grid's
// threads); the edge loop is block-uniform, so the kept edges are appended with one atomic per
// block (one per warp on a single counter serialises in L2).
template <bool kL2>
__device__ __forceinline__ void scan_round(const UwWork& w, unsigned long long* best, int r, int32_t tid,
                                           int32_t stride, int32_t* s_wcnt, int32_t* s_base) {
    const int32_t nn = n_nodes(w);
    for (int32_t i = tid; i < nn; i += stride) {
        const int32_t c = w.nodes[i];
        const int32_t x = ldx<kL2>(w.comp2 + c);
        const unsigned long long hw = find_root(w.hook, x, nn);
        const int32_t root = hook_par(hw);
        if (root != x) {
            w.comp2[c] = root;
            w.kk2[c] = ldx<kL2>(w.kk2 + c) + hook_sh(hw);
            if (x == c) atomicMin(w.minpix + root, ldx<kL2>(w.minpix + c));  // nobody hands pixels to a hooked root
        }
    }
    const uint4* ein = (r & 1) ? w.edges2 : w.edges;
    uint4* eout = (r & 1) ? w.edges : w.edges2;
    const int32_t ne = r == 0 ? n_edges(w) : ldx<kL2>(w.ecount + r);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int32_t b0 = tid - (int32_t)threadIdx.x; b0 < ne; b0 += stride) {
        const int32_t i = b0 + threadIdx.x;
        bool keep = false;
        uint4 rc = make_uint4(0u, 0u, 0u, 0u);
        if (i < ne) {
            rc = ldx<kL2>(ein + i);
            if (rc.w & 0x80000000u) {  // an edge out of a tile as its tile listed it: completed once
                const int32_t p = (int32_t)(rc.x >> 1), q = (int32_t)(rc.w & 0x7fffffffu);
                rc.y = __float_as_uint(__fadd_rn(w.rel[p], w.rel[q]));
                rc.w = (uint32_t)w.comp[q];
            }
            const int32_t cp = hook_par(find_root(w.hook, ldx<kL2>(w.comp2 + rc.z), nn));
            const int32_t cq = hook_par(find_root(w.hook, ldx<kL2>(w.comp2 + rc.w), nn));
            keep = cp != cq;
            if (keep) {
                const unsigned long long key =
                    ((unsigned long long)rc.y << 32) | (unsigned long long)(0xffffffffu - rc.x);
                offer(best + cp, key);
                offer(best + cq, key);
            }
        }
        const unsigned kept = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_wcnt[wid] = __popc(kept);
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int k = 0; k < kUwThreads / 32; ++k) {
                const int32_t v = s_wcnt[k];
                s_wcnt[k] = tot;
                tot += v;
            }
            *s_base = tot ? atomicAdd(w.ecount + r + 1, tot) : 0;
        }
        __syncthreads();
        if (keep) eout[*s_base + s_wcnt[wid] + __popc(kept & ((1u << lane) - 1u))] = rc;
        __syncthreads();  // s_wcnt and s_base are reused by the next pass
    }
}

// Round r, hook: every root hooks onto the component across its best edge (hook = (parent,
// shift); of two roots that chose the same edge the smaller stays) and clears its slot of
// best[(r + 1) & 1] for the next round (its roots are among this round's); flags[r + 1] = 1 if any
// root hooked.
template <bool kL2>
__device__ __forceinline__ void hook_round(const UwArgs& a, const UwWork& w, const unsigned long long* best,
                                           unsigned long long* best_next, int r, int32_t tid, int32_t stride) {
    const int32_t n = n_nodes(w);
    for (int32_t i = tid; i < n; i += stride) {
        const int32_t rt = w.nodes[i];
        if (ldx<kL2>(w.comp2 + rt) != rt) continue;  // not a root
        const unsigned long long key = ldx<kL2>(best + rt);
        best_next[rt] = 0ull;
        if (!key) continue;
        const uint32_t e = key_edge(key);
        const int32_t p = (int32_t)(e >> 1);
        const int32_t q = p + ((e & 1u) ? a.fr[w.fid[p]].W : 1);
        const int32_t lp = w.comp[p], lq = w.comp[q];
        const int32_t cp = ldx<kL2>(w.comp2 + lp), cq = ldx<kL2>(w.comp2 + lq);
        const int32_t other = cp == rt ? cq : cp;
        if (ldx<kL2>(best + other) == key && rt < other) continue;  // both chose this edge: rt stays the root
        const int s = jump(w.wph[p], w.wph[q]);                        // k_q - k_p must equal s
        const int32_t kp = w.kk[p] + ldx<kL2>(w.kk2 + lp), kq = w.kk[q] + ldx<kL2>(w.kk2 + lq);
        w.hook[rt] = pack_hook(other, cq == rt ? kp + s - kq : kq - s - kp);
        w.flags[r + 1] = 1;
    }
}

// Round r as two launches (the rounds with most of the work: every CTA of a full grid on it).
// Both return at once when round r - 1 joined nothing (flags[r] == 0).
__global__ void __launch_bounds__(kUwThreads) uw_gscan(UwWork w, int r) {
    __shared__ int32_t s_wcnt[kUwThreads / 32];
    __shared__ int32_t s_base;
    if (!w.flags[r]) return;
    unsigned long long* best = w.best + (size_t)(r & 1) * (size_t)w.npx;
    scan_round<false>(w, best, r, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, s_wcnt, &s_base);
}
__global__ void __launch_bounds__(kUwThreads) uw_ghook(UwArgs a, UwWork w, int r) {
    if (!w.flags[r]) return;
    const unsigned long long* best = w.best + (size_t)(r & 1) * (size_t)w.npx;
    unsigned long long* best_next = w.best + (size_t)((r + 1) & 1) * (size_t)w.npx;
    hook_round<false>(a, w, best, best_next, r, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kWaitNs = 500ull * 1000ull * 1000ull;  // a grid-wide wait gives up after 0.5 s
constexpr unsigned int kWaitSpins = 1u << 24;                        // ... or after this many polls

// Grid-wide barrier of the cooperative kernel uw_gtail: every CTA adds one to *ctr, the last one
// to arrive (the barrier's index times the grid) publishes the index in *gen, on its own cache
// line, and the others wait for it there. The wait is bounded: a CTA that gives up sets *stop
// (counting the first give-up in *timeouts) and returns false, and so does every CTA that finds
// *stop set while it waits, so the whole grid leaves the kernel at its next barrier at the latest.
// Returns true when every CTA has arrived; their writes before it are then visible.
__device__ bool grid_barrier(unsigned int* ctr, unsigned int* gen, unsigned int target, int32_t* stop,
                             unsigned long long* timeouts) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int old = atomicAdd(ctr, 1u);
        if (old + 1u == target) atomicExch(gen, target);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        for (unsigned int it = 0; ld_acquire(gen) < target; ++it) {
            if (*(volatile int32_t*)stop) {
                ok = 0;
                break;
            }
            if (it >= kWaitSpins || global_ns() - t0 > kWaitNs) {
                if (atomicExch(stop, 1) == 0 && timeouts) atomicAdd(timeouts, 1ull);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Rounds r0 .. rounds - 1 in one cooperative launch (every CTA resident), the two halves of each
// round separated by grid barriers: the tail of rounds with little work left, where separate
// launches would cost more than the work. Returns at once when round r0 - 1 joined nothing, and
// after the first round that joins nothing (every CTA reads the same flag after the same barrier).
__global__ void __launch_bounds__(kUwThreads) uw_gtail(UwArgs a, UwWork w, int r0, int rounds) {
    __shared__ int32_t s_wcnt[kUwThreads / 32];
    __shared__ int32_t s_base;
    const int32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    unsigned int target = 0;
    for (int r = r0; r < rounds; ++r) {
        if (!ldx<true>(w.flags + r)) return;
        unsigned long long* best = w.best + (size_t)(r & 1) * (size_t)w.npx;
        unsigned long long* best_next = w.best + (size_t)((r + 1) & 1) * (size_t)w.npx;
        scan_round<true>(w, best, r, tid, stride, s_wcnt, &s_base);
        target += gridDim.x;
        if (!grid_barrier(w.sync, w.sync + 32, target, w.stop, a.timeouts)) return;
        hook_round<true>(a, w, best, best_next, r, tid, stride);
        target += gridDim.x;
        if (!grid_barrier(w.sync, w.sync + 32, target, w.stop, a.timeouts)) return;
    }
}

// After the rounds, for every listed local root r: ka[r] = its shift to its final root minus the k
// of that root's anchor (its smallest pixel), so that a pixel's k relative to the anchor is
// kk[g] + ka[comp[g]]. (Local roots outside the list got their ka in the tile kernel.)
__global__ void __launch_bounds__(kUwThreads) uw_anchor(UwWork w) {
    const int32_t nn = n_nodes(w);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const int32_t r = w.nodes[i];
        const unsigned long long hw = find_root(w.hook, w.comp2[r], nn);  // the comp2 itself once relabelled
        const int32_t m = w.minpix[hook_par(hw)];
        const int32_t lm = w.comp[m];
        const unsigned long long hm = find_root(w.hook, w.comp2[lm], nn);
        w.ka[r] = w.kk2[r] + hook_sh(hw) - (w.kk[m] + w.kk2[lm] + hook_sh(hm));
    }
}

// phi + 2 pi (k - k at the region's first pixel)
__global__ void __launch_bounds__(kUwThreads) uw_write(UwArgs a, UwWork w) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.npx; g += (int64_t)gridDim.x * blockDim.x) {
        const FrameDev& F = a.fr[w.fid[g]];
        const int64_t local = g - (int64_t)F.gam_off;
        const float p = w.wph[g];
        float v = p;
        if (!isnan(p)) {
            const int32_t k = w.kk[g] + w.ka[w.comp[g]];
            v = __fadd_rn(p, __fmul_rn(kTwoPiF, (float)k));
        }
        a.out[F.out_off + a.out_maps * (int64_t)F.H * F.W + local] = v;
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

UwWork carve(void* base, int64_t npx, int rounds) {
    UwWork w;
    char* p = static_cast<char*>(base);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += align256(bytes);
        return r;
    };
    const size_t n = (size_t)npx;
    w.best = reinterpret_cast<unsigned long long*>(take(16 * n));
    w.hook = reinterpret_cast<unsigned long long*>(take(8 * n));
    w.edges = reinterpret_cast<uint4*>(take(32 * n));
    w.edges2 = reinterpret_cast<uint4*>(take(32 * n));
    w.wph = reinterpret_cast<float*>(take(4 * n));
    w.rel = reinterpret_cast<float*>(take(4 * n));
    w.fid = reinterpret_cast<int32_t*>(take(4 * n));
    w.comp = reinterpret_cast<int32_t*>(take(4 * n));
    w.kk = reinterpret_cast<int32_t*>(take(4 * n));
    w.minpix = reinterpret_cast<int32_t*>(take(4 * n));
    w.comp2 = reinterpret_cast<int32_t*>(take(4 * n));
    w.kk2 = reinterpret_cast<int32_t*>(take(4 * n));
    w.ka = reinterpret_cast<int32_t*>(take(4 * n));
    w.nodes = reinterpret_cast<int32_t*>(take(4 * n));
    w.tile_start = reinterpret_cast<int32_t*>(take(4 * (n + 2)));  // a call has at most npx frames
    w.counts = reinterpret_cast<unsigned long long*>(take(8));
    w.sync = reinterpret_cast<unsigned int*>(take(256));
    w.stop = reinterpret_cast<int32_t*>(w.sync + 1);
    w.npx = npx;
    w.flags = reinterpret_cast<int32_t*>(take(4 * (size_t)(rounds + 1)));
    w.ecount = reinterpret_cast<int32_t*>(take(4 * (size_t)(rounds + 1)));
    return w;
}

int ceil_log2(int64_t n) {
    int r = 0;
    while (((int64_t)1 << r) < n) ++r;
    return r;
}

}  // namespace

int unwrap_rounds(int64_t max_frame_nodes) { return ceil_log2(max_frame_nodes < 2 ? 2 : max_frame_nodes) + 1; }

int64_t unwrap_frame_nodes(int H, int W) {
    // the global phase's components of a frame are local roots on a tile's border: at most the
    // 4 * 32 - 4 border pixels of each 32 x 32 tile, and never more than the frame's pixels
    const int64_t tiles = (int64_t)((H + kTile - 1) / kTile) * ((W + kTile - 1) / kTile);
    const int64_t px = (int64_t)H * W, b = tiles * (4 * kTile - 4);
    return b < px ? b : px;
}

size_t unwrap_workspace_bytes(int64_t npx, int64_t max_frame_nodes) {
    const int R = unwrap_rounds(max_frame_nodes);
    const size_t n = (size_t)npx;
    return align256(16 * n) + align256(8 * n) + 2 * align256(32 * n) + 10 * align256(4 * n) + align256(4 * (n + 2)) +
           align256(8) + align256(256) + 2 * align256(4 * (size_t)(R + 1));
}

cudaError_t launch_unwrap(const FrameDev* d_frames, int nframes, int64_t npx, int64_t max_frame_nodes,
                          const float* in, int64_t in_maps, float* out, int64_t out_maps, void* work,
                          int launched_rounds, unsigned long long* timeouts, int* launches, cudaStream_t s) {
    if (npx <= 0 || nframes <= 0) return cudaSuccess;
    const int R = unwrap_rounds(max_frame_nodes);
    UwWork w = carve(work, npx, R);
    UwArgs a{d_frames, nframes, npx, in, in_maps, out, out_maps, timeouts};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (npx + kUwThreads - 1) / kUwThreads;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    // persistent over the tiles (their count is known on the device only): no more CTAs than the
    // tiles of a call can need, about npx / 32 + nframes at most
    const int64_t tiles_max = npx / kTile + nframes;
    const unsigned tgrid = (unsigned)(tiles_max < (int64_t)sms * 4 ? tiles_max : (int64_t)sms * 4);
    // the global rounds: at most two listed edges per pixel
    const int64_t ewant = (2 * npx + kUwThreads - 1) / kUwThreads;
    const unsigned egrid = (unsigned)(ewant < (int64_t)sms * 8 ? ewant : (int64_t)sms * 8);
    // The first half of the rounds bound as separate launches (each round at least halves the
    // components that still have edges, but typically does much more, so the work is in the first
    // rounds); the rest in one cooperative launch that stops after the first round that joins
    // nothing (usually at once), every CTA resident.
    const int R1 = launched_rounds < 0 ? (R + 1) / 2 : (launched_rounds < R ? launched_rounds : R);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, uw_gtail, kUwThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const int64_t twant = ewant < (int64_t)sms * per_sm ? ewant : (int64_t)sms * per_sm;
    uw_prepare<<<1, kUwThreads, 0, s>>>(a, w, R);
    uw_init<<<grid, kUwThreads, 0, s>>>(a, w.wph, w.fid, w.rel);
    e = cudaFuncSetAttribute(uw_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    if (e != cudaSuccess) return e;
    uw_tiles<<<tgrid, kUwThreads, kTileSmem, s>>>(a, w);
    *launches += 3;
    for (int r = 0; r < R1; ++r) {
        uw_gscan<<<egrid, kUwThreads, 0, s>>>(w, r);
        uw_ghook<<<grid, kUwThreads, 0, s>>>(a, w, r);
        *launches += 2;
    }
    if (R1 < R) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)twant);
        cfg.blockDim = dim3(kUwThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, uw_gtail, a, w, R1, R);
        if (e != cudaSuccess) return e;
        *launches += 1;
    }
    uw_anchor<<<grid, kUwThreads, 0, s>>>(w);
    uw_write<<<grid, kUwThreads, 0, s>>>(a, w);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace rmusic
