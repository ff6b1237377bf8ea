// square_kernel.cuh -- FP32 solver for the paper's own geometry: the M x M block Gamma_w,
// M = 2 Lp + 1, centred on each pixel (Sec. 3, Eq. 4-15; Algorithm 1). Both local phase
// derivatives and the local phase alpha come out of one block:
//   R_y = Gamma_w Gamma_w^H  (the block's columns are the snapshots), u1 its signal eigenvector,
//   R_x = Gamma_w^H Gamma_w  (the conjugated rows), v1 its signal eigenvector,
//   Q_y, Q_x the root-MUSIC polynomials of u1 and v1 (Eq. 12, 13), z_y, z_x their roots nearest
//   the unit circle inside it, omega_y = arg z_y, omega_x = -arg z_x, and
//   alpha = angle of the block mean of Gamma_w exp(-j(omega_x x + omega_y y)) (Eq. 15), with
//   x, y centred on the pixel.
//
// Work decomposition: one thread per pixel; each CTA of a persistent grid takes four consecutive
// items from a global atomic counter, one per warp -- an item is a 32 x 8 strip of pixels, or, once
// every frame's strips are taken, one 32-pixel row of a frame's last eighth (short items at the
// end, so that the warps finish within about one row of each other). Each warp stages its item's
// (32 + 2 Lp) x (rows + 2 Lp) analytic-signal samples in its own part of shared memory with
// coalesced loads and walks its rows top to bottom, each lane reading its block from there; the
// CTA's warps take each row in step (a barrier per row), so that they run the same code at the
// same time (the kernel is bound by instruction fetch: 1.5 % faster than warps left to drift). Items sit at absolute positions of their frame, so the warps
// -- and with them every warp-level iteration count and every start vector -- are the same
// whether a frame runs alone or batched.
//
// Eigenvectors: u1 and v1 are the first left and right singular vectors of Gamma_w (the paper
// takes them from an SVD), computed by the power iteration u <- G G^H u / |.| on the block itself
// (two M x M products per step, no M x M covariance is formed). The first row of a strip starts
// from the centre column; a row below a usable block starts from G v1 of the row above (the
// block moves down one row, so v1, over its columns, barely moves: at 0 dB 5.7 steps per row on
// average instead of 7.5 from the centre column). The vectors live in shared memory (one column per thread) and the
// loops over rows are rolled, so only one M-vector is held in registers.
// Each step shrinks the other singular directions by (s_2 / s_1)^2 ~ 4 sigma^2 / (M A^2), or,
// with the shift by twice the mean noise eigenvalue that the kernel applies from the first step,
// by about half of that; the iteration stops when the step changes u by less than 3e-5 in every
// lane of the warp. v1 is G^H u from the last step. Degenerate blocks (all zero) get a stand-in vector so every lane of
// the warp runs the same bounded loops.
//
// Polynomials: the root stage of roots_device.cuh (coefficients, the signal root by Newton's
// method with a Schur-Cohn certificate -- Aberth on all inner roots where it fails -- and the
// polish) with L = M, run once per axis in one rolled loop that reads the axis' vector (u1 or v1)
// from shared memory, which keeps the code within the instruction cache.
#pragma once

#include <math.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"
#include "roots_device.cuh"

namespace rmusic {

constexpr int kSqThreads = kSqTX * kSqWarps;

// Dynamic shared memory of square_kernel<LP>: per warp its strip's staged samples
// ((kSqTY + 2 LP) x (kSqTX + 2 LP) float2), per thread two M-vectors of float2 (the scratch), per
// warp its statistics.
__host__ __device__ constexpr int square_stage_elems(int LP) { return (kSqTY + 2 * LP) * (kSqTX + 2 * LP); }
__host__ __device__ constexpr size_t square_smem_bytes(int LP) {
    return (size_t)kSqWarps * square_stage_elems(LP) * 8 + (size_t)2 * (2 * LP + 1) * kSqThreads * 8 +
           (size_t)kSqWarps * kStatSlots * 8;
}

template <int LP, int CTAS>
__global__ void __launch_bounds__(kSqThreads, CTAS)
square_kernel(const FrameDev* __restrict__ fr, int nframes, int64_t total_items,
              unsigned long long* __restrict__ counter, const float2* __restrict__ gam,
              float* __restrict__ out, uint8_t* __restrict__ status, SquareArgs args) {
    static_assert(LP >= 1 && 2 * LP + 1 <= 2 * kMaxSquareLp + 1, "half-width out of range");
    constexpr int M = 2 * LP + 1;
    constexpr int SW = kSqTX + 2 * LP;     // staged columns
    constexpr int NST = square_stage_elems(LP);
    extern __shared__ __align__(16) unsigned char sq_smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* const tile = reinterpret_cast<float2*>(sq_smem) + wid * NST;  // this warp's strip
    // per-thread scratch, two float2 M-vectors: the power iteration's pair; afterwards u1 (the
    // last iterate) and v1 (G^H of the one before), which the next row of the strip starts from
    float2* const scr = reinterpret_cast<float2*>(sq_smem) + kSqWarps * NST;
    // this warp's iteration statistics, flushed to args.counters once when the warp leaves its loop
    unsigned long long* const stat =
        reinterpret_cast<unsigned long long*>(scr + 2 * M * kSqThreads) + wid * kStatSlots;
    if (lane < kStatSlots) stat[lane] = 0ull;
    const float tol2 = args.tol2;
    float2* const vec0 = scr + threadIdx.x;  // entry m at [m * kSqThreads]
    float2* const vec1 = vec0 + M * kSqThreads;

    __shared__ long long sh_item;
    for (;;) {
        __syncthreads();  // every warp is done with its previous item
        if (threadIdx.x == 0) sh_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        if (sh_item * kSqWarps >= total_items) break;
        const long long item = sh_item * kSqWarps + wid;
        const bool active = item < total_items;
        // a strip (the first fr[0].item_start2 items) or one row of a frame's last rows
        const bool strip = item < fr[0].item_start2;
        const int f = strip ? find_frame(fr, nframes, (int64_t)item, [](const FrameDev& F) { return F.item_start; })
                            : find_frame(fr, nframes, (int64_t)item, [](const FrameDev& F) { return F.item_start2; });
        const FrameDev& F = fr[f];
        const int64_t local = (int64_t)item - (strip ? F.item_start : F.item_start2);
        // a frame's items number below 2^31: 32-bit division (a 64-bit one is a long routine)
        const int q = (int)((uint32_t)local / (uint32_t)F.nchunks);
        const int tx = (int)((uint32_t)local % (uint32_t)F.nchunks);
        const int row0 = strip ? q * kSqTY : F.sq_strip_rows + q;
        int nrows = !active ? 0 : strip ? kSqTY : 1;
        const int H = F.H, W = F.W;
        // every index below follows from these (the staged rows and each lane's block inside them
        // have compile-time extents); checked builds test them and skip a bad item whole (the item
        // is the warp's, so the skip is uniform)
        if (active && !rm_check(f >= 0 && f < nframes && local >= 0 && F.L == LP && F.sq_strip_rows % kSqTY == 0 &&
                          (strip ? local < (int64_t)(F.sq_strip_rows / kSqTY) * F.nchunks
                                 : local < (int64_t)(H - F.sq_strip_rows) * F.nchunks),
                      args.counters))
            nrows = 0;

        // ---- stage the item's samples (coalesced rows) -----------------------------------------
        if (nrows > 0) {
            const int x0 = tx * kSqTX - LP, y0 = row0 - LP;
            // the analytic signal: the workspace (row-major, W per row), or a complex64 frame in place
            const float2* g = args.direct ? reinterpret_cast<const float2*>(args.direct + F.in_off) : gam + F.gam_off;
            const int64_t pitch = args.direct ? (int64_t)F.pitch : (int64_t)W;
            const int nst = (nrows + 2 * LP) * SW;
#pragma unroll 4
            for (int i = lane; i < nst; i += 32) {
                const int r = i / SW, c = i - r * SW;
                const int gy = y0 + r, gx = x0 + c;
                tile[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? g[(int64_t)gy * pitch + gx]
                                                                     : make_float2(0.f, 0.f);
            }
        }
        __syncwarp();
        const int px = tx * kSqTX + lane;
        // v1 of the row above, in the scratch vector `carry` (valid when prev_ok)
        bool prev_ok = false;
        float2* carry = vec1;
#pragma unroll 1
        for (int k = 0; k < kSqTY; ++k) {
            __syncthreads();  // the CTA's warps walk their rows in step: one code region at a time
            if (k >= nrows) continue;
            const int py = row0 + k;
            const bool inside = px < W && py < H;
            const bool valid = inside && px - LP >= 0 && px + LP < W && py - LP >= 0 && py + LP < H;
            const float2* Gb = tile + k * SW + lane;  // block entry (r, c) at Gb[r * SW + c]
            auto G = [&](int r, int c) {
                const float2 v = Gb[r * SW + c];
                return mkc(v.x, v.y);
            };

            // ---- power iteration for u1 (and v1) --------------------------------------------------
            // u (unit norm) lives in one scratch vector, G y is written to the other, then the roles
            // swap. Start: below a row whose block was usable, u = G v1 of that row normalised (the
            // block has moved down by one row, its right singular vector barely moves); otherwise
            // the centre column.
            float nu2 = 0.f;
#pragma unroll 1
            for (int m = 0; m < M; ++m) nu2 += norm2(G(m, LP));
            const bool nonzero = valid && nu2 > 0.f && isfinite(nu2);
            const bool warm = nonzero && prev_ok;
            float2* uv = carry == vec0 ? vec1 : vec0;
            float2* wv = carry;
            cx<float> y[M];
            bool started = false;
            if (warm) {
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const float2 v = carry[c * kSqThreads];
                    y[c] = mkc(v.x, v.y);
                }
                float n2 = 0.f;
#pragma unroll 1
                for (int m = 0; m < M; ++m) {
                    cx<float> a = mkc(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        const cx<float> g = G(m, c);  // (G v)_m
                        a = mkc(fmaf(g.r, y[c].r, fmaf(-g.i, y[c].i, a.r)), fmaf(g.r, y[c].i, fmaf(g.i, y[c].r, a.i)));
                    }
                    uv[m * kSqThreads] = make_float2(a.r, a.i);
                    n2 += norm2(a);
                }
                if (n2 > 0.f && isfinite(n2)) {
                    const float inv = rsqrtf(n2);
#pragma unroll 1
                    for (int m = 0; m < M; ++m) {
                        const float2 v = uv[m * kSqThreads];
                        uv[m * kSqThreads] = make_float2(inv * v.x, inv * v.y);
                    }
                    started = true;
                }
            }
            if (!started) {
                const float inv = nonzero ? rsqrtf(nu2) : 0.f;
#pragma unroll 1
                for (int m = 0; m < M; ++m) {
                    const cx<float> g = G(m, LP);
                    uv[m * kSqThreads] = make_float2(inv * g.r, inv * g.i);
                }
            }
            const bool warm_any = __any_sync(kFull, started);
            // trace of G G^H: the sum of its eigenvalues, for the shift below
            float tr = 0.f;
#pragma unroll 1
            for (int m = 0; m < M; ++m) {
#pragma unroll
                for (int c = 0; c < M; ++c) tr += norm2(G(m, c));
            }
            bool pconv = !nonzero;
            int pits = 0;
            float sig = 0.f;
            for (;;) {
                // y = G^H u
#pragma unroll
                for (int c = 0; c < M; ++c) y[c] = mkc(0.f, 0.f);
#pragma unroll 1
                for (int m = 0; m < M; ++m) {
                    const float2 um = uv[m * kSqThreads];
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        const cx<float> g = G(m, c);  // y_c += conj(g) u_m
                        y[c] = mkc(fmaf(g.r, um.x, fmaf(g.i, um.y, y[c].r)), fmaf(g.r, um.y, fmaf(-g.i, um.x, y[c].i)));
                    }
                }
                if (pits == 0) {
                    // Shift: iterate with G G^H - sig I, which shrinks the noise directions by
                    // (l_i - sig) / (l_1 - sig) instead of l_i / l_1. The noise eigenvalues of a
                    // square block spread over about [0, 4 mean], so sig = 2 mean centres them; the
                    // mean comes from the trace and the Rayleigh quotient |G^H u|^2 <= l_1. sig stays
                    // below l_1 / 4, so the signal direction keeps the largest |l - sig|.
                    float rho = 0.f;
#pragma unroll
                    for (int c = 0; c < M; ++c) rho += norm2(y[c]);
                    const float mean_noise = fmaxf(tr - rho, 0.f) * (1.f / (float)(M - 1));
                    sig = fminf(2.f * mean_noise, 0.25f * rho);
                }
                // w = G y - sig u
                float n2 = 0.f;
#pragma unroll 1
                for (int m = 0; m < M; ++m) {
                    const float2 um = uv[m * kSqThreads];
                    cx<float> a = mkc(-sig * um.x, -sig * um.y);
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        const cx<float> g = G(m, c);  // w_m += g y_c
                        a = mkc(fmaf(g.r, y[c].r, fmaf(-g.i, y[c].i, a.r)), fmaf(g.r, y[c].i, fmaf(g.i, y[c].r, a.i)));
                    }
                    wv[m * kSqThreads] = make_float2(a.r, a.i);
                    n2 += norm2(a);
                }
                // normalise w, measure the step |w - u|^2, swap
                const float inv = n2 > 0.f ? rsqrtf(n2) : 0.f;
                float d2 = 0.f;
#pragma unroll 1
                for (int m = 0; m < M; ++m) {
                    const float2 w = wv[m * kSqThreads], u = uv[m * kSqThreads];
                    const float2 nw = make_float2(inv * w.x, inv * w.y);
                    d2 += (nw.x - u.x) * (nw.x - u.x) + (nw.y - u.y) * (nw.y - u.y);
                    wv[m * kSqThreads] = nw;
                }
                float2* t = uv;
                uv = wv;
                wv = t;
                pconv = pconv || d2 <= tol2;
                ++pits;
                if (pits >= args.max_power_iters) break;
                if (__all_sync(kFull, pconv)) break;
            }
            // u1 stays in uv; v1 = y (G^H of the last step's start) goes to the other vector, where
            // the root stage reads it and the next row starts from it
            if (!nonzero) {
                // stand-in: the noise-free vector of angle 0, so the root stage runs its short path
#pragma unroll 1
                for (int m = 0; m < M; ++m) uv[m * kSqThreads] = make_float2(1.f, 0.f);
#pragma unroll
                for (int m = 0; m < M; ++m) y[m] = mkc(1.f, 0.f);
            }
#pragma unroll
            for (int c = 0; c < M; ++c) wv[c * kSqThreads] = make_float2(y[c].r, y[c].i);
            carry = wv;
            prev_ok = nonzero;

            // Newton's starting radius. (A start fitted to the noise's share of the block's energy, as
            // on row windows, measured 30 % fewer Newton steps but twice the Aberth fallbacks at 0 dB,
            // and near ties between roots then went the other way in FP32 more often than the tests
            // allow.)
            const float r0 = 0.99f;

            // ---- roots, selection and angle: axis 0 is y (u1, z_y), axis 1 is x (v1, z_x) ---------
            float om_y = 0.f, om_x = 0.f;
            bool rconv_all = true, found_all = true;
            int riters = 0, revals = 0, rupdates = 0, rnewton = 0, rfallback = 0, rpolish = 0;
#pragma unroll 1
            for (int ax = 0; ax < 2; ++ax) {
                const float2* src = ax == 0 ? uv : wv;
                cx<float> c[M];
                float res2;
                {
                    cx<float> vr[M];
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const float2 v = src[m * kSqThreads];
                        vr[m] = mkc(v.x, v.y);
                    }
                    res2 = music_coefs<M>(vr, c);
                }
                bool rconv, found, cluster;
                RootStats rs;
                const cx<float> zz = signal_root<M>(c, res2, args.max_iters, args.exhaustive, nonzero, r0, found,
                                                    cluster, rconv, rs);
                const float a = args.polish64 ? (float)polish_arg64<M>(c, zz, cluster) : atan2f(zz.i, zz.r);
                if (ax == 0)
                    om_y = a;
                else
                    om_x = -a;  // z_x = exp(-j omega_x) (Eq. 15)
                rconv_all = rconv_all && rconv;
                found_all = found_all && found;
                riters += rs.iters;
                revals += rs.evals;
                rupdates += rs.updates;
                rnewton += rs.newton;
                rfallback += rs.fallback;
                rpolish += rs.polish;
            }

            // ---- alpha: angle of the demodulated block mean (Eq. 15) ------------------------------
            // exp(-j omega (k - Lp)) for k = 0 .. M-1 by recurrence from exp(j omega Lp)
            cx<float> ex[M];
            {
                float s1, c1, s0, c0;
                sincosf(om_x, &s1, &c1);
                sincosf(om_x * (float)LP, &s0, &c0);
                const cx<float> e1 = mkc(c1, -s1);
                ex[0] = mkc(c0, s0);
#pragma unroll
                for (int c = 1; c < M; ++c) ex[c] = ex[c - 1] * e1;
            }
            cx<float> acc = mkc(0.f, 0.f);
            {
                float s1, c1, s0, c0;
                sincosf(om_y, &s1, &c1);
                sincosf(om_y * (float)LP, &s0, &c0);
                const cx<float> e1 = mkc(c1, -s1);
                cx<float> ey = mkc(c0, s0);
#pragma unroll 1
                for (int r = 0; r < M; ++r) {
                    cx<float> t = mkc(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < M; ++c) t = t + G(r, c) * ex[c];
                    acc = acc + t * ey;
                    ey = ey * e1;
                }
            }

            if (lane == 0 && args.counters) {
                stat[2] += 1ull;
                stat[0] += (unsigned long long)pits;
                stat[1] += (unsigned long long)riters;
                stat[3] += (unsigned long long)rupdates;
                stat[4] += (unsigned long long)revals;
                stat[5] += warm_any ? 1ull : 0ull;
                stat[7] += (unsigned long long)rnewton;
                stat[8] += (unsigned long long)rfallback;
                stat[9] += (unsigned long long)rpolish;
            }

            // ---- store the three maps --------------------------------------------------------------
            if (inside) {
                const uint64_t o = F.out_off + (uint64_t)py * (uint64_t)W + (uint64_t)px;
                const uint64_t hw = (uint64_t)H * (uint64_t)W;
                uint8_t st = kStOk;
                if (!valid)
                    st = kStBorder;
                else if (!nonzero || !found_all)
                    st = kStDegenerate;
                else if (!pconv || !rconv_all)
                    st = kStNotConverged;
                const float w0 = (float)F.omega_ref;
                float dx = F.carrier_axis == 0 ? wrap_pi(om_x - w0) : wrap_pi(om_x);
                float dy = F.carrier_axis == 1 ? wrap_pi(om_y - w0) : wrap_pi(om_y);
                // carrier phase at the pixel: 2 pi frac(f0 X), X its coordinate along the carrier
                double t = F.f0 * (double)(F.carrier_axis == 0 ? px : py);
                t -= floor(t);
                float al = wrap_pi(atan2f(acc.i, acc.r) - (float)(6.283185307179586477 * t));
                if (st == kStBorder || st == kStDegenerate) {
                    const float qnan = __int_as_float(0x7fc00000);
                    dx = dy = al = qnan;
                }
                out[o] = dx;
                out[o + hw] = dy;
                out[o + 2 * hw] = al;
                if (status) status[o] = st;
            }
        }
    }
    __syncwarp();
    if (args.counters && lane < kStatSlots && stat[lane]) atomicAdd(args.counters + lane, stat[lane]);
}

}  // namespace rmusic
