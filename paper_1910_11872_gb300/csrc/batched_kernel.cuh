// batched.cu -- the FP32 batched path: one persistent kernel over every pixel of every frame of
// a call (frames of uneven sizes and windows mixed), one window-line run of 32 P consecutive pixels
// per warp work item, P consecutive pixels per lane (P = 16, or 8 on lines where that leaves fewer
// lanes idle: a property of the frame), items taken from a global atomic counter.
//
// Per warp item (a run of one window line; lane l owns pixels l P .. l P + P - 1):
//   stage     the 32 P + N - 1 analytic-signal samples the run's windows cover, one coalesced read
//             into shared memory (Sec. 3, Eq. 2: the moving window), padded by one sample every P
//             so that the lanes' strided reads fall in distinct banks
//   S         with forward-backward averaging R = (R_f + J conj(R_f) J)/2 is centro-Hermitian,
//             so with the unitary Q = [[I, jI], [J, -jJ]] / sqrt(2) (even L) S = Q^H R Q =
//             Re(Q^H R_f Q) is real symmetric; R u = l u  <=>  S x = l x with u = Q x. Written out,
//             S = sum over the window's K = N - L + 1 snapshots s_j (Eq. 4-5) of X_j X_j^T + Y_j Y_j^T
//             with the real L-vectors X_j = [Re p, Im q], Y_j = [Im p, -Re q] of the folded snapshot
//             p_i = s_j[i] + s_j[L-1-i], q_i = s_j[i] - s_j[L-1-i] (i < L/2). A lane sums the K rank-2
//             terms of its first pixel's window (its anchor, at an absolute position of the line) and
//             moves to each next pixel by one sliding update: + the entering snapshot's rank-2 term
//             - the leaving one's (4 L(L+1)/2 multiply-adds). Anchors sit at fixed positions, so
//             each pixel's arithmetic does not depend on how frames are batched or scheduled.
//   eigen     the signal eigenvector x1 of S (Eq. 8-11) by the shifted power iteration, from the
//             column of S with the largest diagonal entry (2-3 steps on signal-dominated windows);
//             lanes whose iteration does not settle or whose eigen-gap is not certified by the
//             Frobenius bound |l2| <= sqrt(|S|_F^2 - l1^2) take cyclic Jacobi sweeps on S (real,
//             register resident, tournament order) and three steps of inverse iteration.
//   poly,     u1 = Q x1; the root-MUSIC coefficients; the root nearest the unit circle inside it,
//   roots,    by Newton's method with a Schur-Cohn certificate (full Aberth-Ehrlich when the
//   select    certificate fails), and its polish (roots_device.cuh, shared with the square-block
//             solver).
//   angle     atan2 of the root minus the carrier step, wrapped (Eq. 15).
// This header holds the kernel template; batched_l*.cu instantiate it for each covariance order
// and register-cap variant (compiled in parallel), batched.cu dispatches among them.
#pragma once

#include <math.h>

#include "batched_variants.h"
#include "rmusic_device.cuh"
#include "rmusic_launch.h"
#include "roots_device.cuh"

namespace rmusic {

constexpr int kBatWarps = 4;
constexpr int kBatThreads = kBatWarps * 32;
// staged samples of one run: 32 P + N - 1 <= 32 P + kMaxN - 1, plus one pad every P, for P = 16 and 8
constexpr int seg_len(int P) { return 32 * P + kMaxN + (32 * P + kMaxN) / P; }
constexpr int kSegLen = seg_len(kRowP) > seg_len(kRowPMin) ? seg_len(kRowP) : seg_len(kRowPMin);
static_assert(kRowP == 2 * kRowPMin, "the frames' pixels per lane are 16 or 8");

// Shared-memory slot of staged sample e of a run with P = 1 << ps pixels per lane (one pad slot after
// every P samples): lane l's sample i is e = l P + i at (P + 1) l + i + i / P, so 32 lanes reading
// their own sample i touch 32 slots P + 1 apart -- 16 distinct 8-byte bank pairs (P + 1 is odd),
// each read by two lanes (the two wavefronts a 64-bit load takes anyway).
__device__ __forceinline__ int seg_slot(int e, int ps) { return e + (e >> ps); }

__host__ __device__ constexpr int tri(int r, int c, int L) {
    return r <= c ? r * L - (r * (r - 1)) / 2 + (c - r) : c * L - (c * (c - 1)) / 2 + (r - c);
}

// Fixed relabeling of the Jacobi tournament: after a step over the pairs (0,1), (2,3), ...,
// position p takes the index previously at tperm(p). Over L - 1 steps every pair of indices
// meets once (the circle method: 0 stays, the others move around a ring).
__host__ __device__ constexpr int tperm(int p, int L) {
    return p == 0 ? 0 : (p == 1 ? (L > 2 ? 2 : 1) : (p % 2 == 1 ? p - 2 : (p == L - 2 ? L - 1 : p + 2)));
}

__device__ __forceinline__ cx<float> shfl_up_c(cx<float> v, int o) {
    return mkc(__shfl_up_sync(kFull, v.r, o), __shfl_up_sync(kFull, v.i, o));
}

// Add entry (r, s) of R_f (value v) to S = Re(Q^H R_f Q) up to the factor 1/2, with the
// unitary Q = [[I, jI], [J, -jJ]] / sqrt(2) of even order L = 2h. Writing R_f in h x h blocks,
// with i = fold(r), k = fold(s) (fold(t) = t for t < h, L - 1 - t otherwise):
//   S11[i][k] =  Re(a + b + c + d),  S22[i][k] = Re(a - b - c + d),  S12[i][k] = -Im(a - b + c - d)
// where a, b, c, d are the entries (i, k), (i, L-1-k), (L-1-i, k), (L-1-i, L-1-k). Only the upper
// triangles of the symmetric blocks S11, S22 are kept (i <= k); S12 is kept whole.
template <int L>
__device__ __forceinline__ void accumulate_s(float* S, int r, int s, cx<float> v) {
    constexpr int h = L / 2;
    const int i = r < h ? r : L - 1 - r;
    const int k = s < h ? s : L - 1 - s;
    if (s < h)
        S[tri(i, h + k, L)] -= v.i;
    else
        S[tri(i, h + k, L)] += v.i;
    if (i <= k) {
        S[tri(i, k, L)] += v.r;
        if ((r < h) == (s < h))
            S[tri(h + i, h + k, L)] += v.r;
        else
            S[tri(h + i, h + k, L)] -= v.r;
    }
}

// The eigenvalue sweeps of the 32 matrices of a warp item done by the whole warp, one matrix at a
// time (the warp-per-matrix schedule): lane l holds entries (r, 2j) and (r, 2j + 1) of the full
// symmetric S of one pixel, r = l / (L/2), j = l % (L/2) (L <= 8: at most two entries per lane).
// A tournament step rotates the pairs (2k, 2k + 1) on both sides -- rows with the partner lane's
// values (one shuffle pair), columns within the lane -- with the angle computed from the pair's
// diagonal block (shuffled from the two lanes that hold it), then relabels rows and columns by
// tperm (shuffles from the source lanes). The stopping rule is the thread-per-matrix one, applied
// per matrix. Returns, in the caller's lane, l1, l2 and k1 of its own pixel (sh holds the parked
// S of all 128 pixels of the CTA, one column each, to be multiplied by the pixel's sh_sc).
template <int L>
__device__ __forceinline__ void warp_jacobi_item(const float* __restrict__ sh, const float* __restrict__ sh_sc,
                                                 int wid, int lane, int max_sweeps, float* res_l1, float* res_l2,
                                                 int* res_k1, int* res_sw, bool* res_conv) {
    static_assert(L * L <= 64, "two entries per lane at most");
    constexpr int hL = L / 2;
    const bool act = lane < L * hL;
    const int r = act ? lane / hL : 0, j = act ? lane % hL : 0;
    const int c0 = 2 * j;
    const int partner = act ? (r ^ 1) * hL + j : lane;
    for (int mat = 0; mat < 32; ++mat) {
        const float* Sm = sh + wid * 32 + mat;
        const float sc = sh_sc[wid * 32 + mat];
        float a0 = act ? sc * Sm[tri(r, c0, L) * kBatThreads] : 0.f;
        float a1 = act ? sc * Sm[tri(r, c0 + 1, L) * kBatThreads] : 0.f;
        int sweeps = 0;
        bool conv = false;
        float l1 = 0.f, l2 = 0.f;
        int k1 = 0;
        for (;;) {
#pragma unroll 1
            for (int stp = 0; stp < L - 1; ++stp) {
                // rotation of the row pair kr = r / 2 and of the column pair kc = j
                auto angle = [&](int k, float& c, float& s) {
                    const int lp = (2 * k) * hL + k, lq = (2 * k + 1) * hL + k;
                    const float app = __shfl_sync(kFull, a0, lp), apq = __shfl_sync(kFull, a1, lp);
                    const float aqq = __shfl_sync(kFull, a1, lq);
                    const float dq = aqq - app;
                    const float den = fabsf(dq) + sqrtf(fmaf(dq, dq, 4.f * apq * apq));
                    float t = den > 0.f ? __fdividef(2.f * apq, den) : 0.f;
                    t = dq < 0.f ? -t : t;
                    c = rsqrtf(fmaf(t, t, 1.f));
                    s = t * c;
                };
                float cr, sr, cc, sc;
                angle(r >> 1, cr, sr);
                angle(j, cc, sc);
                // rows: row_p' = c row_p - s row_q, row_q' = s row_p + c row_q
                const float b0 = __shfl_sync(kFull, a0, partner), b1 = __shfl_sync(kFull, a1, partner);
                if ((r & 1) == 0) {
                    a0 = fmaf(cr, a0, -sr * b0);
                    a1 = fmaf(cr, a1, -sr * b1);
                } else {
                    a0 = fmaf(sr, b0, cr * a0);
                    a1 = fmaf(sr, b1, cr * a1);
                }
                // columns: col_p' = c col_p - s col_q, col_q' = s col_p + c col_q
                const float n0 = fmaf(cc, a0, -sc * a1), n1 = fmaf(sc, a0, cc * a1);
                a0 = n0;
                a1 = n1;
                // relabel: new (r, c) is old (tperm(r), tperm(c))
                const int rr = tperm(r, L);
                const int s0 = tperm(c0, L), s1 = tperm(c0 + 1, L);
                const int lane0 = act ? rr * hL + (s0 >> 1) : lane, lane1 = act ? rr * hL + (s1 >> 1) : lane;
                const float x0 = __shfl_sync(kFull, a0, lane0), y0 = __shfl_sync(kFull, a1, lane0);
                const float x1 = __shfl_sync(kFull, a0, lane1), y1 = __shfl_sync(kFull, a1, lane1);
                a0 = act ? ((s0 & 1) ? y0 : x0) : 0.f;
                a1 = act ? ((s1 & 1) ? y1 : x1) : 0.f;
            }
            ++sweeps;
            // off-diagonal mass (upper triangle) and the two largest diagonal entries
            float off = 0.f, dg = -1e30f;
            int di = L;
            if (act) {
                if (c0 > r) off = fmaf(a0, a0, off);
                if (c0 + 1 > r) off = fmaf(a1, a1, off);
                if (c0 == r) {
                    dg = a0;
                    di = r;
                }
                if (c0 + 1 == r) {
                    dg = a1;
                    di = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(kFull, off, o);
            // largest diagonal entry, the smaller index on ties (as the sequential scan)
            float bv = dg;
            int bi = di;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(kFull, bv, o);
                const int oi = __shfl_xor_sync(kFull, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            float sv = di == bi ? -1e30f : dg;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sv = fmaxf(sv, __shfl_xor_sync(kFull, sv, o));
            l1 = bv;
            l2 = sv;
            k1 = bi;
            const float gap = l1 - l2;
            conv = off <= 1e-3f * gap * gap;
            if (sweeps >= max_sweeps || conv) break;
        }
        if (lane == mat) {
            *res_l1 = l1;
            *res_l2 = l2;
            *res_k1 = k1;
            *res_sw = sweeps;
            *res_conv = conv;
        }
    }
}

// Signal eigenvector x of the real-symmetric S (packed upper triangle, trace-normalised) by the
// shifted power iteration x <- (S - sig I) x / |.|, started from the column of S with the largest
// diagonal entry (for a rank-one S that column is already the eigenvector; read from the parked
// column, any positive multiple of S; inactive lanes, whose S is a diagonal stand-in, start from the
// unit vector of that entry). The shift
// sig = min(mean of the other eigenvalues, rho / 4), rho the current Rayleigh quotient, centres
// the noise eigenvalues, which lie around their mean, so each step shrinks them by
// max |l_i - sig| / (l1 - sig) instead of l2 / l1. A lane stops moving when a step changes x by
// less than 1e-6; the warp stops when every lane has or after 24 steps (conv false). Returns
// l1 = rho and, as l2, the bound sqrt(|S|_F^2 - rho^2) >= sqrt(sum_{i > 1} l_i^2) >= |l2|.
template <int L>
__device__ __forceinline__ void power_eigvec(const float (&S)[L * (L + 1) / 2], const float* Ssh, bool active,
                                             float (&x)[L], float& l1, float& l2, int& steps, bool& conv) {
    float trS = 0.f, fro2 = 0.f, dmax = -1.f;
    int kd = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const float v = S[tri(i, i, L)];
        trS += v;
        if (v > dmax) {
            dmax = v;
            kd = i;
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
        for (int j = i; j < L; ++j) fro2 = fmaf((i == j ? 1.f : 2.f) * S[tri(i, j, L)], S[tri(i, j, L)], fro2);
    {
        float n2 = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            x[i] = active ? Ssh[tri(i, kd, L) * kBatThreads] : (i == kd ? 1.f : 0.f);
            n2 = fmaf(x[i], x[i], n2);
        }
        const float inv = rsqrtf(n2);
#pragma unroll
        for (int i = 0; i < L; ++i) x[i] *= inv;
    }
    steps = 0;
    conv = false;
    float rho = dmax;
#pragma unroll 1
    for (;;) {
        float y[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < L; ++j) a = fmaf(S[tri(i, j, L)], x[j], a);
            y[i] = a;
        }
        float rr = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) rr = fmaf(x[i], y[i], rr);
        rho = rr;
        const float sig = fminf((trS - rr) * (1.f / (float)(L - 1)), 0.25f * rr);
        float n2 = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            y[i] = fmaf(-sig, x[i], y[i]);
            n2 = fmaf(y[i], y[i], n2);
        }
        const float inv = rsqrtf(n2);
        float d2 = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const float v = y[i] * inv;
            const float d = v - x[i];
            d2 = fmaf(d, d, d2);
            x[i] = v;
        }
        ++steps;
        conv = conv || d2 <= 1e-12f;
        if (steps >= 24 || __all_sync(kFull, conv)) break;
    }
    l1 = rho;
    const float u2 = fro2 - rho * rho;
    l2 = u2 > 0.f ? sqrtf(u2) : 0.f;
}

// Three steps of inverse iteration with (mu I - S) = L D L^T, mu = l1 (1 + 1e-5) just above the
// largest eigenvalue estimate l1, from column k1 of S (S = sc times the thread's parked column).
template <int L>
__device__ __forceinline__ void inverse_iteration(const float* Ssh, float sc, float l1, int k1, float (&x)[L]) {
    constexpr int NS = L * (L + 1) / 2;
    const float mu = l1 + 1e-5f * l1 + 1e-30f;
    float Lm[NS];  // unit lower factor in the packed layout, D on the diagonal slots
#pragma unroll
    for (int j = 0; j < L; ++j) {
        float dj = mu - sc * Ssh[tri(j, j, L) * kBatThreads];
#pragma unroll
        for (int k = 0; k < j; ++k) dj = fmaf(-Lm[tri(j, k, L)] * Lm[tri(j, k, L)], Lm[tri(k, k, L)], dj);
        if (fabsf(dj) < 1e-30f) dj = dj < 0.f ? -1e-30f : 1e-30f;
        Lm[tri(j, j, L)] = dj;
        const float inv = frcp(dj);
#pragma unroll
        for (int i = j + 1; i < L; ++i) {
            float v = -sc * Ssh[tri(i, j, L) * kBatThreads];
#pragma unroll
            for (int k = 0; k < j; ++k) v = fmaf(-Lm[tri(i, k, L)] * Lm[tri(j, k, L)], Lm[tri(k, k, L)], v);
            Lm[tri(i, j, L)] = v * inv;
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i) x[i] = sc * Ssh[tri(i, k1, L) * kBatThreads];
#pragma unroll 1
    for (int step = 0; step < 3; ++step) {
#pragma unroll
        for (int i = 0; i < L; ++i)
#pragma unroll
            for (int k = 0; k < i; ++k) x[i] = fmaf(-Lm[tri(i, k, L)], x[k], x[i]);
#pragma unroll
        for (int i = 0; i < L; ++i) x[i] *= frcp(Lm[tri(i, i, L)]);
#pragma unroll
        for (int i = L - 1; i >= 0; --i)
#pragma unroll
            for (int k = i + 1; k < L; ++k) x[i] = fmaf(-Lm[tri(k, i, L)], x[k], x[i]);
        float n2 = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) n2 = fmaf(x[i], x[i], n2);
        const float inv = rsqrtf(n2);
#pragma unroll
        for (int i = 0; i < L; ++i) x[i] *= inv;
    }
}

// Cyclic Jacobi sweeps on S (in registers, destroyed) in tournament ("circle") order: each of the
// L - 1 steps of a sweep rotates the disjoint pairs (0,1), (2,3), ... and then relabels the
// indices by the fixed permutation tperm, so that every pair (p, q) is rotated exactly once per
// sweep and the labels return to the identity after the sweep; the step is one rolled loop body.
// The sweeps only have to place the inverse iteration's shift near l1: the largest diagonal entry
// a_kk differs from l1 by at most about off / gap, so once off <= 1e-3 gap^2 the shift is within
// ~1e-3 gap of l1 and three inverse-iteration steps reduce the other eigenvectors' share by ~1e-9.
// More sweeps run only while some lane of the warp is short of that (up to max_sweeps).
// The fallback of the power iteration: out of line (a call), so that its register demand does not set
// the register budget of the hot path; S is read back from the thread's parked column (times sc),
// the results go through the caller's small local copies.
template <int L>
__device__ __noinline__ void jacobi_eigvec(const float* Ssh, float sc, int max_sweeps, float* x_out, float* l12_out,
                                           int* sweeps_out, bool* jconv_out) {
    constexpr int NS = L * (L + 1) / 2;
    float S[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) S[i] = sc * Ssh[i * kBatThreads];
    float x[L];
    float l1 = 0.f, l2 = 0.f;
    int sweeps = 0;
    bool jconv = false;
    int k1 = 0;
    for (;;) {
#pragma unroll 1
        for (int stp = 0; stp < L - 1; ++stp) {
#pragma unroll
            for (int p = 0; p < L; p += 2) {
                const int q = p + 1;
                const float apq = S[tri(p, q, L)];
                const float dq = S[tri(q, q, L)] - S[tri(p, p, L)];
                const float den = fabsf(dq) + sqrtf(fmaf(dq, dq, 4.f * apq * apq));
                float t = den > 0.f ? __fdividef(2.f * apq, den) : 0.f;
                t = dq < 0.f ? -t : t;
                const float c = rsqrtf(fmaf(t, t, 1.f));
                const float s = t * c;
                S[tri(p, p, L)] = fmaf(-t, apq, S[tri(p, p, L)]);
                S[tri(q, q, L)] = fmaf(t, apq, S[tri(q, q, L)]);
                S[tri(p, q, L)] = 0.f;
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    if (r == p || r == q) continue;
                    const float g = S[tri(r, p, L)], hh = S[tri(r, q, L)];
                    S[tri(r, p, L)] = fmaf(c, g, -s * hh);
                    S[tri(r, q, L)] = fmaf(s, g, c * hh);
                }
            }
            float B[NS];
#pragma unroll
            for (int r = 0; r < L; ++r)
#pragma unroll
                for (int cc = r; cc < L; ++cc) B[tri(r, cc, L)] = S[tri(tperm(r, L), tperm(cc, L), L)];
#pragma unroll
            for (int i = 0; i < NS; ++i) S[i] = B[i];
        }
        ++sweeps;
        float off = 0.f;
#pragma unroll
        for (int p = 0; p < L - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < L; ++q) off = fmaf(S[tri(p, q, L)], S[tri(p, q, L)], off);
        l1 = S[tri(0, 0, L)];
        l2 = -1e30f;
        k1 = 0;
#pragma unroll
        for (int i = 1; i < L; ++i) {
            const float v = S[tri(i, i, L)];
            if (v > l1) {
                l2 = l1;
                l1 = v;
                k1 = i;
            } else if (v > l2) {
                l2 = v;
            }
        }
        const float gap = l1 - l2;
        jconv = off <= 1e-3f * gap * gap;
        if (sweeps >= max_sweeps) break;
        if (__all_sync(kFull, jconv)) break;
    }
    inverse_iteration<L>(Ssh, sc, l1, k1, x);
#pragma unroll
    for (int i = 0; i < L; ++i) x_out[i] = x[i];
    l12_out[0] = l1;
    l12_out[1] = l2;
    *sweeps_out = sweeps;
    *jconv_out = jconv;
}

// The folded snapshot of Eq. 4-5 at local sample index i0 of the lane's staged run, as the two real
// L-vectors X = [Re p, Im q], Y = [Im p, -Re q] (p_i = s[i] + s[L-1-i], q_i = s[i] - s[L-1-i]).
template <int L>
__device__ __forceinline__ void folded_snapshot(const float2* __restrict__ seg_l, int ps, int i0, float (&X)[L],
                                                float (&Y)[L]) {
    constexpr int h = L / 2;
#pragma unroll
    for (int i = 0; i < h; ++i) {
        const float2 a = seg_l[seg_slot(i0 + i, ps)], b = seg_l[seg_slot(i0 + L - 1 - i, ps)];
        X[i] = a.x + b.x;
        Y[i] = a.y + b.y;
        X[h + i] = a.y - b.y;
        Y[h + i] = b.x - a.x;
    }
}

// S += sg (X X^T + Y Y^T) on the packed upper triangle (sg = +1 or -1).
template <int L>
__device__ __forceinline__ void rank2_update(float (&S)[L * (L + 1) / 2], const float (&X)[L], const float (&Y)[L],
                                             float sg) {
#pragma unroll
    for (int r = 0; r < L; ++r) {
        const float xr = sg * X[r], yr = sg * Y[r];
#pragma unroll
        for (int c = r; c < L; ++c) S[tri(r, c, L)] = fmaf(xr, X[c], fmaf(yr, Y[c], S[tri(r, c, L)]));
    }
}

// CTAS is the number of 128-thread CTAs the kernel is compiled to keep resident per SM
// (__launch_bounds__ minimum blocks, i.e. a register cap of 65536 / (128 CTAS)). More CTAs hide
// more latency but spill more; the best cap depends on L and is chosen by measurement (the
// variants of each L are listed in batched_variants.h). WJ selects the warp-per-matrix schedule
// of the eigenvalue sweeps (warp_jacobi_item) instead of one matrix per thread.
template <int L, int CTAS, bool WJ = false>
__global__ void __launch_bounds__(kBatThreads, CTAS)
batched_kernel(const FrameDev* __restrict__ fr, int nframes, int64_t total_items,
               unsigned long long* __restrict__ counter, const float2* __restrict__ gam,
               float* __restrict__ out, uint8_t* __restrict__ status, BatchedArgs args) {
    static_assert(L % 2 == 0 && L >= 2 && L <= kMaxL, "even L only");
    constexpr int h = L / 2;
    constexpr int NS = L * (L + 1) / 2;
    __shared__ float2 sh_seg[kBatWarps][kSegLen];
    // each thread's running (unnormalised) S, one column per thread, and the factor 1 / trace that
    // normalises it (0 for pixels without a result)
    __shared__ float sh_S[NS * kBatThreads];
    __shared__ float sh_sc[kBatThreads];
    // this warp's iteration statistics, added up per item and flushed to args.counters once when
    // the warp leaves the persistent loop (one atomic per statistic per warp, not per item: the
    // per-item atomics on one L2 line cost 4 % of the launch)
    __shared__ unsigned long long sh_stat[kBatWarps][kStatSlots];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kStatSlots) sh_stat[wid][lane] = 0ull;
    __syncwarp();
    float2* seg = sh_seg[wid];
    float* const Ssh = sh_S + threadIdx.x;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)total_items) break;
        const int f = find_frame(fr, nframes, (int64_t)item, [](const FrameDev& F) { return F.item_start; });
        const FrameDev& F = fr[f];
        const int64_t local = (int64_t)item - F.item_start;
        // a frame's items number below 2^31: 32-bit division (a 64-bit one is a long routine)
        const int wline = (int)((uint32_t)local / (uint32_t)F.nchunks);
        const int run = (int)((uint32_t)local % (uint32_t)F.nchunks);
        const int N = F.N, K = N - L + 1, wlen = F.wlen;
        const int ps = F.rowp_shift, P = 1 << ps, run_len = 32 << ps;
        // every index below follows from these (the staging reads 32 P + N - 1 samples into at most
        // kSegLen slots, a lane's windows reach its sample P - 1 + N - 1, the store stays in window
        // line wline);
        // checked builds test them and skip a bad item whole (the test is uniform over the warp)
        if (!rm_check(f >= 0 && f < nframes && local >= 0 && local < (int64_t)F.wlines * F.nchunks && F.L == L &&
                          N >= L && N <= kMaxN && P >= kRowPMin && P <= kRowP,
                      args.counters))
            continue;
        const int a0 = run * run_len - N / 2;
        const float2* seg_l = seg + (P + 1) * lane;  // the lane's own samples: seg_l[seg_slot(i, ps)]
        const float2* gl = gam + F.gam_off + (uint64_t)wline * wlen;

        // ---- stage the run's samples (coalesced) --------------------------------------------
        __syncwarp();  // every lane is done with the previous item's samples
        for (int e = lane; e < run_len + N - 1; e += 32) {
            const int p = a0 + e;
            seg[seg_slot(e, ps)] = (p >= 0 && p < wlen) ? gl[p] : make_float2(0.f, 0.f);
        }
        __syncwarp();

#pragma unroll 1
        for (int t = 0; t < P; ++t) {
            const int pos = run * run_len + lane * P + t;
            const bool inside = pos < wlen;
            const bool valid = inside && (pos - N / 2 >= 0) && (pos - N / 2 + N - 1 <= wlen - 1);

            // ---- S of this pixel: at the lane's first pixel (its anchor) the sum of the window's K
            // rank-2 terms; at each next pixel the previous pixel's S plus the entering and minus the
            // leaving snapshot's term. One rolled loop over one copy of the update code. (Constant
            // factors 1/K and 1/2 are dropped: S is normalised by its trace below, which leaves its
            // eigenvectors unchanged.)
            float S[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) S[i] = t == 0 ? 0.f : Ssh[i * kBatThreads];
            const int nupd = t == 0 ? K : 2;
#pragma unroll 1
            for (int s = 0; s < nupd; ++s) {
                const int i0 = t == 0 ? s : (s == 0 ? t - 1 + K : t - 1);
                float X[L], Y[L];
                folded_snapshot<L>(seg_l, ps, i0, X, Y);
                rank2_update<L>(S, X, Y, (t > 0 && s == 1) ? -1.f : 1.f);
            }
            if (WJ) __syncwarp();  // the warp-per-matrix sweeps of the previous pixel read every lane's S
#pragma unroll
            for (int i = 0; i < NS; ++i) Ssh[i * kBatThreads] = S[i];
            float tr = 0.f;
#pragma unroll
            for (int i = 0; i < L; ++i) tr += S[tri(i, i, L)];
            const bool nonzero = valid && tr > 0.f && isfinite(tr);
            const float itr = frcp(tr);
            sh_sc[threadIdx.x] = nonzero ? itr : 0.f;
#pragma unroll
            for (int i = 0; i < NS; ++i) S[i] *= itr;
            if (!nonzero) {  // border or empty windows: any well-separated stand-in
#pragma unroll
                for (int i = 0; i < NS; ++i) S[i] = 0.f;
#pragma unroll
                for (int i = 0; i < L; ++i) S[tri(i, i, L)] = (float)(L - i);
            }

            // ---- signal eigenvector of S --------------------------------------------------------------
            // The running S is parked in shared memory (one column per thread, times sh_sc): the power
            // iteration starts from one of its columns, the fallback's inverse iteration reads it back.
            int sweeps = 0, psteps = 0, eig_fb = 0;
            bool jconv = false;
            float l1 = 0.f, l2 = 0.f;
            float x[L];
            if constexpr (WJ) {
                int k1 = 0;
                __syncwarp();  // every lane's S and scale are parked before the warp reads them
                warp_jacobi_item<L>(sh_S, sh_sc, wid, lane, args.max_sweeps, &l1, &l2, &k1, &sweeps, &jconv);
                // the warp-level sweep count, as the thread-per-matrix schedule reports it
                sweeps = __reduce_max_sync(kFull, (unsigned)sweeps);
                inverse_iteration<L>(Ssh, sh_sc[threadIdx.x], l1, k1, x);
            } else {
                // Shifted power iteration; lanes whose iteration did not settle, or whose eigen-gap the
                // Frobenius bound cannot certify, take the cyclic Jacobi sweeps and inverse iteration
                // instead (run by the whole warp when any lane needs them).
                power_eigvec<L>(S, Ssh, nonzero, x, l1, l2, psteps, jconv);
                const bool need = nonzero && (args.exhaustive || !jconv || !(l1 - l2 > 4e-6f * l1));
                if (__any_sync(kFull, need)) {
                    eig_fb = 1;
                    float xj[L], jl[2];
                    bool jc;
                    jacobi_eigvec<L>(Ssh, sh_sc[threadIdx.x], args.max_sweeps, xj, jl, &sweeps, &jc);
                    if (need) {
#pragma unroll
                        for (int i = 0; i < L; ++i) x[i] = xj[i];
                        l1 = jl[0];
                        l2 = jl[1];
                        jconv = jc;
                    }
                }
            }
            const bool separated = l1 - l2 > 4e-6f * l1;

            // ---- u1 = Q x1 and the polynomial coefficients ---------------------------------------------
            cx<float> u[L];
            const float r2 = 0.70710678118654752f;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                u[i] = mkc(r2 * x[i], r2 * x[h + i]);
                u[h + i] = mkc(r2 * x[h - 1 - i], -r2 * x[L - 1 - i]);
            }
            cx<float> c[L];
            const float res_lim2 = music_coefs<L>(u, c);

            // ---- the selected root (Algorithm 1) -----------------------------------------------------------
            bool found, cluster, rconv;
            RootStats rs;
            // Newton's starting radius from the noise's share of the window's energy, 1 - l1 (S has unit
            // trace): on row windows the signal root sits at about 1 - 0.18 (1 - l1) (fitted to the FP64
            // estimator's roots at 5-40 dB, median error 2e-4), close enough for one Newton step
            const float r0 = 1.f - 0.18f * (1.f - l1);
            const cx<float> zz = signal_root_polished_cert<L>(c, res_lim2, args.max_iters, args.exhaustive, nonzero,
                                                              r0, found, cluster, rconv, rs);
            const double omd = args.polish64 ? wrap_pi(polish_arg64<L>(c, zz, cluster) - F.omega_ref) : 0.0;
            float om = args.polish64 ? (float)omd : wrap_pi(atan2f(zz.i, zz.r) - (float)F.omega_ref);

            if (lane == 0 && args.counters) {
                unsigned long long* cs = sh_stat[wid];
                cs[0] += (unsigned long long)sweeps;
                cs[1] += (unsigned long long)rs.iters;
                cs[2] += 1ull;
                cs[3] += (unsigned long long)rs.updates;
                cs[4] += (unsigned long long)rs.evals;
                cs[5] += (unsigned long long)psteps;
                cs[6] += (unsigned long long)eig_fb;
                cs[7] += (unsigned long long)rs.newton;
                cs[8] += (unsigned long long)rs.fallback;
                cs[9] += (unsigned long long)rs.polish;
            }

            // ---- store ---------------------------------------------------------------------------------
            if (inside) {
                const uint64_t o = out_index(F, wline, pos);
                uint8_t st = kStOk;
                if (!valid) {
                    st = kStBorder;
                } else if (!nonzero || !separated || !found) {
                    st = kStDegenerate;
                } else if (!rconv || !jconv) {
                    st = kStNotConverged;
                }
                out[o] = (st == kStOk || st == kStNotConverged) ? om : __int_as_float(0x7fc00000);
                if (status) status[o] = st;
            }
        }
    }
    __syncwarp();
    if (args.counters && lane < kStatSlots && sh_stat[wid][lane]) atomicAdd(args.counters + lane, sh_stat[wid][lane]);
}

// Launch and occupancy of variant v of the solver for covariance order L (batched_variants.h).
template <int L, int V>
static cudaError_t launch_solver_v(const FrameDev* d_frames, int nframes, int64_t total_items,
                                   unsigned long long* d_counter, const float2* d_gamma, float* d_out,
                                   uint8_t* d_status, BatchedArgs a, int grid, cudaStream_t stream) {
    batched_kernel<L, solver_variant_ctas(L, V), solver_variant_warp(V)><<<grid, kBatThreads, 0, stream>>>(
        d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a);
    return cudaGetLastError();
}

template <int L, int V>
static int occupancy_solver_v() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, batched_kernel<L, solver_variant_ctas(L, V), solver_variant_warp(V)>, kBatThreads, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <int L>
cudaError_t launch_solver_t(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                            unsigned long long* d_counter, const float2* d_gamma, float* d_out, uint8_t* d_status,
                            BatchedArgs a, int grid, cudaStream_t s) {
    switch (v) {
        case 0: return launch_solver_v<L, 0>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
        case 1: return launch_solver_v<L, 1>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
        case 2: return launch_solver_v<L, 2>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
        case 3:
            if constexpr (L <= 8)
                return launch_solver_v<L, 3>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
            else
                return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

template <int L>
int occupancy_solver_t(int v) {
    switch (v) {
        case 0: return occupancy_solver_v<L, 0>();
        case 1: return occupancy_solver_v<L, 1>();
        case 2: return occupancy_solver_v<L, 2>();
        case 3:
            if constexpr (L <= 8)
                return occupancy_solver_v<L, 3>();
            else
                return 1;
        default: return 1;
    }
}

}  // namespace rmusic
