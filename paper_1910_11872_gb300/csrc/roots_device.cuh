// roots_device.cuh -- the FP32 polynomial stage shared by the batched solvers (row windows and
// the paper's square block): root-MUSIC coefficients from a signal vector, Aberth-Ehrlich on the
// roots inside the unit disk, selection of the root nearest the circle and its polish (Sec. 3,
// Eq. 12-15; Algorithm 1).
//
//   poly      u1 the signal vector (any norm); c_0 = L - 1, c_k = -(1 - 2e-6) sum_m u1[m]
//             conj(u1[m+k]) / |u1|^2, c_-k = conj(c_k); Q(z) = sum_k c_k z^(k+L-1) (Eq. 12-14).
//             The 2e-6 shrink keeps the polynomial strictly positive on the circle in FP32.
//   roots     the root Algorithm 1 selects, found without computing every root where a
//             certificate allows: Newton's method (with the root's mirror divided out) from the
//             estimator's start -- radius 0.99 at the angle of conj(rho_1) -- converges to the
//             signal root in 3-7 steps; a Schur-Cohn count of the roots of Q inside |z| < r - 0.02
//             (r the found root's modulus) equal to L - 2 proves it is the only inner root that
//             close to the circle, hence the selected one. Warps with a lane lacking the
//             certificate run the full root finder: Aberth-Ehrlich on the L - 1 roots inside the
//             unit disk; the other L - 1 roots are their mirrors 1/conj(z) (the coefficients are
//             conjugate-symmetric). Its starting points come from the estimator's structure: the
//             signal root just inside the circle at the angle of conj(rho_1), the others at radius
//             r = L / (L + 7.3) at the side-lobe angles arg + 2 pi (k + 1/2) / L, k = 1 .. L-2,
//             where a noise-free window puts them. A root stops (freezes) when its residual is at
//             the FP32 rounding level (|Q(z)| <= 3e-6 sum |q_i|), or, if it lies at least 0.05
//             inside the outermost tracked root, when its Newton step is below 1e-3: only the root
//             nearest the circle needs full accuracy (it is polished after the selection), the
//             others only have to be resolved well enough not to change the selection, and
//             Aberth's fixed point for the remaining roots does not depend on where a frozen root
//             stopped. Iterations stop when every root of every lane of the warp is frozen.
//   select    the inner root nearest the unit circle (Algorithm 1). A noise-free window gives a
//             double root on the circle, which FP32 splits by ~sqrt(eps); when another root lies
//             within 4e-3 the pair is located as the root of Q' between them, otherwise the root
//             is refined by Newton on Q with its partner 1/conj(z) divided out. Optionally one
//             more such step runs in FP64.
// Every function here is called by all 32 lanes of a warp together (warp votes decide when the
// iterations stop), one polynomial per lane.
#pragma once

#include <math.h>

#include "rmusic_device.cuh"
#include "rouche_table.h"

namespace rmusic {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

__device__ __forceinline__ cx<float> cdivf(cx<float> a, cx<float> b) {
    const float inv = frcp(b.r * b.r + b.i * b.i);
    return mkc((a.r * b.r + a.i * b.i) * inv, (a.i * b.r - a.r * b.i) * inv);
}

// Coefficient i of Q(z) from c_0 (real) and c_1..c_{L-1}.
template <int L>
__device__ __forceinline__ cx<float> qcoef(const cx<float>* c, int i) {
    const int k = i - (L - 1);
    if (k == 0) return c[0];
    return k > 0 ? c[k] : conjg(c[-k]);
}

template <int L>
__device__ __forceinline__ void horner_pd(const cx<float>* c, cx<float> z, cx<float>& p, cx<float>& d) {
    p = qcoef<L>(c, 2 * L - 2);
    d = mkc(0.f, 0.f);
#pragma unroll
    for (int i = 2 * L - 3; i >= 0; --i) {
        d = d * z + p;
        p = p * z + qcoef<L>(c, i);
    }
}

template <int L>
__device__ __forceinline__ void horner_pdd(const cx<float>* c, cx<float> z, cx<float>& p, cx<float>& d1,
                                           cx<float>& d2) {
    p = qcoef<L>(c, 2 * L - 2);
    d1 = mkc(0.f, 0.f);
    d2 = mkc(0.f, 0.f);
#pragma unroll
    for (int i = 2 * L - 3; i >= 0; --i) {
        d2 = d2 * z + d1;
        d1 = d1 * z + p;
        p = p * z + qcoef<L>(c, i);
    }
    d2 = 2.f * d2;
}

template <int L>
__device__ __forceinline__ void horner_pdd64(const cx<float>* c, cx<double> z, cx<double>& p, cx<double>& d1,
                                             cx<double>& d2) {
    auto q64 = [&](int i) {
        cx<float> v = qcoef<L>(c, i);
        return mkc((double)v.r, (double)v.i);
    };
    p = q64(2 * L - 2);
    d1 = mkc(0.0, 0.0);
    d2 = mkc(0.0, 0.0);
#pragma unroll
    for (int i = 2 * L - 3; i >= 0; --i) {
        d2 = d2 * z + d1;
        d1 = d1 * z + p;
        p = p * z + q64(i);
    }
    d2 = 2.0 * d2;
}

// Coefficients c_0 .. c_{L-1} of Q from the signal vector u (Eq. 12-14). Returns
// res_lim2 = (3e-6 sum_i |q_i|)^2, the squared FP32 rounding level of Q inside the unit disk.
template <int L>
__device__ __forceinline__ float music_coefs(const cx<float>* u, cx<float>* c) {
    float nu2 = 0.f;
#pragma unroll
    for (int i = 0; i < L; ++i) nu2 += norm2(u[i]);
    // Shrinking the lag coefficients by (1 - eta) makes Q(e^jw) e^-j(L-1)w =
    // (1 - eta) P(w) + eta (L - 1) >= eta (L - 1) > 0 on the circle, above the FP32 rounding
    // of the coefficients (~1e-6 of P). Without it, rounding can push a noise-free double root
    // apart along the circle (two roots at w0 +- d, d ~ 1e-3); with it the pair always splits
    // radially and keeps the angle of the minimum of P.
    const float inu2 = (1.f - 2e-6f) * frcp(nu2);
    c[0] = mkc((float)(L - 1), 0.f);
    // sum_i |q_i| bounds sum_i |q_i| |z|^i for every tracked root (all stay in the unit disk):
    // the scale of Q's rounding error in the residual test
    float qsum = (float)(L - 1);
#pragma unroll
    for (int k = 1; k < L; ++k) {
        cx<float> rho = mkc(0.f, 0.f);
#pragma unroll
        for (int m = 0; m + k < L; ++m) rho = rho + mulc(u[m], u[m + k]);
        c[k] = (-inu2) * rho;
        const float n2 = norm2(c[k]);
        qsum += n2 > 0.f ? 2.f * n2 * rsqrtf(n2) : 0.f;  // 2 |c_k| (a bound: approximate is fine)
    }
    return (3e-6f * qsum) * (3e-6f * qsum);
}

// Aberth-Ehrlich on the L - 1 roots of Q inside the unit disk. On return z[] holds them and
// mz[] their mirrors 1/conj(z); iters counts sweeps, evals the evaluations of Q and Q' that ran
// (a root frozen in every lane of the warp is skipped), updates the root updates that ran; rconv
// is false if max_iters sweeps ended before every root of this lane converged.
// inner_roots with the signal root's starting direction e (unit modulus) given by the caller.
template <int L>
__device__ __forceinline__ void inner_roots_from(const cx<float>* c, float res_lim2, int max_iters, cx<float> e,
                                                 cx<float> (&z)[L - 1], cx<float> (&mz)[L - 1], int& iters,
                                                 int& evals, int& updates, bool& rconv) {
    constexpr int NI = L - 1;
    // Q's coefficients satisfy c_-k = conj(c_k), so its roots come in pairs z, 1/conj(z). Only
    // the L - 1 roots inside the unit disk are iterated; each Aberth sum runs over the other
    // inner roots and over all mirrors 1/conj(z_j) (the root's own partner included), and a
    // root that steps outside is folded back to its mirror. The loop over roots is rolled:
    // the current root is always position 0 and the arrays rotate by one after each update,
    // which keeps the code small enough for the instruction cache.
    {
        z[0] = 0.99f * e;
        float sh, ch;
        sincospif(1.0f / (float)L, &sh, &ch);                           // exp(j pi / L)
        const cx<float> step = mkc(ch * ch - sh * sh, 2.f * sh * ch);  // exp(2 j pi / L)
        cx<float> ek = e * mkc(ch, sh) * step;                           // angle + 2 pi (1 + 1/2) / L
        const float rin = (float)L / ((float)L + 7.3f);
#pragma unroll
        for (int k = 1; k < NI; ++k) {
            z[k] = rin * ek;
            ek = ek * step;
        }
#pragma unroll
        for (int k = 0; k < NI; ++k) mz[k] = frcp(norm2(z[k])) * z[k];
    }
    iters = 0;
    evals = 0;
    updates = 0;
    rconv = false;
    unsigned frozen = 0;  // bit r: the root now at position r has converged in this lane
    for (;;) {
        rconv = true;
        // roots this far inside the outermost one may stop at a 1e-3 Newton step
        float rb2 = 0.f;
#pragma unroll
        for (int j = 0; j < NI; ++j) rb2 = fmaxf(rb2, norm2(z[j]));
        const float rfar = sqrtf(rb2) - 0.05f;
        const float far2 = rfar > 0.f ? rfar * rfar : 0.f;
#pragma unroll 1
        for (int r = 0; r < NI; ++r) {
            const cx<float> z0 = z[0];
            cx<float> nz = z0, nm = mz[0];
            // A root whose residual reached the rounding level is frozen: near a double root
            // the corrections below that level are noise and would push it off its angle.
            // Roots frozen in every lane of the warp are skipped altogether.
            if (!__all_sync(kFull, frozen & 1u)) {
                ++evals;
                cx<float> p, dp;
                horner_pd<L>(c, z0, p, dp);
                const cx<float> Ni = cdivf(p, dp);
                const bool cv = (frozen & 1u) || norm2(p) <= res_lim2 ||
                                (norm2(z0) < far2 && norm2(Ni) <= 1e-6f);
                frozen |= cv ? 1u : 0u;
                rconv = rconv && cv;
                if (!__all_sync(kFull, cv)) {
                    ++updates;
                    cx<float> Si = mkc(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < NI; ++j) {
                        if (j > 0) {
                            const cx<float> dz = z0 - z[j];
                            const float inv = frcp(norm2(dz));
                            Si = mkc(fmaf(dz.r, inv, Si.r), fmaf(-dz.i, inv, Si.i));
                        }
                        const cx<float> dm = z0 - mz[j];
                        const float invm = frcp(norm2(dm));
                        Si = mkc(fmaf(dm.r, invm, Si.r), fmaf(-dm.i, invm, Si.i));
                    }
                    const cx<float> w = cdivf(Ni, mkc(1.f, 0.f) - Ni * Si);
                    if (!cv && isfinite(w.r) && isfinite(w.i)) nz = z0 - w;
                    const float r2n = norm2(nz);
                    const float ir2 = frcp(r2n);
                    nm = ir2 * nz;
                    if (r2n > 1.f) {  // fold back inside: swap the root and its mirror
                        const cx<float> t = nz;
                        nz = nm;
                        nm = t;
                    }
                }
            }
            frozen = (frozen >> 1) | ((frozen & 1u) << (NI - 1));
#pragma unroll
            for (int j = 0; j + 1 < NI; ++j) {
                z[j] = z[j + 1];
                mz[j] = mz[j + 1];
            }
            z[NI - 1] = nz;
            mz[NI - 1] = nm;
        }
        ++iters;
        if (iters >= max_iters) break;
        if (__all_sync(kFull, rconv)) break;
    }
}

template <int L>
__device__ __forceinline__ void inner_roots(const cx<float>* c, float res_lim2, int max_iters,
                                            cx<float> (&z)[L - 1], cx<float> (&mz)[L - 1], int& iters,
                                            int& evals, int& updates, bool& rconv) {
    const cx<float> rho1 = (-1.f) * c[1];  // proportional to rho_1
    const float n1 = norm2(rho1);
    const cx<float> e = n1 > 0.f ? rsqrtf(n1) * conjg(rho1) : mkc(1.f, 0.f);
    inner_roots_from<L>(c, res_lim2, max_iters, e, z, mz, iters, evals, updates, rconv);
}

// The candidate of Algorithm 1 among the roots of inner_roots: the inner root nearest the unit
// circle (every tracked root is inside the disk, so the one of largest modulus), and the root of the
// full set nearest to it (its own mirror, another inner root or a mirror), which decides whether
// the two form a split double root. found is false if no root was tracked (never for L >= 2).
template <int L>
__device__ __forceinline__ void nearest_pair(const cx<float> (&z)[L - 1], const cx<float> (&mz)[L - 1],
                                             cx<float>& zs, cx<float>& zn, bool& found) {
    constexpr int NI = L - 1;
    int best = -1;
    float bestr = -1.f;
    zs = mkc(1.f, 0.f);
    cx<float> ms = zs;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const float r = norm2(z[i]);
        if (r > bestr) {
            bestr = r;
            best = i;
            zs = z[i];
            ms = mz[i];
        }
    }
    float neard = norm2(ms - zs);
    zn = ms;
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        const float dj = norm2(z[j] - zs), dmj = norm2(mz[j] - zs);
        if (j != best && dj < neard) {
            neard = dj;
            zn = z[j];
        }
        if (j != best && dmj < neard) {
            neard = dmj;
            zn = mz[j];
        }
    }
    found = best >= 0;
}

// The Newton step on Q with the root's mirror 1/conj(z) divided out -- the one-term Aberth
// correction N / (1 - N / D), N = Q / Q', D = z - 1/conj(z) -- written with one complex division:
// N / (1 - N / D) = Q D / (Q' D - Q). At a critical point of Q (Q' = 0) it is the limit -D.
__device__ __forceinline__ cx<float> mirror_newton_step(cx<float> z, cx<float> p, cx<float> dp) {
    const cx<float> D = z - frcp(norm2(z)) * z;  // z - 1/conj(z)
    const cx<float> pD = p * D;
    return cdivf(pD, dp * D - p);
}

// Polish steps of the selected root.
constexpr int kPolishSteps = 2;

// kPolishSteps FP32 refinement steps of the selected root zs: on Q' from the midpoint of zs and its
// nearest root zn when the two form a split double root (cluster), otherwise Newton on Q with the
// partner 1/conj(z) divided out.
template <int L>
__device__ __forceinline__ cx<float> polish_root(const cx<float>* c, cx<float> zs, cx<float> zn, bool cluster) {
    cx<float> zz = cluster ? 0.5f * (zs + zn) : zs;
#pragma unroll 1
    for (int it = 0; it < kPolishSteps; ++it) {
        cx<float> p, d1, d2;
        horner_pdd<L>(c, zz, p, d1, d2);
        const cx<float> stp = cluster ? cdivf(d1, d2) : mirror_newton_step(zz, p, d1);
        if (isfinite(stp.r) && isfinite(stp.i)) zz = zz - stp;
    }
    return zz;
}

// polish_root for an isolated root only: the same kPolishSteps steps without Q'' (Horner on Q and
// Q' alone gives the same Q and Q' bit for bit, so the result equals polish_root's). Each step is
// taken whenever it is finite, also at the FP32 rounding level of the residual: a lane that
// Newton's method left there can still be ~3e-5 rad from the root, and the steps land it on the
// iteration's FP32 fixed point. (Iterating until the step falls below 1e-6 instead ran into the
// noise floor of the step in most warps and random-walked the root by ~1e-5.)
template <int L>
__device__ __forceinline__ cx<float> polish_isolated(const cx<float>* c, cx<float> zz) {
#pragma unroll 1
    for (int it = 0; it < kPolishSteps; ++it) {
        cx<float> p, d1;
        horner_pd<L>(c, zz, p, d1);
        const cx<float> stp = mirror_newton_step(zz, p, d1);
        if (isfinite(stp.r) && isfinite(stp.i)) zz = zz - stp;
    }
    return zz;
}

// polish_root out of line, for warps where some lane holds a split double root (rare on noisy
// frames): the second derivative it needs then stays out of the certified path's code and
// registers. Takes the caller's copy of the coefficients, made inside the branch.
template <int L>
__device__ __noinline__ void polish_cold(const cx<float>* c_in, cx<float> zs, cx<float> zn, bool cluster,
                                         cx<float>* out) {
    cx<float> c[L];
#pragma unroll
    for (int i = 0; i < L; ++i) c[i] = c_in[i];
    *out = polish_root<L>(c, zs, zn, cluster);
}

// Signal root of Q by Newton's method with the root's mirror divided out -- the one-term
// Aberth correction z <- z - N / (1 - N / (z - 1/conj(z))), N = Q / Q' (mirror_newton_step) -- from
// r0 exp(j arg conj(rho_1)): the signal root's direction from the estimator's lag-1 coefficient and
// the caller's estimate r0 < 1 of its radius (the root sits the closer to the circle the smaller
// the noise's share of the window's energy). A step that
// leaves the disk is folded back onto the mirror. A lane stops when |Q| is at the FP32 rounding
// level (the step is then not taken, as in inner_roots) or after a step below 3.2e-3 (the root is
// then known to ~1e-5, far inside the certificate's 0.02 margin, and the two polish steps that
// follow converge quadratically from there; a 1e-3 stop took a third step in most warps, a 1e-2
// stop left the two polish steps short by up to 1.3e-5 rad in a few pixels per million); the warp
// stops when every lane has or after max_iters steps (conv false for the lanes still moving).
// Inactive lanes (pixels without a result) count as stopped from the start.
template <int L>
__device__ __forceinline__ cx<float> newton_signal_root(const cx<float>* c, float res_lim2, int max_iters,
                                                        bool active, float r0, bool& conv, int& steps) {
    const cx<float> rho1 = (-1.f) * c[1];
    const float n1 = norm2(rho1);
    cx<float> z = n1 > 0.f ? (r0 * rsqrtf(n1)) * conjg(rho1) : mkc(r0, 0.f);
    conv = !active;
    steps = 0;
#pragma unroll 1
    for (;;) {
        cx<float> p, dp;
        horner_pd<L>(c, z, p, dp);
        ++steps;
        const cx<float> w = mirror_newton_step(z, p, dp);
        const bool small = norm2(p) <= res_lim2;
        const bool fin = isfinite(w.r) && isfinite(w.i);
        if (!conv && !small && fin) {
            z = z - w;
            const float r2 = norm2(z);
            if (r2 > 1.f) z = frcp(r2) * z;
        }
        conv = conv || small || (fin && norm2(w) <= 1e-5f);
        if (steps >= max_iters || __all_sync(kFull, conv)) break;
    }
    return z;
}

// Number of roots of Q inside the disk |z| < r, by the Schur-Cohn recursion on P(z) = Q(r z):
// with P*(z) = z^n conj(P(1/conj z)) and g = P(0) / conj(lead P), the polynomial
// P1(z) = (P(z) - g P*(z)) / z has degree n - 1, and Rouche's theorem on the unit circle (where
// |P*| = |P|) gives N(P) = N(P1) + 1 if |P(0)| < |lead P|, else N(P) = n - 1 - N(P1). Returns -1
// when some |P(0)|^2 is within 2e-4 of |lead P|^2 (relative), where FP32 rounding could decide
// the comparison, or when |lead P|^2 is zero, infinite or NaN (the coefficients are not rescaled
// between levels, which keeps this straight-line code short; on the root-MUSIC polynomials with
// r > 0.48 their magnitudes stay within 2^+-40). One test covers all of these: with la = |lead P|^2
// infinite or NaN, |la - l0| > 2e-4 la is false; with l0 = |P(0)|^2 infinite and la finite the
// comparison l0 < la is still decided correctly, and a NaN l0 fails the test.
template <int L>
__device__ __forceinline__ int roots_inside(const cx<float>* c, float r) {
    constexpr int n = 2 * L - 2;
    cx<float> a[n + 1];
    {
        float s = 1.f;
#pragma unroll
        for (int i = 0; i <= n; ++i) {
            a[i] = s * qcoef<L>(c, i);
            s *= r;
        }
    }
    unsigned long long inside = 0ull;
    bool ok = true;
#pragma unroll
    for (int deg = n; deg >= 1; --deg) {
        const float la = norm2(a[deg]), l0 = norm2(a[0]);
        ok = ok && la > 0.f && fabsf(la - l0) > 2e-4f * la;
        if (l0 < la) inside |= 1ull << deg;
        const cx<float> g = frcp(la) * (a[0] * a[deg]);  // a0 / conj(a_deg)
        cx<float> b[n];
#pragma unroll
        for (int k = 1; k <= deg; ++k) b[k - 1] = a[k] - g * conjg(a[deg - k]);
#pragma unroll
        for (int k = 0; k < deg; ++k) a[k] = b[k];
    }
    int N = 0;
#pragma unroll
    for (int d = 1; d <= n; ++d) N = ((inside >> d) & 1ull) ? N + 1 : d - 1 - N;
    return ok ? N : -1;
}

// The noise-free deflated polynomial G_L and the lower bounds of min |G_L| on |w| = rho of the Rouche
// certificate below (rouche_table.h), for the row solver's covariance orders.
template <int L>
__device__ __forceinline__ constexpr float rouche_g(int k) {
    static_assert(L >= 3 && L <= 12, "tabulated for L = 3 .. 12");
    if constexpr (L == 3) return rouche_g3(k);
    else if constexpr (L == 4) return rouche_g4(k);
    else if constexpr (L == 5) return rouche_g5(k);
    else if constexpr (L == 6) return rouche_g6(k);
    else if constexpr (L == 7) return rouche_g7(k);
    else if constexpr (L == 8) return rouche_g8(k);
    else if constexpr (L == 9) return rouche_g9(k);
    else if constexpr (L == 10) return rouche_g10(k);
    else if constexpr (L == 11) return rouche_g11(k);
    else return rouche_g12(k);
}
template <int L>
__device__ __forceinline__ const float* rouche_min() {
    if constexpr (L == 3) return kRcMin3;
    else if constexpr (L == 4) return kRcMin4;
    else if constexpr (L == 5) return kRcMin5;
    else if constexpr (L == 6) return kRcMin6;
    else if constexpr (L == 7) return kRcMin7;
    else if constexpr (L == 8) return kRcMin8;
    else if constexpr (L == 9) return kRcMin9;
    else if constexpr (L == 10) return kRcMin10;
    else if constexpr (L == 11) return kRcMin11;
    else return kRcMin12;
}

// roots_inside out of line, for the lanes where the Rouche test does not decide: its straight-line
// code (about 0.7 K instructions at L = 8) then stays out of the hot path's instruction stream. Takes
// the caller's copy of the coefficients, made inside the branch.
template <int L>
__device__ __noinline__ int roots_inside_cold(const cx<float>* c_in, float r) {
    cx<float> c[L];
#pragma unroll
    for (int i = 0; i < L; ++i) c[i] = c_in[i];
    return roots_inside<L>(c, r);
}

// A cheaper exact certificate that Q has exactly L - 2 roots in |z| < rho = r - 0.02 (r = |zs|, zs
// the Newton root; the claim roots_inside checks), by Rouche's theorem against the noise-free
// polynomial. With e = zs / r and w = z / e, the coefficients c_k e^k (c_0, c_{-k} = conj) give the
// polynomial Qh(w) = e^{-(L-1)} Q(e w), whose roots are Q's rotated onto zs's ray: r, 1/r among them.
// Dividing Qh by (w - r)(w - 1/r) = w^2 - (r + 1/r) w + 1 from the top gives the quotient Qh2 of
// degree 2L - 4 and a remainder R1 w + R0. A window of one complex exponential has u1 = a steering
// vector and Qh = the real polynomial of rouche_table.h with its double root at w = 1, whose
// deflation is G_L. On |w| = rho:
// Write the remainder as R(w) = R1 (w - r) + R(r); since quad = (w - r)(w - 1/r), on |w| = rho
//   |Qh - quad G_L| <= |quad| (sum_k |Qh2_k - G_L,k| rho^k + |R1| / (1/r - rho) + |R(r)| / qmin),
//   |quad G_L| >= |quad| min |G_L|,   with |quad| >= qmin = (r - rho)(1/r - rho), |w - 1/r| >= 1/r - rho.
// So if sum_k |Qh2_k - G_L,k| rho^k + |R1| / (1/r - rho) + |R(r)| / qmin < min_{|w| = rho} |G_L|, Qh
// has as many roots in |w| < rho as (w - r)(w - 1/r) G_L: G_L's L - 2 inner roots (rho is above all of
// them where the table's bound is positive; r and 1/r lie outside rho). The test uses
// |x| <= |Re x| + |Im x|, adds 4e-6 sum_i |q_i| / qmin for the FP32 rounding of the rotated
// coefficients and of the division, and compares with 0.9 times the tabulated bound (itself rounded
// down). R(r) = Q(zs) up to a unit factor is the root's residual, so zs must be the polished root:
// from Newton's unpolished root (~1e-4 off on near-circle pairs) the test fails in a few per cent of
// lanes. On noisy row windows (5-40 dB, L = 8, polished roots) it holds in every lane measured, at
// under half the bound; where it fails, the Schur-Cohn count decides. For L = 2 there is nothing to
// exclude. res_lim2 is music_coefs' (3e-6 sum_i |q_i|)^2.
template <int L>
__device__ __forceinline__ bool rouche_certify(const cx<float>* c, cx<float> zs, float r, float res_lim2) {
    if constexpr (L == 2) {
        return true;
    } else {
        constexpr int n = 2 * L - 2;  // degree of Q
        const float rho = r - 0.02f;
        const float ft = (rho - kRcRho0) * (1.f / kRcStep);
        if (!(ft >= 0.f && ft < (float)kRcN)) return false;
        const float mlow = __ldg(rouche_min<L>() + (int)ft);
        if (!(mlow > 0.f)) return false;
        const float ir = frcp(r);
        const cx<float> e = ir * zs;
        cx<float> ch[L];  // c_k e^k
        ch[0] = c[0];
        {
            cx<float> ep = e;
#pragma unroll
            for (int k = 1; k < L; ++k) {
                ch[k] = c[k] * ep;
                if (k + 1 < L) ep = ep * e;
            }
        }
        auto qh = [&](int i) {  // coefficient of w^i in Qh
            const int k = i - (L - 1);
            return k == 0 ? ch[0] : (k > 0 ? ch[k] : conjg(ch[-k]));
        };
        const float sig = r + ir;
        // top-down division: b_{n-2} = qh_n, b_{n-3} = qh_{n-1} + sig b_{n-2},
        // b_k = qh_{k+2} + sig b_{k+1} - b_{k+2}; the sum over k by Horner in rho
        cx<float> b2 = mkc(0.f, 0.f), b1 = mkc(0.f, 0.f);
        float sum = 0.f;
#pragma unroll
        for (int k = n - 2; k >= 0; --k) {
            const cx<float> q = qh(k + 2);
            const cx<float> b = mkc(fmaf(sig, b1.r, q.r) - b2.r, fmaf(sig, b1.i, q.i) - b2.i);
            sum = fmaf(sum, rho, fabsf(b.r - rouche_g<L>(k)) + fabsf(b.i));
            b2 = b1;
            b1 = b;
        }
        // b1 = b_0, b2 = b_1: remainder R1 = qh_1 + sig b_0 - b_1, R0 = qh_0 - b_0, R(r) = R1 r + R0
        const cx<float> q1 = qh(1), q0 = qh(0);
        const cx<float> R1 = mkc(fmaf(sig, b1.r, q1.r) - b2.r, fmaf(sig, b1.i, q1.i) - b2.i);
        const cx<float> Rr = mkc(fmaf(R1.r, r, q0.r - b1.r), fmaf(R1.i, r, q0.i - b1.i));
        const float qmin = (r - rho) * (ir - rho);
        const float qsum = sqrtf(res_lim2) * (1.f / 3e-6f);
        const float lhs = sum + (fabsf(R1.r) + fabsf(R1.i)) * frcp(ir - rho) +
                          (fabsf(Rr.r) + fabsf(Rr.i) + 4e-6f * qsum) * frcp(qmin);
        return lhs < 0.9f * mlow;
    }
}

// Newton steps of the signal root before a lane counts as not converged (it then takes the full
// root finder): 3-4 on row windows, 4-7 on square blocks at 0-10 dB.
constexpr int kNewtonSteps = 16;

// The full root finder of the fallback, out of line: inner_roots and nearest_pair on a copy of the
// coefficients. It runs only in warps where some lane lacks the certificate; compiled as a call, its
// register demand (every inner root and mirror live at once) does not set the register budget of
// the certified path, which then fits a tighter cap without spilling. The arguments are the
// caller's copies made inside the fallback branch, so the hot path's arrays stay in registers.
template <int L>
__device__ __noinline__ void aberth_select(const cx<float>* c_in, float res_lim2, int max_iters, cx<float>* zs,
                                           cx<float>* zn, bool* found, bool* conv, int* stats) {
    constexpr int NI = L - 1;
    cx<float> c[L];
#pragma unroll
    for (int i = 0; i < L; ++i) c[i] = c_in[i];
    cx<float> z[NI], mz[NI];
    int iters, evals, updates;
    bool aconv, afound;
    cx<float> a, b;
    inner_roots<L>(c, res_lim2, max_iters, z, mz, iters, evals, updates, aconv);
    nearest_pair<L>(z, mz, a, b, afound);
    *zs = a;
    *zn = b;
    *found = afound;
    *conv = aconv;
    stats[0] = iters;
    stats[1] = evals;
    stats[2] = updates;
}

struct RootStats {
    int newton;   // Newton steps of the signal root
    int polish;   // polish steps of the selected root
    int fallback; // 1 if the warp ran the full Aberth iteration
    int iters;    // Aberth sweeps, evaluations and root updates (fallback only)
    int evals;
    int updates;
};

// The root stage (Algorithm 1): the inner root of Q nearest the unit circle, refined. The signal
// root comes from newton_signal_root, started at radius r0 (clamped to [0.5, 0.9995]: on the
// circle the mirror deflation has no step); it is the selected root when it is the only root in
// the annulus r - 0.02 <= |z| < 1 (r its modulus), i.e. when Q has exactly L - 2 roots inside
// |z| < r - 0.02 (roots_inside). Lanes without that certificate -- and with them the whole warp,
// which executes the loop together -- take every inner root from inner_roots and select among
// them (nearest_pair). Both end in polish_root; a selected root whose nearest other root is
// closer than 4e-3 is a split double root (cluster). (The polish also lands a certified root on
// the FP32 fixed point of the iteration: Newton's own last step, stopped at the rounding level of
// the residual, leaves up to ~3e-5 rad on noisy windows.) exhaustive (uniform over the launch)
// skips the Newton root and its certificate: every lane takes the full root finder. Inactive lanes
// (border or degenerate pixels, whose result is not used) neither hold the warp in Newton's loop
// nor send it to the full root finder.
template <int L>
__device__ __forceinline__ cx<float> signal_root(const cx<float>* c, float res_lim2, int max_iters, int exhaustive,
                                                 bool active, float r0, bool& found, bool& cluster, bool& rconv,
                                                 RootStats& rs) {
    bool nconv = false, cert = false;
    cx<float> zs = mkc(0.f, 0.f), zn = zs;
    rs.newton = 0;
    if (!exhaustive) {
        // on the circle the mirror deflation has no step: start strictly inside
        zs = newton_signal_root<L>(c, res_lim2, kNewtonSteps, active, fminf(fmaxf(r0, 0.5f), 0.9995f), nconv,
                                   rs.newton);
        const float r2 = norm2(zs);
        const float r = sqrtf(r2);
        int nin = -1;
        if (active && nconv && r > 0.5f) nin = roots_inside<L>(c, r - 0.02f);
        cert = !active || nin == L - 2;
        zn = frcp(r2) * zs;
    }
    found = true;
    rconv = nconv;
    rs.fallback = 0;
    rs.iters = rs.evals = rs.updates = 0;
    if (__any_sync(kFull, !cert)) {
        rs.fallback = 1;
        cx<float> cl[L];
#pragma unroll
        for (int i = 0; i < L; ++i) cl[i] = c[i];
        bool aconv, afound;
        cx<float> azs, azn;
        int st[3];
        aberth_select<L>(cl, res_lim2, max_iters, &azs, &azn, &afound, &aconv, st);
        rs.iters = st[0];
        rs.evals = st[1];
        rs.updates = st[2];
        if (!cert) {
            zs = azs;
            zn = azn;
            found = afound;
            rconv = aconv;
        }
    }
    cluster = norm2(zn - zs) < 4e-3f * 4e-3f;
    if (__any_sync(kFull, cluster)) {
        cx<float> cl[L];
#pragma unroll
        for (int i = 0; i < L; ++i) cl[i] = c[i];
        cx<float> zp;
        polish_cold<L>(cl, zs, zn, cluster, &zp);
        rs.polish = kPolishSteps;
        return zp;
    }
    rs.polish = kPolishSteps;
    return polish_isolated<L>(c, zs);
}

// polish_root of the selected root zs (zn its nearest other root, cluster: the two form a split double
// root), with the second derivative only in warps where some lane holds a cluster.
template <int L>
__device__ __forceinline__ cx<float> polish_selected(const cx<float>* c, cx<float> zs, cx<float> zn, bool cluster) {
    if (__any_sync(kFull, cluster)) {
        cx<float> cl[L];
#pragma unroll
        for (int i = 0; i < L; ++i) cl[i] = c[i];
        cx<float> zp;
        polish_cold<L>(cl, zs, zn, cluster, &zp);
        return zp;
    }
    return polish_isolated<L>(c, zs);
}

// The root stage of the row solver: signal_root's steps in another order. Newton's root is polished
// first and the certificate then checks the polished root -- by rouche_certify, and by the
// Schur-Cohn count (roots_inside at |zp| - 0.02) in lanes where that test does not decide. Lanes
// without a certificate take the full root finder, whose selected root is polished in turn. The
// selected roots are signal_root's: the same Newton root and polish where certified, the same Aberth
// selection and polish otherwise. Newton's steps and the polish of an isolated root run in one rolled
// loop over one copy of the Horner code (newton_signal_root's steps, then polish_isolated's), which
// keeps the hot code small; warps with a split double root polish out of line (polish_cold).
template <int L>
__device__ __forceinline__ cx<float> signal_root_polished_cert(const cx<float>* c, float res_lim2, int max_iters,
                                                               int exhaustive, bool active, float r0, bool& found,
                                                               bool& cluster, bool& rconv, RootStats& rs) {
    bool nconv = false, cert = false;
    cx<float> zs = mkc(0.f, 0.f), zn = zs, zp = zs;
    rs.newton = 0;
    rs.polish = 0;
    cluster = false;
    if (!exhaustive) {
        // Newton's method on the signal root (newton_signal_root), then kPolishSteps polish steps
        const float rs0 = fminf(fmaxf(r0, 0.5f), 0.9995f);  // start strictly inside the circle
        const cx<float> rho1 = (-1.f) * c[1];
        const float n1 = norm2(rho1);
        cx<float> z = n1 > 0.f ? (rs0 * rsqrtf(n1)) * conjg(rho1) : mkc(rs0, 0.f);
        nconv = !active;
        bool polishing = false, cold = false;
        int pol = 0;
#pragma unroll 1
        for (;;) {
            cx<float> p, dp;
            horner_pd<L>(c, z, p, dp);
            const cx<float> w = mirror_newton_step(z, p, dp);
            const bool fin = isfinite(w.r) && isfinite(w.i);
            if (!polishing) {
                ++rs.newton;
                const bool small = norm2(p) <= res_lim2;
                if (!nconv && !small && fin) {
                    z = z - w;
                    const float r2 = norm2(z);
                    if (r2 > 1.f) z = frcp(r2) * z;
                }
                nconv = nconv || small || (fin && norm2(w) <= 1e-5f);
                if (rs.newton >= kNewtonSteps || __all_sync(kFull, nconv)) {
                    zs = z;
                    zn = frcp(norm2(zs)) * zs;
                    cluster = norm2(zn - zs) < 4e-3f * 4e-3f;
                    cold = __any_sync(kFull, cluster);
                    if (cold) break;
                    polishing = true;
                }
            } else {
                if (fin) z = z - w;
                if (++pol == kPolishSteps) break;
            }
        }
        if (cold) {
            cx<float> cl[L];
#pragma unroll
            for (int i = 0; i < L; ++i) cl[i] = c[i];
            polish_cold<L>(cl, zs, zn, cluster, &zp);
        } else {
            zp = z;
        }
        rs.polish = kPolishSteps;
        const float rp = sqrtf(norm2(zp));
        bool counted = false;
        // The Rouche test pays where it decides nearly every lane: at L <= 10 (on the workloads'
        // windows all but a few lanes per thousand). At L = 12 it fails in many lanes of windows with
        // few snapshots (N = 24: K = 13), and a warp then runs both tests: measured 5.19 ms with it
        // and 3.87 ms without on the uneven batch's L = 12 frames.
        if constexpr (L <= 10) {
            if (active && nconv && rp > 0.5f) counted = rouche_certify<L>(c, zp, rp, res_lim2);
        }
        if (active && nconv && rp > 0.5f && !counted) {
            cx<float> cl[L];
#pragma unroll
            for (int i = 0; i < L; ++i) cl[i] = c[i];
            counted = roots_inside_cold<L>(cl, rp - 0.02f) == L - 2;
        }
        cert = !active || counted;
    }
    found = true;
    rconv = nconv;
    rs.fallback = 0;
    rs.iters = rs.evals = rs.updates = 0;
    if (__any_sync(kFull, !cert)) {
        rs.fallback = 1;
        cx<float> cl[L];
#pragma unroll
        for (int i = 0; i < L; ++i) cl[i] = c[i];
        bool aconv, afound;
        cx<float> azs, azn;
        int st[3];
        aberth_select<L>(cl, res_lim2, max_iters, &azs, &azn, &afound, &aconv, st);
        rs.iters = st[0];
        rs.evals = st[1];
        rs.updates = st[2];
        if (!cert) {
            zs = azs;
            zn = azn;
            found = afound;
            rconv = aconv;
        }
        const bool cl2 = norm2(zn - zs) < 4e-3f * 4e-3f;
        const cx<float> zq = polish_selected<L>(c, zs, zn, cl2);
        rs.polish += kPolishSteps;
        if (!cert) {
            zp = zq;
            cluster = cl2;
        }
    }
    return zp;
}

// One more refinement step of the selected root in FP64; returns arg z in double.
template <int L>
__device__ __forceinline__ double polish_arg64(const cx<float>* c, cx<float> zz, bool cluster) {
    cx<double> z64 = mkc((double)zz.r, (double)zz.i);
    cx<double> p, d1, d2;
    horner_pdd64<L>(c, z64, p, d1, d2);
    cx<double> stp;
    if (cluster) {
        stp = cdiv(d1, d2);
    } else {
        const double in2 = 1.0 / norm2(z64);
        const cx<double> dzp = z64 - in2 * z64;
        stp = cdiv(p, d1 - cdiv(p, dzp));
    }
    if (isfinite(stp.r) && isfinite(stp.i)) z64 = z64 - stp;
    return atan2(z64.i, z64.r);
}

}  // namespace rmusic
