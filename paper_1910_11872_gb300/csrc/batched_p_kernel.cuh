// batched_p_kernel.cuh -- the FP32 batched path for model order p = 2 or 3 (Sec. 3 with p complex
// exponentials per window: the noise projector removes the p largest eigenvalues' eigenvectors) on
// raw real lines (no band-pass; the line minus its mean), where a real fringe a + b cos(omega n +
// phi) holds the two exponentials exp(+-j omega) and a local offset one more at zero frequency.
// The same persistent warp-scheduled launch as batched_kernel.cuh: runs of 32 P pixels of a window
// line per warp item, P consecutive pixels per lane, staged samples, anchors at fixed positions.
//
// Per pixel (lane):
//   R       the window's K snapshots s_j (Eq. 4-5) are real, so R_f = sum_j s_j s_j^T is real
//           symmetric (packed upper triangle); the lane's first pixel sums the K rank-1 terms, each
//           next pixel adds the entering and subtracts the leaving snapshot's term. With the
//           forward-backward average R = R_f + J R_f J (1/K and 1/2 dropped: R is normalised by its
//           trace, which leaves its eigenvectors unchanged).
//   subspace  the p dominant eigenvectors span the signal subspace (Eq. 8-11 with p signal
//           eigenvalues); only the subspace matters (the projector I - V V^T), so the kernel runs
//           shifted subspace iteration V <- orth((R - sigma I) V) (Gram-Schmidt) from R's first p
//           columns, sigma = min(mean noise eigenvalue, half the smallest Ritz value). A lane stops
//           when span(V) is invariant to 1e-6 of its weakest direction: |R V - V T|_F <=
//           max(1e-6 theta_p, 3e-7 |T|_F), T = V^T R V, theta_p its smallest eigenvalue. The gap
//           lambda_p > lambda_{p+1} is certified by the smallest eigenvalue of T (the p-th Ritz
//           value, <= lambda_p by interlacing) against sqrt(|R|_F^2 - |T|_F^2) >= lambda_{p+1};
//           where that bound is too loose, against lambda_{p+1} from power iteration on R with
//           span(V) projected out. Lanes whose subspace has not settled after 24 steps (lambda_{p+1}
//           near lambda_p) take cyclic Jacobi on R with accumulated eigenvectors (out of line).
//   poly    c_0 = L - p, c_k = -sum_i sum_m V_i[m] V_i[m+k] (Eq. 12-14 with the projector of p
//           orthonormal vectors); real coefficients. Roots and polish on the lags shrunk by 2e-6
//           (as for p = 1); the optional FP64 step on Q itself.
//   roots   p = 2: Newton's method on the signal root from the carrier's angle, polished, certified
//           by a Schur-Cohn count (the real coefficients make the signal roots an exact pair z,
//           conj(z): L - 3 roots inside |z| - 0.02 prove the pair the two nearest the circle), the
//           pair's member whose angle is nearest the carrier's. Otherwise (p = 3, or a lane without
//           the certificate, and with it its warp) every root inside the unit disk by the symmetric
//           Aberth iteration of roots_device.cuh, started at the carrier's angle (with real
//           coefficients, starting points placed symmetrically about the real axis would stay so,
//           and a real one would stay real); of the p inner roots nearest the circle the one whose
//           angle is nearest the carrier's 2 pi f0 (the positive frequency of the fringe); a split
//           double root located on Q' between its halves as for p = 1; two polish steps.
#pragma once

#include "batched_kernel.cuh"

namespace rmusic {

// R += sg s s^T on the packed upper triangle for the real snapshot at local sample index i0 (the
// staged samples are complex64 with zero imaginary parts on raw lines: the real parts are read).
template <int L>
__device__ __forceinline__ void real_rank1(float (&R)[L * (L + 1) / 2], const float2* __restrict__ seg_l, int ps,
                                           int i0, float sg) {
    float s[L];
#pragma unroll
    for (int m = 0; m < L; ++m) s[m] = seg_l[seg_slot(i0 + m, ps)].x;
#pragma unroll
    for (int r = 0; r < L; ++r) {
        const float a = sg * s[r];
#pragma unroll
        for (int c = r; c < L; ++c) R[tri(r, c, L)] = fmaf(a, s[c], R[tri(r, c, L)]);
    }
}

// Entry (m, l) of the symmetric R from its packed upper triangle.
template <int L>
__device__ __forceinline__ float sym_at(const float (&R)[L * (L + 1) / 2], int m, int l) {
    return m <= l ? R[tri(m, l, L)] : R[tri(l, m, L)];
}

// Smallest eigenvalue of the symmetric PM x PM matrix T (PM = 2: closed form; PM = 3: the
// trigonometric form of the cubic's roots).
template <int PM>
__device__ __forceinline__ float sym_min_eig(const float (&T)[PM][PM]) {
    if constexpr (PM == 2) {
        const float a = T[0][0], d = T[1][1], b = 0.5f * (T[0][1] + T[1][0]);
        const float h = 0.5f * (a - d);
        return 0.5f * (a + d) - sqrtf(h * h + b * b);
    } else {
        const float a = T[0][0], d = T[1][1], f = T[2][2];
        const float b = 0.5f * (T[0][1] + T[1][0]), c = 0.5f * (T[0][2] + T[2][0]), e = 0.5f * (T[1][2] + T[2][1]);
        const float q = (a + d + f) * (1.f / 3.f);
        const float p1 = b * b + c * c + e * e;
        const float p2 = (a - q) * (a - q) + (d - q) * (d - q) + (f - q) * (f - q) + 2.f * p1;
        if (!(p2 > 0.f)) return q;  // a multiple of the identity
        const float pp = sqrtf(p2 * (1.f / 6.f)), ip = 1.f / pp;
        const float A = (a - q) * ip, D = (d - q) * ip, Fq = (f - q) * ip, B = b * ip, C = c * ip, E = e * ip;
        const float r = 0.5f * (A * (D * Fq - E * E) - B * (B * Fq - E * C) + C * (B * E - D * C));
        const float phi = acosf(fminf(fmaxf(r, -1.f), 1.f)) * (1.f / 3.f);
        return q + 2.f * pp * cosf(phi + 2.0943951023931953f);  // the smallest of q + 2 pp cos(phi + 2 pi k / 3)
    }
}

// Modified Gram-Schmidt on the PM rows of V; a row that vanishes is replaced by the unit vector e_i
// (its Gram-Schmidt remainder, or e_i itself when that vanishes too).
template <int L, int PM>
__device__ __forceinline__ void orthonormalise(float (&V)[PM][L]) {
#pragma unroll
    for (int i = 0; i < PM; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j) {
            float d = 0.f;
#pragma unroll
            for (int m = 0; m < L; ++m) d = fmaf(V[i][m], V[j][m], d);
#pragma unroll
            for (int m = 0; m < L; ++m) V[i][m] = fmaf(-d, V[j][m], V[i][m]);
        }
        float n2 = 0.f;
#pragma unroll
        for (int m = 0; m < L; ++m) n2 = fmaf(V[i][m], V[i][m], n2);
        if (n2 > 1e-30f) {
            const float inv = rsqrtf(n2);
#pragma unroll
            for (int m = 0; m < L; ++m) V[i][m] *= inv;
        } else {
#pragma unroll
            for (int m = 0; m < L; ++m) V[i][m] = m == i ? 1.f : 0.f;
        }
    }
}

// W_i = R V_i for the PM rows of V (each packed entry read once and applied to every row).
template <int L, int PM>
__device__ __forceinline__ void sym_matvecs(const float (&R)[L * (L + 1) / 2], const float (&V)[PM][L],
                                            float (&W)[PM][L]) {
#pragma unroll
    for (int i = 0; i < PM; ++i)
#pragma unroll
        for (int m = 0; m < L; ++m) W[i][m] = 0.f;
#pragma unroll
    for (int r = 0; r < L; ++r) {
#pragma unroll
        for (int c = r; c < L; ++c) {
            const float a = R[tri(r, c, L)];
#pragma unroll
            for (int i = 0; i < PM; ++i) {
                W[i][r] = fmaf(a, V[i][c], W[i][r]);
                if (c != r) W[i][c] = fmaf(a, V[i][r], W[i][c]);
            }
        }
    }
}

// The PM inner roots of largest modulus (a root within 1e-6 of one already taken is the other half
// of a double root and not counted, as in the selection rule for p exponentials), the one of them
// whose angle is nearest omega_ref, and the root of the full set nearest to it (its mirror, another
// inner root or a mirror), which decides whether the two form a split double root.
template <int L, int PM>
__device__ __forceinline__ void select_p(const cx<float> (&z)[L - 1], const cx<float> (&mz)[L - 1], float omega_ref,
                                         cx<float>& zs, cx<float>& zn, bool& found) {
    constexpr int NI = L - 1;
    int taken[PM];
    cx<float> zt[PM];
#pragma unroll
    for (int t = 0; t < PM; ++t) {
        taken[t] = -1;
        zt[t] = mkc(0.f, 0.f);
        float bestr = -1.f;
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            bool skip = false;
#pragma unroll
            for (int u = 0; u < t; ++u) skip = skip || taken[u] == i || norm2(z[i] - zt[u]) < 1e-12f;
            const float r = norm2(z[i]);
            if (!skip && r > bestr) {
                bestr = r;
                taken[t] = i;
                zt[t] = z[i];
            }
        }
    }
    int best = -1;
    float bestd = 1e30f;
#pragma unroll
    for (int t = 0; t < PM; ++t) {
        if (taken[t] < 0) continue;
        const float d = fabsf(wrap_pi(atan2f(zt[t].i, zt[t].r) - omega_ref));
        if (d < bestd) {
            bestd = d;
            best = taken[t];
        }
    }
    found = best >= 0;
    zs = mkc(1.f, 0.f);
    cx<float> ms = zs;
#pragma unroll
    for (int i = 0; i < NI; ++i)
        if (i == best) {
            zs = z[i];
            ms = mz[i];
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
}

// Steps of the subspace iteration at most (the warp stops when every lane has converged); lanes
// still short of the stop take the Jacobi fallback below. Slow lanes are those whose lambda_{p+1}
// comes near lambda_p (at 10 dB with p = 3 about 5 % of the windows need more than 32 steps).
constexpr int kMaxSubspaceSteps = 24;

// Fallback, out of line: cyclic Jacobi on the real symmetric R (packed Rp, copied by the caller
// inside its branch) with the rotations accumulated; returns the PM eigenvectors of the largest
// eigenvalues as the rows of Vout, the PM + 1 largest eigenvalues in lam (decreasing), the sweeps
// and whether the off-diagonal mass fell below 1e-12 of the total within max_sweeps.
template <int L, int PM>
__device__ __noinline__ void sym_jacobi_top(const float* Rp_in, float* Vout, float* lam, int max_sweeps, int* sweeps_out,
                                            bool* conv_out) {
    float A[L][L], Q[L][L];
#pragma unroll 1
    for (int r = 0; r < L; ++r)
#pragma unroll 1
        for (int c = 0; c < L; ++c) {
            A[r][c] = r <= c ? Rp_in[tri(r, c, L)] : Rp_in[tri(c, r, L)];
            Q[r][c] = r == c ? 1.f : 0.f;
        }
    bool conv = false;
    int sweeps = 0;
#pragma unroll 1
    for (; sweeps < max_sweeps; ++sweeps) {
        float off = 0.f, fro = 0.f;
#pragma unroll 1
        for (int r = 0; r < L; ++r)
#pragma unroll 1
            for (int c = 0; c < L; ++c) {
                fro = fmaf(A[r][c], A[r][c], fro);
                if (r != c) off = fmaf(A[r][c], A[r][c], off);
            }
        if (off <= 1e-12f * fro) {
            conv = true;
            break;
        }
#pragma unroll 1
        for (int pi = 0; pi < L - 1; ++pi)
#pragma unroll 1
            for (int qi = pi + 1; qi < L; ++qi) {
                const float apq = A[pi][qi];
                if (apq == 0.f) continue;
                // rotation that zeroes A[p][q]: t = tan(angle), the smaller root of t^2 + 2 th t - 1 = 0
                const float th = (A[qi][qi] - A[pi][pi]) / (2.f * apq);
                const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                const float cs = rsqrtf(fmaf(t, t, 1.f)), sn = t * cs;
#pragma unroll 1
                for (int k = 0; k < L; ++k) {  // columns p, q of A
                    const float akp = A[k][pi], akq = A[k][qi];
                    A[k][pi] = cs * akp - sn * akq;
                    A[k][qi] = sn * akp + cs * akq;
                }
#pragma unroll 1
                for (int k = 0; k < L; ++k) {  // rows p, q of A
                    const float apk = A[pi][k], aqk = A[qi][k];
                    A[pi][k] = cs * apk - sn * aqk;
                    A[qi][k] = sn * apk + cs * aqk;
                }
#pragma unroll 1
                for (int k = 0; k < L; ++k) {  // the eigenvectors are Q's columns
                    const float qkp = Q[k][pi], qkq = Q[k][qi];
                    Q[k][pi] = cs * qkp - sn * qkq;
                    Q[k][qi] = sn * qkp + cs * qkq;
                }
            }
    }
    // the PM + 1 largest eigenvalues, largest first, and the first PM eigenvectors
    unsigned used = 0u;
#pragma unroll 1
    for (int i = 0; i <= PM; ++i) {
        int bi = 0;
        float bv = -3.4e38f;
#pragma unroll 1
        for (int k = 0; k < L; ++k)
            if (!((used >> k) & 1u) && A[k][k] > bv) {
                bv = A[k][k];
                bi = k;
            }
        used |= 1u << bi;
        lam[i] = bv;
        if (i < PM)
#pragma unroll 1
            for (int m = 0; m < L; ++m) Vout[i * L + m] = Q[m][bi];
    }
    *sweeps_out = sweeps;
    *conv_out = conv;
}


template <int L, int PM, int CTAS>
__global__ void __launch_bounds__(kBatThreads, CTAS)
batched_p_kernel(const FrameDev* __restrict__ fr, int nframes, int64_t total_items,
                 unsigned long long* __restrict__ counter, const float2* __restrict__ gam,
                 float* __restrict__ out, uint8_t* __restrict__ status, BatchedArgs args) {
    static_assert(PM >= 2 && PM <= 3 && L > PM && L <= kMaxL, "model order 2 or 3, L > p");
    constexpr int NS = L * (L + 1) / 2;
    __shared__ float2 sh_seg[kBatWarps][kSegLen];
    // each thread's running (unnormalised) R_f, packed upper triangle, one column per thread
    __shared__ float sh_R[NS * kBatThreads];
    __shared__ unsigned long long sh_stat[kBatWarps][kStatSlots];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kStatSlots) sh_stat[wid][lane] = 0ull;
    __syncwarp();
    float2* seg = sh_seg[wid];
    float* const Rsh = sh_R + threadIdx.x;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= (unsigned long long)total_items) break;
        const int f = find_frame(fr, nframes, (int64_t)item, [](const FrameDev& F) { return F.item_start; });
        const FrameDev& F = fr[f];
        const int64_t local = (int64_t)item - F.item_start;
        const int wline = (int)((uint32_t)local / (uint32_t)F.nchunks);
        const int run = (int)((uint32_t)local % (uint32_t)F.nchunks);
        const int N = F.N, K = N - L + 1, wlen = F.wlen;
        const int ps = F.rowp_shift, P = 1 << ps, run_len = 32 << ps;
        // the indices below follow from these (as in batched_kernel); checked builds test them and skip
        // a bad item whole (the test is uniform over the warp)
        if (!rm_check(f >= 0 && f < nframes && local >= 0 && local < (int64_t)F.wlines * F.nchunks && F.L == L &&
                          N >= L && N <= kMaxN && P >= kRowPMin && P <= kRowP,
                      args.counters))
            continue;
        const int a0 = run * run_len - N / 2;
        const float2* seg_l = seg + (P + 1) * lane;
        const float2* gl = gam + F.gam_off + (uint64_t)wline * wlen;
        const float omega_ref = (float)F.omega_ref;
        // the signal root's starting direction: the carrier's angle, moved off the real axis
        float th0 = omega_ref;
        if (fabsf(sinf(th0)) < 0.1f) th0 = 0.5f;
        float sn0, cs0;
        sincosf(th0, &sn0, &cs0);
        const cx<float> e0 = mkc(cs0, sn0);

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

            // ---- R_f of this pixel (anchor: K rank-1 terms; then + entering - leaving snapshot) -----
            float R[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) R[i] = t == 0 ? 0.f : Rsh[i * kBatThreads];
            const int nupd = t == 0 ? K : 2;
#pragma unroll 1
            for (int s = 0; s < nupd; ++s) {
                const int i0 = t == 0 ? s : (s == 0 ? t - 1 + K : t - 1);
                real_rank1<L>(R, seg_l, ps, i0, (t > 0 && s == 1) ? -1.f : 1.f);
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) Rsh[i * kBatThreads] = R[i];
            // forward-backward average in place: R[r][c] + R[L-1-c][L-1-r] on both entries of a pair
            if (args.fb) {
#pragma unroll
                for (int r = 0; r < L; ++r) {
#pragma unroll
                    for (int c = r; c < L; ++c) {
                        const int a = tri(r, c, L), b = tri(L - 1 - c, L - 1 - r, L);
                        if (a < b) {
                            const float v = R[a] + R[b];
                            R[a] = v;
                            R[b] = v;
                        } else if (a == b) {
                            R[a] = 2.f * R[a];
                        }
                    }
                }
            }
            float tr = 0.f;
#pragma unroll
            for (int i = 0; i < L; ++i) tr += R[tri(i, i, L)];
            const bool nonzero = valid && tr > 0.f && isfinite(tr);
            const float itr = nonzero ? frcp(tr) : 0.f;
#pragma unroll
            for (int i = 0; i < NS; ++i) R[i] *= itr;
            if (!nonzero) {  // border or empty windows: any well-separated stand-in
#pragma unroll
                for (int i = 0; i < NS; ++i) R[i] = 0.f;
#pragma unroll
                for (int i = 0; i < L; ++i) R[tri(i, i, L)] = (float)(L - i);
            }

            // ---- signal subspace: shifted subspace iteration from R's first PM columns ------------
            float V[PM][L], W[PM][L], T[PM][PM];
#pragma unroll
            for (int i = 0; i < PM; ++i)
#pragma unroll
                for (int m = 0; m < L; ++m) V[i][m] = sym_at<L>(R, m, i);
            orthonormalise<L, PM>(V);
            bool sconv = !nonzero;
            float sig = 0.f, t2 = 0.f;
            int steps = 0;
#pragma unroll 1
            for (;;) {
                sym_matvecs<L, PM>(R, V, W);
#pragma unroll
                for (int i = 0; i < PM; ++i)
#pragma unroll
                    for (int j = 0; j < PM; ++j) {
                        float d = 0.f;
#pragma unroll
                        for (int m = 0; m < L; ++m) d = fmaf(V[i][m], W[j][m], d);
                        T[i][j] = d;
                    }
                // residual of the invariant-subspace equation R V = V T
                float e2 = 0.f;
                t2 = 0.f;
#pragma unroll
                for (int j = 0; j < PM; ++j) {
#pragma unroll
                    for (int m = 0; m < L; ++m) {
                        float e = W[j][m];
#pragma unroll
                        for (int i = 0; i < PM; ++i) e = fmaf(-V[i][m], T[i][j], e);
                        e2 = fmaf(e, e, e2);
                    }
#pragma unroll
                    for (int i = 0; i < PM; ++i) t2 = fmaf(T[i][j], T[i][j], t2);
                }
                // the weakest signal direction is resolved to |E| / (lambda_p - lambda_{p+1}): the stop is
                // relative to the smallest Ritz value, down to FP32's resolution of R (~3e-7 |T|_F)
                const float lm = sym_min_eig<PM>(T);
                sconv = sconv || e2 <= fmaxf(1e-12f * lm * lm, 1e-13f * t2);
                if (steps == 0) {
                    float trT = 0.f;
#pragma unroll
                    for (int i = 0; i < PM; ++i) trT += T[i][i];
                    const float noise_mean = fmaxf(1.f - trT, 0.f) * (1.f / (float)(L - PM));
                    sig = fminf(noise_mean, 0.5f * fmaxf(sym_min_eig<PM>(T), 0.f));
                }
                ++steps;
                if (steps >= kMaxSubspaceSteps || __all_sync(kFull, sconv)) break;
#pragma unroll
                for (int i = 0; i < PM; ++i)
#pragma unroll
                    for (int m = 0; m < L; ++m) V[i][m] = fmaf(-sig, V[i][m], W[i][m]);
                orthonormalise<L, PM>(V);
            }
            // the gap: smallest Ritz value (<= lambda_p) against sqrt(|R|_F^2 - |T|_F^2) (>= lambda_{p+1})
            float rf2 = 0.f, trT = 0.f;
#pragma unroll
            for (int r = 0; r < L; ++r)
#pragma unroll
                for (int c = r; c < L; ++c) rf2 = fmaf(r == c ? 1.f : 2.f, R[tri(r, c, L)] * R[tri(r, c, L)], rf2);
#pragma unroll
            for (int i = 0; i < PM; ++i) trT += T[i][i];
            float lmin = sym_min_eig<PM>(T);
            float lam_next = -1.f;  // lambda_{p+1} where the Jacobi fallback gives it
            int sweeps = 0, eig_fb = 0;
            const bool need = nonzero && !sconv;
            if (__any_sync(kFull, need)) {
                eig_fb = 1;
                float Rc[NS], Vj[PM * L], lj[PM + 1];
#pragma unroll
                for (int i = 0; i < NS; ++i) Rc[i] = R[i];
                bool jc;
                sym_jacobi_top<L, PM>(Rc, Vj, lj, 16, &sweeps, &jc);
                if (need) {
#pragma unroll
                    for (int i = 0; i < PM; ++i)
#pragma unroll
                        for (int m = 0; m < L; ++m) V[i][m] = Vj[i * L + m];
                    lmin = lj[PM - 1];
                    lam_next = lj[PM];
                    trT = 0.f;
#pragma unroll
                    for (int i = 0; i < PM; ++i) trT += lj[i];
                    sconv = jc;
                }
            }
            const float bound = sqrtf(fmaxf(rf2 - t2, 0.f));
            bool separated = lam_next >= 0.f ? lmin - lam_next > 4e-6f * trT : lmin - bound > 4e-6f * trT;
            // The Frobenius bound counts every noise eigenvalue; where it does not certify the gap,
            // lambda_{p+1} itself: power iteration on R with span(V) projected out (8 steps from a
            // fixed vector; its Rayleigh quotient is the largest eigenvalue of the deflated R).
            if (__any_sync(kFull, nonzero && !separated)) {
                float xv[L], yv[L];
#pragma unroll
                for (int m = 0; m < L; ++m) xv[m] = sinf(1.7f * (float)m + 0.3f);
                float lam = 0.f;
#pragma unroll 1
                for (int it = 0; it < 9; ++it) {
                    // x <- (I - V V^T) x, normalised
#pragma unroll
                    for (int i = 0; i < PM; ++i) {
                        float d = 0.f;
#pragma unroll
                        for (int m = 0; m < L; ++m) d = fmaf(V[i][m], xv[m], d);
#pragma unroll
                        for (int m = 0; m < L; ++m) xv[m] = fmaf(-d, V[i][m], xv[m]);
                    }
                    float n2 = 0.f;
#pragma unroll
                    for (int m = 0; m < L; ++m) n2 = fmaf(xv[m], xv[m], n2);
                    const float inv = n2 > 1e-30f ? rsqrtf(n2) : 0.f;
#pragma unroll
                    for (int m = 0; m < L; ++m) xv[m] *= inv;
                    // y = R x, lam = x^T R x
#pragma unroll
                    for (int m = 0; m < L; ++m) yv[m] = 0.f;
#pragma unroll
                    for (int r = 0; r < L; ++r)
#pragma unroll
                        for (int c = r; c < L; ++c) {
                            const float a = R[tri(r, c, L)];
                            yv[r] = fmaf(a, xv[c], yv[r]);
                            if (c != r) yv[c] = fmaf(a, xv[r], yv[c]);
                        }
                    lam = 0.f;
#pragma unroll
                    for (int m = 0; m < L; ++m) {
                        lam = fmaf(xv[m], yv[m], lam);
                        xv[m] = yv[m];
                    }
                }
                if (nonzero && !separated && lam_next < 0.f) separated = lmin - lam > 4e-6f * trT;
            }

            // ---- coefficients of Q from the projector I - V V^T (Eq. 12-14) ----------------------
            // c: the lags shrunk by 2e-6, as for p = 1 (Q stays strictly positive on the circle in FP32,
            // which keeps double roots apart radially, and the FP32 polish stable: on Q itself it
            // wanders near its double roots, where Q' vanishes); cu: Q itself, for the optional FP64
            // step, which removes the shrink's own displacement of the root (up to ~1e-4 rad at
            // L = p + 2 with the forward-backward average)
            cx<float> c[L], cu[L];
            c[0] = mkc((float)(L - PM), 0.f);
            cu[0] = c[0];
            float qsum = (float)(L - PM);
#pragma unroll
            for (int k = 1; k < L; ++k) {
                float a = 0.f;
#pragma unroll
                for (int i = 0; i < PM; ++i)
#pragma unroll
                    for (int m = 0; m + k < L; ++m) a = fmaf(V[i][m], V[i][m + k], a);
                c[k] = mkc(-(1.f - 2e-6f) * a, 0.f);
                cu[k] = mkc(-a, 0.f);
                qsum += 2.f * fabsf(c[k].r);
            }
            const float res_lim2 = (3e-6f * qsum) * (3e-6f * qsum);

            // ---- the selected root ---------------------------------------------------------------
            // p = 2, certified: the coefficients are real, so the signal roots are an exact pair z,
            // conj(z). Newton's method (the root's mirror divided out) from radius 0.99 at the
            // carrier's angle, two polish steps, and a Schur-Cohn count of exactly L - 3 roots inside
            // |z| - 0.02 prove that z and conj(z) are the two inner roots nearest the circle; of them
            // the selection takes the one whose angle is nearest omega_ref. Lanes without the
            // certificate (and all lanes for p = 3, exhaustive runs) take every inner root by Aberth.
            cx<float> zz = mkc(1.f, 0.f);
            bool found = true, rconv = true, cluster = false, cert = false;
            int riters = 0, revals = 0, rupdates = 0, newton = 0, rfb = 0;
            if constexpr (PM == 2) {
                if (!args.exhaustive) {
                    cx<float> z = 0.99f * e0;
                    bool nconv = !nonzero;
#pragma unroll 1
                    for (int it = 0; it < kNewtonSteps; ++it) {
                        cx<float> pv, dv;
                        horner_pd<L>(c, z, pv, dv);
                        const cx<float> wv = mirror_newton_step(z, pv, dv);
                        const bool fin = isfinite(wv.r) && isfinite(wv.i);
                        const bool small = norm2(pv) <= res_lim2;
                        if (!nconv && !small && fin) {
                            z = z - wv;
                            const float r2 = norm2(z);
                            if (r2 > 1.f) z = frcp(r2) * z;
                        }
                        nconv = nconv || small || (fin && norm2(wv) <= 1e-5f);
                        ++newton;
                        if (__all_sync(kFull, nconv)) break;
                    }
                    z = polish_isolated<L>(c, z);
                    const float r = sqrtf(norm2(z));
                    // a pair near the real axis may be a split double root: the full root finder
                    if (nonzero && nconv && r > 0.5f && fabsf(z.i) > 4e-3f) cert = roots_inside<L>(c, r - 0.02f) == L - 3;
                    cert = cert || !nonzero;
                    const cx<float> zc = conjg(z);
                    zz = fabsf(wrap_pi(atan2f(z.i, z.r) - omega_ref)) <= fabsf(wrap_pi(atan2f(zc.i, zc.r) - omega_ref)) ? z : zc;
                    rconv = nconv;
                }
            }
            if (__any_sync(kFull, !cert)) {
                rfb = 1;
                cx<float> z[L - 1], mz[L - 1];
                bool aconv, afound;
                inner_roots_from<L>(c, res_lim2, args.max_iters, e0, z, mz, riters, revals, rupdates, aconv);
                cx<float> zs, zn;
                select_p<L, PM>(z, mz, omega_ref, zs, zn, afound);
                const bool cl = norm2(zn - zs) < 4e-3f * 4e-3f;
                const cx<float> za = polish_root<L>(c, zs, zn, cl);
                if (!cert) {
                    zz = za;
                    cluster = cl;
                    found = afound;
                    rconv = aconv;
                }
            }
            const float om = args.polish64 ? (float)wrap_pi(polish_arg64<L>(cu, zz, cluster) - F.omega_ref)
                                           : wrap_pi(atan2f(zz.i, zz.r) - omega_ref);

            if (lane == 0 && args.counters) {
                unsigned long long* cs = sh_stat[wid];
                cs[0] += (unsigned long long)sweeps;
                cs[1] += (unsigned long long)riters;
                cs[2] += 1ull;
                cs[3] += (unsigned long long)rupdates;
                cs[4] += (unsigned long long)revals;
                cs[5] += (unsigned long long)steps;
                cs[6] += (unsigned long long)eig_fb;
                cs[7] += (unsigned long long)newton;
                cs[8] += (unsigned long long)rfb;
                cs[9] += (unsigned long long)kPolishSteps;
            }

            if (inside) {
                const uint64_t o = out_index(F, wline, pos);
                uint8_t st = kStOk;
                if (!valid) {
                    st = kStBorder;
                } else if (!nonzero || !separated || !found) {
                    st = kStDegenerate;
                } else if (!rconv || !sconv) {
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

// Resident 128-thread CTAs per SM of the model-order solver for order L (one register cap each).
__host__ __device__ constexpr int p_ctas(int L) { return L <= 6 ? 4 : L <= 8 ? 3 : 2; }

template <int L, int PM>
cudaError_t launch_p_t(const FrameDev* d_frames, int nframes, int64_t total_items, unsigned long long* d_counter,
                       const float2* d_gamma, float* d_out, uint8_t* d_status, BatchedArgs a, int grid,
                       cudaStream_t s) {
    batched_p_kernel<L, PM, p_ctas(L)><<<grid, kBatThreads, 0, s>>>(d_frames, nframes, total_items, d_counter,
                                                                     d_gamma, d_out, d_status, a);
    return cudaGetLastError();
}

template <int L, int PM>
int occupancy_p_t() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_p_kernel<L, PM, p_ctas(L)>, kBatThreads, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace rmusic
