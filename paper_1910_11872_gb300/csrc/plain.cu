// plain.cu -- the plain GPU path: one thread per pixel, one launch per frame, every step of the
// method done by that thread in precision T (float or double), with the window, matrices and
// polynomial in thread-local arrays. This is the structure of the paper's own GPU kernel
// (Algorithm 1: pixel index -> window -> eigen-decomposition -> polynomial -> roots ->
// selection -> Eq. 15), kept as the baseline the batched path is measured against and, in FP64,
// as the GPU path that reproduces the CPU oracle to ~1e-9 rad/pixel.
//
// Per pixel:
//   window   w[i] = Gamma[n - N/2 + i], i < N (border pixels: NaN)                (Sec. 3, Eq. 2)
//   R        R_f[m][l] = (1/K) sum_{i<K} w[i+m] conj(w[i+l]), K = N - L + 1, optional
//            forward-backward average (R_f + J conj(R_f) J) / 2                      (Eq. 4-5)
//   eigen    cyclic complex Jacobi; u1 = eigenvector of the largest eigenvalue      (Eq. 8-11)
//            (model order p > 1: the eigenvectors of the p largest eigenvalues)
//   poly     Q(z) = sum_k c_k z^(k+L-1), c_k = sum_{l-m=k} (I - u1 u1^H)[m][l]        (Eq. 12-14)
//            (p > 1: I - sum_{i<p} u_i u_i^H)
//   roots    Aberth-Ehrlich on all 2L-2 roots from a circle of starting points
//   select   the root with |z| <= 1 + tau_in nearest the unit circle; if another root lies
//            within tau_c of it the pair is one split double root, located on Q'; otherwise two
//            Newton steps on Q with the conjugate-reciprocal partner 1/conj(z) divided out
//            refine it                                                          (Algorithm 1)
//            (p > 1: among the p roots nearest the circle, a split double root counted once,
//            the one whose angle is nearest the expected angle)
//   angle    arg(z) minus the carrier step, wrapped to (-pi, pi]                     (Eq. 15)
#include <math.h>

#include "rmusic_device.cuh"
#include "rmusic_launch.h"

namespace rmusic {

template <typename T>
struct PlainTol;
template <>
struct PlainTol<double> {
    static constexpr double jacobi = 1e-14;  // off-diagonal norm / ||R||_F at convergence
    static constexpr double gap = 1e-12;     // (l1 - l2) / l1 below this: degenerate
    static constexpr double resid = 1e-14;   // |Q(z)| / sum |q_k| |z|^k at a root
    static constexpr double cand = 1e-9;     // candidates: |z| <= 1 + cand
    static constexpr double cluster = 1e-6;  // two roots closer than this are one double root
    static constexpr double shrink = 0.0;    // relative shrink of the lag coefficients c_k, k != 0
};
template <>
struct PlainTol<float> {
    static constexpr float jacobi = 2e-6f;
    static constexpr float gap = 4e-6f;
    static constexpr float resid = 8e-6f;
    static constexpr float cand = 1e-3f;
    static constexpr float cluster = 4e-3f;
    // keeps Q(e^jw) e^-j(L-1)w >= 2e-6 (L - 1) > 0 above the FP32 rounding of the coefficients,
    // so a noise-free double root splits radially (same angle) instead of along the circle
    static constexpr float shrink = 2e-6f;
};

template <typename T>
__device__ __forceinline__ T tsqrt(T x);
template <>
__device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }

template <typename T>
__device__ __forceinline__ T tatan2(T y, T x);
template <>
__device__ __forceinline__ double tatan2<double>(double y, double x) { return atan2(y, x); }
template <>
__device__ __forceinline__ float tatan2<float>(float y, float x) { return atan2f(y, x); }

template <typename T>
__device__ __forceinline__ void tsincos(T a, T* s, T* c);
template <>
__device__ __forceinline__ void tsincos<double>(double a, double* s, double* c) { sincos(a, s, c); }
template <>
__device__ __forceinline__ void tsincos<float>(float a, float* s, float* c) { sincosf(a, s, c); }

// Q(z), Q'(z), Q''(z) and the bound sum |q_k| |z|^k by Horner's rule, q ascending.
template <typename T>
__device__ void horner3(const cx<T>* q, int deg, cx<T> z, cx<T>* p, cx<T>* d1, cx<T>* d2, T* bound) {
    cx<T> pv = q[deg], a1 = mkc(T(0), T(0)), a2 = mkc(T(0), T(0));
    T b = tsqrt(norm2(q[deg]));
    const T az = tsqrt(norm2(z));
    for (int i = deg - 1; i >= 0; --i) {
        a2 = a2 * z + a1;
        a1 = a1 * z + pv;
        pv = pv * z + q[i];
        b = b * az + tsqrt(norm2(q[i]));
    }
    *p = pv;
    *d1 = a1;
    *d2 = T(2) * a2;
    *bound = b;
}

// Storage type of the analytic signal each precision reads: complex64 / complex128.
template <typename T>
struct GammaOf;
template <>
struct GammaOf<float> {
    using type = float2;
};
template <>
struct GammaOf<double> {
    using type = double2;
};

template <typename T>
__global__ void __launch_bounds__(128)
plain_kernel(const FrameDev* __restrict__ frame, const typename GammaOf<T>::type* __restrict__ gam,
             float* __restrict__ out, uint8_t* __restrict__ status, PlainArgs args) {
    const FrameDev F = *frame;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)F.wlines * F.wlen) return;
    const int wline = (int)(idx / F.wlen);
    const int pos = (int)(idx % F.wlen);
    const uint64_t o = out_index(F, wline, pos);
    const int N = F.N, L = F.L, K = N - L + 1;
    const int start = pos - N / 2;
    if (start < 0 || start + N - 1 > F.wlen - 1) {
        out[o] = __int_as_float(0x7fc00000);
        if (status) status[o] = kStBorder;
        return;
    }
    uint8_t st = kStOk;

    // ---- window (Sec. 3, Eq. 2) -------------------------------------------------------------
    cx<T> w[kMaxN];
    const typename GammaOf<T>::type* g = gam + F.gam_off + (uint64_t)wline * F.wlen + start;
    for (int i = 0; i < N; ++i) {
        const auto v = g[i];
        w[i] = mkc((T)v.x, (T)v.y);
    }

    // ---- auto-correlation matrix (Eq. 4-5) ----------------------------------------------------
    cx<T> A[kMaxL * kMaxL];
    for (int m = 0; m < L; ++m)
        for (int l = m; l < L; ++l) {
            cx<T> acc = mkc(T(0), T(0));
            for (int i = 0; i < K; ++i) acc = acc + mulc(w[i + m], w[i + l]);
            acc = (T(1) / (T)K) * acc;
            A[m * L + l] = acc;
            A[l * L + m] = conjg(acc);
        }
    if (args.fb) {
        // R = (R_f + J conj(R_f) J) / 2; entries (m, l) and (L-1-m, L-1-l) pair up.
        for (int m = 0; m < L; ++m)
            for (int l = 0; l < L; ++l) {
                const int m2 = L - 1 - m, l2 = L - 1 - l;
                if (m * L + l > m2 * L + l2) continue;
                cx<T> a = A[m * L + l], b = A[m2 * L + l2];
                cx<T> na = T(0.5) * (a + conjg(b));
                A[m * L + l] = na;
                A[m2 * L + l2] = conjg(na);
            }
    }

    // ---- cyclic complex Jacobi (Eq. 8-11) ----------------------------------------------------
    cx<T> V[kMaxL * kMaxL];
    T normA = 0;
    for (int i = 0; i < L * L; ++i) normA += norm2(A[i]);
    normA = tsqrt(normA);
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c) V[r * L + c] = mkc(T(r == c), T(0));
    const T tolJ = PlainTol<T>::jacobi * normA;
    bool jac_conv = false;
    if (!(normA > T(0)) || !isfinite((double)normA)) {
        out[o] = __int_as_float(0x7fc00000);
        if (status) status[o] = kStDegenerate;
        return;
    }
    for (int sweep = 0; sweep <= args.max_sweeps; ++sweep) {
        T off = 0;
        for (int p = 0; p < L; ++p)
            for (int q = p + 1; q < L; ++q) off += norm2(A[p * L + q]);
        if (T(2) * off <= tolJ * tolJ) {
            jac_conv = true;
            break;
        }
        if (sweep == args.max_sweeps) break;
        for (int p = 0; p < L - 1; ++p)
            for (int q = p + 1; q < L; ++q) {
                const cx<T> b = A[p * L + q];
                const T ab = tsqrt(norm2(b));
                if (ab == T(0)) continue;
                const cx<T> e = (T(1) / ab) * b;
                const T d = A[q * L + q].r - A[p * L + p].r;
                const T den = fabs(d) + tsqrt(d * d + T(4) * ab * ab);
                T t = T(2) * ab / den;
                if (d < T(0)) t = -t;
                const T c = T(1) / tsqrt(T(1) + t * t);
                const T s = t * c;
                const cx<T> se = s * e, sec = s * conjg(e);
                for (int r = 0; r < L; ++r) {
                    if (r == p || r == q) continue;
                    const cx<T> arp = A[r * L + p], arq = A[r * L + q];
                    const cx<T> nrp = c * arp - sec * arq;
                    const cx<T> nrq = se * arp + c * arq;
                    A[r * L + p] = nrp;
                    A[r * L + q] = nrq;
                    A[p * L + r] = conjg(nrp);
                    A[q * L + r] = conjg(nrq);
                }
                A[p * L + p] = mkc(A[p * L + p].r - t * ab, T(0));
                A[q * L + q] = mkc(A[q * L + q].r + t * ab, T(0));
                A[p * L + q] = mkc(T(0), T(0));
                A[q * L + p] = mkc(T(0), T(0));
                for (int r = 0; r < L; ++r) {
                    const cx<T> vrp = V[r * L + p], vrq = V[r * L + q];
                    V[r * L + p] = c * vrp - sec * vrq;
                    V[r * L + q] = se * vrp + c * vrq;
                }
            }
    }
    if (!jac_conv) st = kStNotConverged;
    // the p + 1 largest eigenvalues, by decreasing value (an earlier index first on ties)
    const int P = args.p;
    int ord[kMaxModelOrder + 1];
    for (int t = 0; t <= P; ++t) ord[t] = -1;
    for (int j = 0; j < L; ++j) {
        const T v = A[j * L + j].r;
        for (int t = 0; t <= P; ++t)
            if (ord[t] < 0 || v > A[ord[t] * L + ord[t]].r) {
                for (int u2 = P; u2 > t; --u2) ord[u2] = ord[u2 - 1];
                ord[t] = j;
                break;
            }
    }
    const T l1 = A[ord[0] * L + ord[0]].r;
    const T lp = A[ord[P - 1] * L + ord[P - 1]].r;
    const T lq = ord[P] >= 0 ? A[ord[P] * L + ord[P]].r : T(-INFINITY);
    if (!(lp - lq > PlainTol<T>::gap * l1)) {
        out[o] = __int_as_float(0x7fc00000);
        if (status) status[o] = kStDegenerate;
        return;
    }

    // ---- root-MUSIC polynomial (Eq. 12-14) of I - sum_{i<p} u_i u_i^H / |u_i|^2 ----------------
    const int deg = 2 * L - 2;
    cx<T> q[2 * kMaxL];
    for (int i = 0; i <= deg; ++i) q[i] = mkc(T(0), T(0));
    T inv_nu[kMaxModelOrder];
    for (int i = 0; i < P; ++i) {
        T nu = 0;
        for (int m = 0; m < L; ++m) nu += norm2(V[m * L + ord[i]]);
        inv_nu[i] = T(1) / nu;
    }
    for (int m = 0; m < L; ++m)
        for (int l = 0; l < L; ++l) {
            cx<T> cml = (-inv_nu[0]) * mulc(V[m * L + ord[0]], V[l * L + ord[0]]);
            for (int i = 1; i < P; ++i) cml = cml - inv_nu[i] * mulc(V[m * L + ord[i]], V[l * L + ord[i]]);
            if (m == l) cml.r += T(1);
            q[l - m + L - 1] = q[l - m + L - 1] + cml;
        }
    if (PlainTol<T>::shrink != T(0))
        for (int i = 0; i <= deg; ++i)
            if (i != L - 1) q[i] = (T(1) - PlainTol<T>::shrink) * q[i];

    // ---- all roots by Aberth-Ehrlich ---------------------------------------------------------
    cx<T> z[2 * kMaxL];
    const T two_pi = T(6.28318530717958647692);
    for (int i = 0; i < deg; ++i) {
        T s, c;
        tsincos(two_pi * (T)i / (T)deg + T(0.7), &s, &c);
        z[i] = mkc(c, s);
    }
    unsigned done = 0;
    const unsigned all = (deg >= 32) ? 0xffffffffu : ((1u << deg) - 1u);
    for (int it = 0; it < args.max_iters && done != all; ++it) {
        for (int i = 0; i < deg; ++i) {
            if (done & (1u << i)) continue;
            cx<T> p, d1, d2;
            T bnd;
            horner3(q, deg, z[i], &p, &d1, &d2, &bnd);
            if (tsqrt(norm2(p)) <= PlainTol<T>::resid * bnd) {
                done |= 1u << i;
                continue;
            }
            if (norm2(d1) == T(0)) {
                z[i] = z[i] * mkc(T(1), T(1e-3));
                continue;
            }
            const cx<T> Ni = cdiv(p, d1);
            cx<T> Si = mkc(T(0), T(0));
            for (int j = 0; j < deg; ++j)
                if (j != i) Si = Si + crecip(z[i] - z[j]);
            const cx<T> corr = cdiv(Ni, mkc(T(1), T(0)) - Ni * Si);
            if (isfinite((double)corr.r) && isfinite((double)corr.i)) z[i] = z[i] - corr;
        }
    }
    if (done != all) st = kStNotConverged;

    // ---- selection (Algorithm 1) and split double roots --------------------------------------
    int best = -1;
    T bestd = INFINITY, bestt = INFINITY;
    if (P == 1) {
        for (int i = 0; i < deg; ++i) {
            const T r = tsqrt(norm2(z[i]));
            if (!(r <= T(1) + PlainTol<T>::cand)) continue;
            const T d = fabs(r - T(1));
            const T t = fabs(wrap_pi(tatan2(z[i].i, z[i].r) - (T)F.omega_ref));
            if (d < bestd || (d == bestd && t < bestt)) {
                best = i;
                bestd = d;
                bestt = t;
            }
        }
    } else {
        // the p candidates nearest the circle (a split double root counted once), then the one
        // whose angle is nearest the expected angle
        int near[kMaxModelOrder];
        for (int t = 0; t < P; ++t) {
            near[t] = -1;
            T nd = INFINITY;
            for (int i = 0; i < deg; ++i) {
                const T r = tsqrt(norm2(z[i]));
                if (!(r <= T(1) + PlainTol<T>::cand)) continue;
                bool taken = false;
                for (int u2 = 0; u2 < t; ++u2)
                    if (near[u2] >= 0 && (i == near[u2] || tsqrt(norm2(z[i] - z[near[u2]])) < PlainTol<T>::cluster))
                        taken = true;
                const T d = fabs(r - T(1));
                if (!taken && d < nd) {
                    nd = d;
                    near[t] = i;
                }
            }
        }
        for (int t = 0; t < P; ++t) {
            if (near[t] < 0) continue;
            const T a = fabs(wrap_pi(tatan2(z[near[t]].i, z[near[t]].r) - (T)F.omega_ref));
            if (a < bestt) {
                bestt = a;
                best = near[t];
            }
        }
    }
    if (best < 0) {
        out[o] = __int_as_float(0x7fc00000);
        if (status) status[o] = kStDegenerate;
        return;
    }
    cx<T> zs = z[best];
    int near = -1;
    T neard = INFINITY;
    for (int j = 0; j < deg; ++j) {
        if (j == best) continue;
        const T d = tsqrt(norm2(z[j] - z[best]));
        if (d < neard) {
            neard = d;
            near = j;
        }
    }
    if (near >= 0 && neard < PlainTol<T>::cluster) {
        cx<T> zm = T(0.5) * (z[best] + z[near]);
        const cx<T> z0 = zm;
        for (int it = 0; it < 16; ++it) {
            cx<T> p, d1, d2;
            T bnd;
            horner3(q, deg, zm, &p, &d1, &d2, &bnd);
            if (norm2(d2) == T(0)) break;
            const cx<T> stp = cdiv(d1, d2);
            zm = zm - stp;
            if (norm2(stp) <= T(1e-32) * norm2(zm)) break;
        }
        zs = (tsqrt(norm2(zm - z0)) <= T(2) * neard) ? zm : z0;
    } else {
        for (int it = 0; it < 2; ++it) {
            cx<T> p, d1, d2;
            T bnd;
            horner3(q, deg, zs, &p, &d1, &d2, &bnd);
            const cx<T> dzp = zs - (T(1) / norm2(zs)) * zs;  // z - 1/conj(z)
            const cx<T> stp = cdiv(p, d1 - cdiv(p, dzp));
            if (isfinite((double)stp.r) && isfinite((double)stp.i)) zs = zs - stp;
        }
    }

    // ---- angle minus carrier (Eq. 15) ----------------------------------------------------------
    const T om = wrap_pi(tatan2(zs.i, zs.r) - (T)F.omega_ref);
    out[o] = (float)om;
    if (status) status[o] = st;
}

template <typename T>
static cudaError_t launch_plain(const FrameDev* d_frame, const FrameDev& h,
                                const typename GammaOf<T>::type* d_gamma,
                                float* d_out, uint8_t* d_status, PlainArgs a, cudaStream_t stream) {
    const int64_t n = (int64_t)h.wlines * h.wlen;
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    const int64_t blocks = (n + threads - 1) / threads;
    plain_kernel<T><<<(unsigned)blocks, threads, 0, stream>>>(d_frame, d_gamma, d_out, d_status, a);
    return cudaGetLastError();
}

cudaError_t launch_plain_fp64(const FrameDev* d_frame, const FrameDev& h, const double2* d_gamma,
                              float* d_out, uint8_t* d_status, PlainArgs a, cudaStream_t stream) {
    return launch_plain<double>(d_frame, h, d_gamma, d_out, d_status, a, stream);
}

cudaError_t launch_plain_fp32(const FrameDev* d_frame, const FrameDev& h, const float2* d_gamma,
                              float* d_out, uint8_t* d_status, PlainArgs a, cudaStream_t stream) {
    return launch_plain<float>(d_frame, h, d_gamma, d_out, d_status, a, stream);
}

}  // namespace rmusic
