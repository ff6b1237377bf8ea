// batched_fwd_kernel.cuh -- the FP32 batched path for the paper's own forward estimate, R = R_f
// without the forward-backward average (Sec. 3, Eq. 4-5): the same persistent warp-scheduled launch
// as batched_kernel.cuh (runs of 32 P pixels of a window line per warp item, P consecutive pixels per
// lane, staged samples, anchors at fixed positions), on the complex Hermitian R instead of the real
// symmetric transform that the forward-backward average allows. Any covariance order 2 .. kMaxL.
//
// Per pixel (lane):
//   R         the window's K snapshots s_j (Eq. 4-5): R = sum_j s_j s_j^H (1/K dropped: R is
//             normalised by its trace), the packed upper triangle in real and imaginary parts; the
//             lane's first pixel sums the K rank-1 terms, each next pixel adds the entering and
//             subtracts the leaving snapshot's term (one rolled loop over one copy of the update).
//   eigen     the signal eigenvector u1 (Eq. 8-11) by the shifted power iteration on the complex
//             Hermitian R (a Hermitian matrix keeps the iterate's phase, so the step size measures
//             convergence as in the real case), from R's column of largest diagonal entry; the
//             eigen-gap certified by |l2| <= sqrt(|R|_F^2 - l1^2). Lanes where that fails take cyclic
//             complex Jacobi sweeps with accumulated eigenvectors (out of line).
//   roots     u1 gives the root-MUSIC coefficients directly; the root stage is the FB path's
//             (roots_device.cuh: Newton, polish, Rouche / Schur-Cohn certificate, Aberth fallback),
//             with Newton started at radius 0.99 (the forward estimate's roots lie further inside).
#pragma once

#include "batched_kernel.cuh"

namespace rmusic {

// S += sg s s^H on the packed upper triangle (Rr real parts, Ri imaginary parts; the diagonal's
// imaginary parts are not touched: they stay 0) for the snapshot at local sample index i0.
template <int L>
__device__ __forceinline__ void herm_rank1(float (&Rr)[L * (L + 1) / 2], float (&Ri)[L * (L + 1) / 2],
                                           const float2* __restrict__ seg_l, int ps, int i0, float sg) {
    float2 s[L];
#pragma unroll
    for (int m = 0; m < L; ++m) s[m] = seg_l[seg_slot(i0 + m, ps)];
#pragma unroll
    for (int r = 0; r < L; ++r) {
        const float ar = sg * s[r].x, ai = sg * s[r].y;
        Rr[tri(r, r, L)] = fmaf(ar, s[r].x, fmaf(ai, s[r].y, Rr[tri(r, r, L)]));
#pragma unroll
        for (int c = r + 1; c < L; ++c) {
            // s_r conj(s_c)
            Rr[tri(r, c, L)] = fmaf(ar, s[c].x, fmaf(ai, s[c].y, Rr[tri(r, c, L)]));
            Ri[tri(r, c, L)] = fmaf(ai, s[c].x, fmaf(-ar, s[c].y, Ri[tri(r, c, L)]));
        }
    }
}

// Entry (m, l) of the Hermitian R from its packed upper triangle.
template <int L>
__device__ __forceinline__ cx<float> herm_at(const float (&Rr)[L * (L + 1) / 2], const float (&Ri)[L * (L + 1) / 2],
                                            int m, int l) {
    return m <= l ? mkc(Rr[tri(m, l, L)], Ri[tri(m, l, L)]) : mkc(Rr[tri(l, m, L)], -Ri[tri(l, m, L)]);
}

// Signal eigenvector x of the complex Hermitian R (packed, trace-normalised) by the shifted power
// iteration x <- (R - sig I) x / |.|, sig = min(mean of the other eigenvalues, rho / 4), from column
// kd of R (largest diagonal entry; read from the parked columns Rsh_r / Rsh_i, any positive multiple of
// R; inactive lanes start from the unit vector). Without the forward-backward average the noise
// eigenvalues spread wider and the iteration can contract slowly, so a small step alone does not
// bound the distance to the eigenvector: a lane stops when the distance that the last two steps'
// contraction q predicts, |step| q / (1 - q), is below 1e-6 (q < 0.9), or at a step below 2e-7 (FP32's
// floor); the warp stops when every lane has or after 48 steps. l1 = the Rayleigh quotient,
// l2 = sqrt(|R|_F^2 - l1^2) >= |l2|.
template <int L>
__device__ __forceinline__ void power_eigvec_herm(const float (&Rr)[L * (L + 1) / 2], const float (&Ri)[L * (L + 1) / 2],
                                                  const float* Rsh_r, const float* Rsh_i, bool active,
                                                  cx<float> (&x)[L], float& l1, float& l2, int& steps, bool& conv) {
    float trR = 0.f, fro2 = 0.f, dmax = -1.f;
    int kd = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const float v = Rr[tri(i, i, L)];
        trR += v;
        fro2 = fmaf(v, v, fro2);
        if (v > dmax) {
            dmax = v;
            kd = i;
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
        for (int j = i + 1; j < L; ++j)
            fro2 = fmaf(2.f * Rr[tri(i, j, L)], Rr[tri(i, j, L)], fmaf(2.f * Ri[tri(i, j, L)], Ri[tri(i, j, L)], fro2));
    {
        float n2 = 0.f;
#pragma unroll
        for (int m = 0; m < L; ++m) {
            if (active) {
                const int a = m <= kd ? m : kd, b = m <= kd ? kd : m;
                const float im = Rsh_i[tri(a, b, L) * kBatThreads];
                x[m] = mkc(Rsh_r[tri(a, b, L) * kBatThreads], m <= kd ? im : -im);
            } else {
                x[m] = mkc(m == kd ? 1.f : 0.f, 0.f);
            }
            n2 += norm2(x[m]);
        }
        const float inv = rsqrtf(n2);
#pragma unroll
        for (int m = 0; m < L; ++m) x[m] = inv * x[m];
    }
    steps = 0;
    conv = false;
    float rho = dmax, d2prev = 0.f;
#pragma unroll 1
    for (;;) {
        cx<float> y[L];
#pragma unroll
        for (int m = 0; m < L; ++m) {
            cx<float> a = mkc(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const cx<float> r = herm_at<L>(Rr, Ri, m, l);
                a = mkc(fmaf(r.r, x[l].r, fmaf(-r.i, x[l].i, a.r)), fmaf(r.r, x[l].i, fmaf(r.i, x[l].r, a.i)));
            }
            y[m] = a;
        }
        float rr = 0.f;
#pragma unroll
        for (int m = 0; m < L; ++m) rr = fmaf(x[m].r, y[m].r, fmaf(x[m].i, y[m].i, rr));
        rho = rr;
        const float sig = fminf((trR - rr) * (1.f / (float)(L > 1 ? L - 1 : 1)), 0.25f * rr);
        float n2 = 0.f;
#pragma unroll
        for (int m = 0; m < L; ++m) {
            y[m] = mkc(fmaf(-sig, x[m].r, y[m].r), fmaf(-sig, x[m].i, y[m].i));
            n2 += norm2(y[m]);
        }
        const float inv = rsqrtf(n2);
        float d2 = 0.f;
#pragma unroll
        for (int m = 0; m < L; ++m) {
            const cx<float> v = inv * y[m];
            d2 += norm2(v - x[m]);
            x[m] = v;
        }
        ++steps;
        const float q = d2prev > 0.f ? sqrtf(d2 / d2prev) : 1.f;
        conv = conv || d2 <= 4e-14f || (q < 0.9f && d2 * q * q <= 1e-12f * (1.f - q) * (1.f - q));
        d2prev = d2;
        if (steps >= 48 || __all_sync(kFull, conv)) break;
    }
    l1 = rho;
    const float u2 = fro2 - rho * rho;
    l2 = u2 > 0.f ? sqrtf(u2) : 0.f;
}

// The fallback: cyclic complex Jacobi sweeps on R (sc times the parked columns) with accumulated
// eigenvectors, out of line (local arrays; its register demand does not set the hot path's). Stops
// once the off-diagonal mass is at the FP32 level, 2 |off|^2 <= (2e-6 |R|_F)^2 (the eigenvectors
// accumulated in V then hold to ~2e-6 |R|_F / gap), or after max_sweeps (jconv false). Returns the
// eigenvector of the largest eigenvalue in u_out, l1 and l2 in l12_out.
template <int L>
__device__ __noinline__ void herm_jacobi_eigvec(const float* Rsh_r, const float* Rsh_i, float sc, int max_sweeps,
                                                cx<float>* u_out, float* l12_out, int* sweeps_out, bool* jconv_out) {
    cx<float> A[L * L], V[L * L];
    for (int m = 0; m < L; ++m)
        for (int l = m; l < L; ++l) {
            const cx<float> v = mkc(sc * Rsh_r[tri(m, l, L) * kBatThreads], m == l ? 0.f : sc * Rsh_i[tri(m, l, L) * kBatThreads]);
            A[m * L + l] = v;
            A[l * L + m] = conjg(v);
        }
    for (int i = 0; i < L * L; ++i) V[i] = mkc((i % (L + 1)) == 0 ? 1.f : 0.f, 0.f);
    float fro2 = 0.f;
    for (int i = 0; i < L * L; ++i) fro2 += norm2(A[i]);
    int sweeps = 0;
    bool jconv = false;
    int k1 = 0;
    float l1 = 0.f, l2 = 0.f;
    for (;;) {
        float off = 0.f;
        for (int p = 0; p < L; ++p)
            for (int q = p + 1; q < L; ++q) off += norm2(A[p * L + q]);
        l1 = -1e30f;
        l2 = -1e30f;
        for (int i = 0; i < L; ++i) {
            const float v = A[i * L + i].r;
            if (v > l1) {
                l2 = l1;
                l1 = v;
                k1 = i;
            } else if (v > l2) {
                l2 = v;
            }
        }
        jconv = 2.f * off <= 4e-12f * fro2;
        if (__all_sync(kFull, jconv) || sweeps >= max_sweeps) break;
        ++sweeps;
        for (int p = 0; p < L - 1; ++p)
            for (int q = p + 1; q < L; ++q) {
                const cx<float> b = A[p * L + q];
                const float ab2 = norm2(b);
                if (!(ab2 > 0.f)) continue;
                const float ab = sqrtf(ab2);
                const cx<float> e = (1.f / ab) * b;
                const float d = A[q * L + q].r - A[p * L + p].r;
                const float den = fabsf(d) + sqrtf(d * d + 4.f * ab2);
                float t = 2.f * ab / den;
                if (d < 0.f) t = -t;
                const float c = rsqrtf(1.f + t * t);
                const float s = t * c;
                const cx<float> se = s * e, sec = s * conjg(e);
                for (int r = 0; r < L; ++r) {
                    if (r == p || r == q) continue;
                    const cx<float> arp = A[r * L + p], arq = A[r * L + q];
                    const cx<float> nrp = c * arp - sec * arq;
                    const cx<float> nrq = se * arp + c * arq;
                    A[r * L + p] = nrp;
                    A[r * L + q] = nrq;
                    A[p * L + r] = conjg(nrp);
                    A[q * L + r] = conjg(nrq);
                }
                A[p * L + p] = mkc(A[p * L + p].r - t * ab, 0.f);
                A[q * L + q] = mkc(A[q * L + q].r + t * ab, 0.f);
                A[p * L + q] = mkc(0.f, 0.f);
                A[q * L + p] = mkc(0.f, 0.f);
                for (int r = 0; r < L; ++r) {
                    const cx<float> vrp = V[r * L + p], vrq = V[r * L + q];
                    V[r * L + p] = c * vrp - sec * vrq;
                    V[r * L + q] = se * vrp + c * vrq;
                }
            }
    }
    for (int m = 0; m < L; ++m) u_out[m] = V[m * L + k1];
    l12_out[0] = l1;
    l12_out[1] = l2;
    *sweeps_out = sweeps;
    *jconv_out = jconv;
}

template <int L, int CTAS>
__global__ void __launch_bounds__(kBatThreads, CTAS)
batched_fwd_kernel(const FrameDev* __restrict__ fr, int nframes, int64_t total_items,
                   unsigned long long* __restrict__ counter, const float2* __restrict__ gam,
                   float* __restrict__ out, uint8_t* __restrict__ status, BatchedArgs args) {
    static_assert(L >= 2 && L <= kMaxL, "covariance order 2 .. kMaxL");
    constexpr int NS = L * (L + 1) / 2;
    __shared__ float2 sh_seg[kBatWarps][kSegLen];
    // each thread's running (unnormalised) R, real and imaginary parts of the packed upper triangle,
    // one column per thread, and the factor 1 / trace that normalises it (0 without a result)
    __shared__ float sh_Rr[NS * kBatThreads];
    __shared__ float sh_Ri[NS * kBatThreads];
    __shared__ float sh_sc[kBatThreads];
    __shared__ unsigned long long sh_stat[kBatWarps][kStatSlots];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kStatSlots) sh_stat[wid][lane] = 0ull;
    __syncwarp();
    float2* seg = sh_seg[wid];
    float* const Rsh_r = sh_Rr + threadIdx.x;
    float* const Rsh_i = sh_Ri + threadIdx.x;

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

            // ---- R of this pixel (anchor: K rank-1 terms; then + entering - leaving snapshot) -------
            float Rr[NS], Ri[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                Rr[i] = t == 0 ? 0.f : Rsh_r[i * kBatThreads];
                Ri[i] = t == 0 ? 0.f : Rsh_i[i * kBatThreads];
            }
            const int nupd = t == 0 ? K : 2;
#pragma unroll 1
            for (int s = 0; s < nupd; ++s) {
                const int i0 = t == 0 ? s : (s == 0 ? t - 1 + K : t - 1);
                herm_rank1<L>(Rr, Ri, seg_l, ps, i0, (t > 0 && s == 1) ? -1.f : 1.f);
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                Rsh_r[i * kBatThreads] = Rr[i];
                Rsh_i[i * kBatThreads] = Ri[i];
            }
            float tr = 0.f;
#pragma unroll
            for (int i = 0; i < L; ++i) tr += Rr[tri(i, i, L)];
            const bool nonzero = valid && tr > 0.f && isfinite(tr);
            const float itr = frcp(tr);
            sh_sc[threadIdx.x] = nonzero ? itr : 0.f;
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                Rr[i] *= itr;
                Ri[i] *= itr;
            }
            if (!nonzero) {  // border or empty windows: any well-separated stand-in
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    Rr[i] = 0.f;
                    Ri[i] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < L; ++i) Rr[tri(i, i, L)] = (float)(L - i);
            }

            // ---- signal eigenvector --------------------------------------------------------------------
            int sweeps = 0, psteps = 0, eig_fb = 0;
            bool jconv = false;
            float l1 = 0.f, l2 = 0.f;
            cx<float> u[L];
            power_eigvec_herm<L>(Rr, Ri, Rsh_r, Rsh_i, nonzero, u, l1, l2, psteps, jconv);
            const bool need = nonzero && (args.exhaustive || !jconv || !(l1 - l2 > 4e-6f * l1));
            if (__any_sync(kFull, need)) {
                eig_fb = 1;
                cx<float> uj[L];
                float jl[2];
                bool jc;
                herm_jacobi_eigvec<L>(Rsh_r, Rsh_i, sh_sc[threadIdx.x], args.max_sweeps, uj, jl, &sweeps, &jc);
                if (need) {
#pragma unroll
                    for (int i = 0; i < L; ++i) u[i] = uj[i];
                    l1 = jl[0];
                    l2 = jl[1];
                    jconv = jc;
                }
            }
            const bool separated = l1 - l2 > 4e-6f * l1;

            // ---- coefficients and the selected root (Eq. 12-15, Algorithm 1) ---------------------------
            cx<float> c[L];
            const float res_lim2 = music_coefs<L>(u, c);
            bool found, cluster, rconv;
            RootStats rs;
            // Newton starts at radius 0.99. The forward estimate's signal root lies further inside than
            // the forward-backward one's (1 - |z_s| up to ~0.1 on noisy windows, weakly tied to l1): a
            // start near the circle sits between the root and its mirror, where each deflated step is
            // about |z - 1/conj(z)| long, and the step-size stop ended Newton up to 3e-4 rad short.
            constexpr float r0 = 0.99f;
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

// Resident 128-thread CTAs per SM of variant v (0 or 1) of the forward solver for order L: register
// caps 2 apart where the shared memory (R parked as 2 L (L + 1) / 2 floats per thread) allows.
__host__ __device__ constexpr int fwd_variant_ctas(int L, int v) {
    return L <= 5 ? (v == 0 ? 4 : 6) : L <= 8 ? (v == 0 ? 3 : 4) : (v == 0 ? 1 : 2);
}

template <int L, int V>
static cudaError_t launch_fwd_v(const FrameDev* d_frames, int nframes, int64_t total_items,
                                unsigned long long* d_counter, const float2* d_gamma, float* d_out, uint8_t* d_status,
                                BatchedArgs a, int grid, cudaStream_t stream) {
    batched_fwd_kernel<L, fwd_variant_ctas(L, V)><<<grid, kBatThreads, 0, stream>>>(d_frames, nframes, total_items,
                                                                                     d_counter, d_gamma, d_out,
                                                                                     d_status, a);
    return cudaGetLastError();
}

template <int L, int V>
static int occupancy_fwd_v() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_fwd_kernel<L, fwd_variant_ctas(L, V)>, kBatThreads,
                                                      0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <int L>
cudaError_t launch_fwd_t(int v, const FrameDev* d_frames, int nframes, int64_t total_items,
                         unsigned long long* d_counter, const float2* d_gamma, float* d_out, uint8_t* d_status,
                         BatchedArgs a, int grid, cudaStream_t s) {
    if (v == 0) return launch_fwd_v<L, 0>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
    if (v == 1) return launch_fwd_v<L, 1>(d_frames, nframes, total_items, d_counter, d_gamma, d_out, d_status, a, grid, s);
    return cudaErrorInvalidValue;
}

template <int L>
int occupancy_fwd_t(int v) {
    return v == 0 ? occupancy_fwd_v<L, 0>() : v == 1 ? occupancy_fwd_v<L, 1>() : 1;
}

}  // namespace rmusic
