/*
 * rmusic_oracle.c -- plain, slow, FP64 CPU oracle for the per-pixel sliding-window
 * root-MUSIC local phase-derivative path of
 *   J. Ramaiah, S. Ajithaprasad, G. Rajshekhar, D. Ambrosini,
 *   "Fast and robust method for flow analysis using GPU assisted diffractive optical
 *    element based background oriented schlieren (BOS)", arXiv:1910.11872.
 *
 * THIS FILE IS TEST INFRASTRUCTURE. It is the independent reference that the CUDA path
 * is checked against. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may build, load or call it. The product path never routes through it,
 * and it shares no code, header, table or helper with the CUDA sources.
 *
 * Every step is written out in the order the paper's method takes it, in double
 * precision, without blocking, fusion or reordering:
 *   step 1  frame sample -> real intensity                       (image stack, Sec. 2)
 *   step 2  analytic signal by DFT band-pass along the carrier    (Sec. 2, Eq. 1)
 *   step 3  moving window along the derivative axis               (Sec. 3, Eq. 2-3)
 *   step 4  sample auto-correlation matrix, optional FB average   (Sec. 3, Eq. 4-5)
 *   step 5  eigen-decomposition, signal / noise subspaces         (Sec. 3, Eq. 6-11)
 *   step 6  root-MUSIC polynomial coefficients                     (Sec. 3, Eq. 12-14)
 *   step 7  all polynomial roots                                   (Sec. 3, companion / roots)
 *   step 8  root closest to the unit circle, magnitude below one  (Sec. 3, root selection;
 *                                                                  Algorithm 1)
 *   step 9  angle of the root, minus the carrier                   (Sec. 3, Eq. 15)
 * and, for the paper's own square block (2 Lp + 1 samples a side), steps 4-9 on the
 * block's columns and conjugated rows plus the local phase alpha (Sec. 3, Eq. 4-15,
 * Algorithm 1).
 *
 * Readings taken where the paper is silent or ambiguous (each is exercised by a pin test):
 *   - band-pass: one-sided FT band |k/W - f0| < B, 1 <= k < W/2, B = f0/2 by default;
 *   - window: N samples starting at n - floor(N/2) along the derivative axis; a pixel whose
 *     window leaves the line is a border pixel (output NaN);
 *   - snapshots: the K = N - L + 1 length-L sub-vectors of the window (covariance order L);
 *     forward-backward averaging is an option (off reproduces the plain forward estimate);
 *   - model order 1: the noise projector is I - u1 u1^H with |u1| = 1;
 *   - polynomial: the standard root-MUSIC continuation u(z)^H -> [1, z^-1, ..., z^-(L-1)],
 *     giving the Laurent polynomial sum_k c_k z^k, c_k = sum_{l-m=k} C[m,l]; it is made a
 *     polynomial of degree 2L-2 by multiplying with z^(L-1);
 *   - selection: roots with |z| <= 1 + 1e-9 are candidates; the one minimising ||z|-1| is
 *     taken; if another root lies within 1e-6 of it, the two are one double root split by
 *     rounding, and the root of Q' between them is returned;
 *   - the eigen-decomposition is a cyclic complex Jacobi iteration; the paper's SVD of the
 *     window data yields the same subspaces;
 *   - square block: alpha of Eq. 15 is taken with coordinates centred on the pixel, so it
 *     is the local phase there; the carrier is removed after the angles, from both the
 *     derivative along the carrier axis and alpha;
 *   - a complex frame (complex64 / complex128) is the analytic signal itself, as for the
 *     complex fringe the paper simulates, and is not band-passed;
 *   - optional 2-D band: the carrier band times a low-pass |k / len| < B_c across the carrier
 *     lines (a rectangle in the 2-D spectrum), applied as a second 1-D pass;
 *   - model order p > 1 (real fringes without the analytic step, Gamma = the line minus its
 *     mean): the noise projector keeps the p largest eigenvalues' eigenvectors out, and the
 *     derivative comes from the one of the p roots nearest the circle whose angle is nearest
 *     the expected angle.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared -fopenmp rmusic_oracle.c -lm
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_MAXL 32

/* Per-pixel status codes. */
#define ORC_OK 0
#define ORC_BORDER 1
#define ORC_DEGENERATE 2
#define ORC_NOT_CONVERGED 3

/* Input sample types. */
#define ORC_F32 0
#define ORC_U16 1
#define ORC_F64 2
#define ORC_C64 3  /* complex64 (re, im float32): already the analytic signal Gamma */
#define ORC_C128 4 /* complex128 (re, im double): already the analytic signal Gamma */

typedef struct {
    int32_t window_len;       /* N: samples in the moving window                     */
    int32_t cov_order;        /* L: length of a snapshot, order of the covariance     */
    int32_t model_order;      /* p: number of exponentials per window (1 supported)   */
    int32_t forward_backward; /* 1: average R with J conj(R) J                        */
    int32_t deriv_axis;       /* 0: windows along x (rows), 1: along y (columns)      */
    int32_t carrier_axis;     /* axis of the fringe carrier and of the band-pass      */
    double carrier_freq;      /* f0, cycles per pixel                                 */
    double band_halfwidth;    /* B, cycles per pixel; <= 0 selects f0 / 2             */
    double band_cross;        /* B_c: low-pass across the carrier lines, |k / len| < B_c
                                 (a rectangular 2-D band); 0 = none                    */
    int32_t raw_input;        /* 1: no band-pass; Gamma = the real line minus its mean  */
} orc_params;

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------------------------
 * Step 1 -- frame sample to a real intensity (Sec. 2: the image stack of carrier
 * fringes). A 12-bit code is divided by 4095; any positive scale and offset leave the
 * output unchanged because the band-pass drops DC and R only scales.
 * ------------------------------------------------------------------------------- */
static double orc_sample(const void* frame, int dtype, size_t idx) {
    switch (dtype) {
        case ORC_F32: return (double)((const float*)frame)[idx];
        case ORC_U16: return (double)((const uint16_t*)frame)[idx] / 4095.0;
        default: return ((const double*)frame)[idx];
    }
}

/* ---------------------------------------------------------------------------------
 * Step 2 -- analytic signal of one line (Sec. 2, Eq. 1: "bandpass filtering and carrier
 * removal" turns the real fringe into Gamma = A exp(j phi) + eta).
 * X = DFT(v) with the unnormalised forward kernel exp(-2 pi j k n / W); bins with
 * 1 <= k < W/2 and |k/W - f0| < B are kept, all others (DC and the negative band
 * included) are zeroed; Gamma = IDFT(X) with the 1/W factor. The carrier itself is
 * removed after the angle (step 9): a rotation of Gamma by exp(-j 2 pi f0 n) rotates
 * every root by the same angle.
 * gamma is interleaved (re, im), length 2W.
 * ------------------------------------------------------------------------------- */
int orc_analytic_line(const double* v, int32_t W, double f0, double B, double* gamma) {
    if (W <= 0) return -1;
    if (B <= 0.0) B = 0.5 * f0;
    cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)W);
    cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)W);
    if (!tw || !X) { free(tw); free(X); return -2; }
    /* tw[m] = exp(-2 pi j m / W); products k*n are reduced mod W so every twiddle is
       evaluated from an angle in [0, 2 pi). */
    for (int32_t m = 0; m < W; ++m) {
        double a = 2.0 * ORC_PI * (double)m / (double)W;
        tw[m] = cos(a) - I * sin(a);
    }
    for (int32_t k = 0; k < W; ++k) {
        cplx acc = 0.0;
        for (int32_t n = 0; n < W; ++n) acc += v[n] * tw[((int64_t)k * n) % W];
        X[k] = acc;
    }
    for (int32_t k = 0; k < W; ++k) {
        int keep = (k >= 1) && (2 * (int64_t)k < W) && (fabs((double)k / (double)W - f0) < B);
        if (!keep) X[k] = 0.0;
    }
    for (int32_t n = 0; n < W; ++n) {
        cplx acc = 0.0;
        for (int32_t k = 0; k < W; ++k) acc += X[k] * conj(tw[((int64_t)k * n) % W]);
        acc /= (double)W;
        gamma[2 * n] = creal(acc);
        gamma[2 * n + 1] = cimag(acc);
    }
    free(tw);
    free(X);
    return 0;
}

/* Analytic signal of a whole frame: one line per row (carrier_axis 0) or per column
   (carrier_axis 1). gamma is H*W interleaved complex, row-major like the frame. */
int orc_analytic_frame(const void* frame, int32_t dtype, int32_t H, int32_t W,
                       int32_t carrier_axis, double f0, double B, double* gamma) {
    if (dtype == ORC_C64 || dtype == ORC_C128) {
        /* a complex frame is the analytic signal already (the complex fringe the paper
           simulates in Sec. 4): it is taken as Gamma without a band-pass */
        for (size_t i = 0; i < 2 * (size_t)H * (size_t)W; ++i)
            gamma[i] = dtype == ORC_C64 ? (double)((const float*)frame)[i] : ((const double*)frame)[i];
        return 0;
    }
    int32_t nlines = carrier_axis == 0 ? H : W;
    int32_t len = carrier_axis == 0 ? W : H;
    int err = 0;
#pragma omp parallel for schedule(dynamic)
    for (int32_t li = 0; li < nlines; ++li) {
        double* v = (double*)malloc(sizeof(double) * (size_t)len);
        double* g = (double*)malloc(sizeof(double) * 2 * (size_t)len);
        if (!v || !g) { err = -2; free(v); free(g); continue; }
        for (int32_t n = 0; n < len; ++n) {
            size_t idx = carrier_axis == 0 ? (size_t)li * W + n : (size_t)n * W + li;
            v[n] = orc_sample(frame, dtype, idx);
        }
        orc_analytic_line(v, len, f0, B, g);
        for (int32_t n = 0; n < len; ++n) {
            size_t idx = carrier_axis == 0 ? (size_t)li * W + n : (size_t)n * W + li;
            gamma[2 * idx] = g[2 * n];
            gamma[2 * idx + 1] = g[2 * n + 1];
        }
        free(v);
        free(g);
    }
    return err;
}

/* ---------------------------------------------------------------------------------
 * Step 2, 2-D variant: the band kept by the Fourier method can also be limited across
 * the carrier (the 2-D transform methods the paper cites for its band-pass, Sec. 2).
 * Reading: a rectangular 2-D band, the one-sided carrier band of orc_analytic_line times
 * |k / len| < B_c across it (k the signed bin, -len/2 <= k < len/2). The band is separable,
 * so it is applied here as a second pass: along every line across the carrier, DFT of the
 * complex signal, keep the bins with |k| < B_c len, inverse DFT with 1/len.
 * ------------------------------------------------------------------------------- */
int orc_cross_band(double* gamma, int32_t H, int32_t W, int32_t carrier_axis, double Bc) {
    if (!(Bc > 0.0)) return 0;
    int32_t nlines = carrier_axis == 0 ? W : H;  /* lines across the carrier */
    int32_t len = carrier_axis == 0 ? H : W;
    int err = 0;
#pragma omp parallel for schedule(dynamic)
    for (int32_t li = 0; li < nlines; ++li) {
        cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)len);
        cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)len);
        cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)len);
        if (!g || !X || !tw) { err = -2; free(g); free(X); free(tw); continue; }
        for (int32_t m = 0; m < len; ++m) {
            double a = 2.0 * ORC_PI * (double)m / (double)len;
            tw[m] = cos(a) - I * sin(a);
        }
        for (int32_t n = 0; n < len; ++n) {
            size_t idx = carrier_axis == 0 ? (size_t)n * W + li : (size_t)li * W + n;
            g[n] = gamma[2 * idx] + I * gamma[2 * idx + 1];
        }
        for (int32_t k = 0; k < len; ++k) {
            int32_t ks = 2 * (int64_t)k < len ? k : k - len; /* signed bin */
            if (!(fabs((double)ks) < Bc * (double)len)) { X[k] = 0.0; continue; }
            cplx acc = 0.0;
            for (int32_t n = 0; n < len; ++n) acc += g[n] * tw[((int64_t)k * n) % len];
            X[k] = acc;
        }
        for (int32_t n = 0; n < len; ++n) {
            cplx acc = 0.0;
            for (int32_t k = 0; k < len; ++k)
                if (X[k] != 0.0) acc += X[k] * conj(tw[((int64_t)k * n) % len]);
            acc /= (double)len;
            size_t idx = carrier_axis == 0 ? (size_t)n * W + li : (size_t)li * W + n;
            gamma[2 * idx] = creal(acc);
            gamma[2 * idx + 1] = cimag(acc);
        }
        free(g);
        free(X);
        free(tw);
    }
    return err;
}

/* Step 2 skipped (model orders p > 1 on real fringes): Gamma is the real frame with the mean
   of every carrier line removed (the band-pass drops that zero frequency too), imaginary part 0. */
static void orc_raw_frame(const void* frame, int32_t dtype, int32_t H, int32_t W, int32_t carrier_axis,
                          double* gamma) {
    int32_t nlines = carrier_axis == 0 ? H : W;
    int32_t len = carrier_axis == 0 ? W : H;
    for (int32_t li = 0; li < nlines; ++li) {
        double mean = 0.0;
        for (int32_t n = 0; n < len; ++n)
            mean += orc_sample(frame, dtype, carrier_axis == 0 ? (size_t)li * W + n : (size_t)n * W + li);
        mean /= (double)len;
        for (int32_t n = 0; n < len; ++n) {
            size_t idx = carrier_axis == 0 ? (size_t)li * W + n : (size_t)n * W + li;
            gamma[2 * idx] = orc_sample(frame, dtype, idx) - mean;
            gamma[2 * idx + 1] = 0.0;
        }
    }
}

/* Step 2 as configured: the analytic signal of the frame, then the cross band if any. */
static int orc_gamma_of(const void* frame, int32_t dtype, int32_t H, int32_t W, const orc_params* p,
                        double* gamma) {
    if (p->raw_input && dtype != ORC_C64 && dtype != ORC_C128) {
        orc_raw_frame(frame, dtype, H, W, p->carrier_axis, gamma);
        return orc_cross_band(gamma, H, W, p->carrier_axis, p->band_cross);
    }
    double B = p->band_halfwidth > 0 ? p->band_halfwidth : 0.5 * p->carrier_freq;
    int err = orc_analytic_frame(frame, dtype, H, W, p->carrier_axis, p->carrier_freq, B, gamma);
    if (!err) err = orc_cross_band(gamma, H, W, p->carrier_axis, p->band_cross);
    return err;
}

/* ---------------------------------------------------------------------------------
 * Step 4 -- sample auto-correlation matrix of one window (Sec. 3, Eq. 4-5:
 * R = E{Gamma_w Gamma_w^H} = R_s + sigma^2 I).
 * The window w[0..N-1] yields K = N - L + 1 snapshots s_i[m] = w[i + m];
 * R_f[m][l] = (1/K) sum_i s_i[m] conj(s_i[l]). With forward-backward averaging
 * R = (R_f + J conj(R_f) J) / 2, i.e. R[m][l] = (R_f[m][l] + conj(R_f[L-1-m][L-1-l])) / 2.
 * R is L*L row-major.
 * ------------------------------------------------------------------------------- */
void orc_covariance(const cplx* w, int32_t N, int32_t L, int32_t fb, cplx* R) {
    int32_t K = N - L + 1;
    cplx Rf[ORC_MAXL * ORC_MAXL];
    for (int32_t m = 0; m < L; ++m)
        for (int32_t l = 0; l < L; ++l) {
            cplx acc = 0.0;
            for (int32_t i = 0; i < K; ++i) acc += w[i + m] * conj(w[i + l]);
            Rf[m * L + l] = acc / (double)K;
        }
    for (int32_t m = 0; m < L; ++m)
        for (int32_t l = 0; l < L; ++l) {
            if (fb)
                R[m * L + l] = 0.5 * (Rf[m * L + l] + conj(Rf[(L - 1 - m) * L + (L - 1 - l)]));
            else
                R[m * L + l] = Rf[m * L + l];
        }
}

/* ---------------------------------------------------------------------------------
 * Step 5 -- eigen-decomposition of the Hermitian R (Sec. 3, Eq. 8-11: u1 is the
 * eigenvector of the largest eigenvalue, the rest span the noise subspace).
 * Cyclic complex Jacobi: for each pivot (p, q) with a_pq = |a_pq| e, the unitary G with
 * G_pp = G_qq = c, G_pq = s e, G_qp = -s conj(e) and t = s/c the smaller root of
 * t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 |a_pq|), annihilates a_pq in G^H A G.
 * Sweeps repeat until the off-diagonal Frobenius norm is below 1e-14 ||R||_F.
 * On return evals[] holds the eigenvalues (unsorted, as the diagonal ends) and column j of
 * V (row-major L*L) the eigenvector of evals[j]. Returns the sweeps used, or -1 if 100
 * sweeps did not converge.
 * ------------------------------------------------------------------------------- */
int orc_eig_hermitian(const cplx* R, int32_t L, double* evals, cplx* V) {
    cplx A[ORC_MAXL * ORC_MAXL];
    memcpy(A, R, sizeof(cplx) * (size_t)L * L);
    for (int32_t r = 0; r < L; ++r)
        for (int32_t c = 0; c < L; ++c) V[r * L + c] = (r == c) ? 1.0 : 0.0;
    double normA = 0.0;
    for (int32_t i = 0; i < L * L; ++i) normA += creal(A[i] * conj(A[i]));
    normA = sqrt(normA);
    int sweeps = 0;
    int converged = 0;
    for (sweeps = 0; sweeps <= 100; ++sweeps) {
        double off = 0.0;
        for (int32_t p = 0; p < L; ++p)
            for (int32_t q = 0; q < L; ++q)
                if (p != q) off += creal(A[p * L + q] * conj(A[p * L + q]));
        off = sqrt(off);
        if (off <= 1e-14 * normA) { converged = 1; break; }
        if (sweeps == 100) break;
        for (int32_t p = 0; p < L - 1; ++p)
            for (int32_t q = p + 1; q < L; ++q) {
                cplx b = A[p * L + q];
                double ab = cabs(b);
                if (ab == 0.0) continue;
                cplx e = b / ab;
                double tau = (creal(A[q * L + q]) - creal(A[p * L + p])) / (2.0 * ab);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                for (int32_t r = 0; r < L; ++r) {
                    if (r == p || r == q) continue;
                    cplx arp = A[r * L + p], arq = A[r * L + q];
                    A[r * L + p] = c * arp - s * conj(e) * arq;
                    A[r * L + q] = s * e * arp + c * arq;
                    A[p * L + r] = conj(A[r * L + p]);
                    A[q * L + r] = conj(A[r * L + q]);
                }
                double app = creal(A[p * L + p]) - t * ab;
                double aqq = creal(A[q * L + q]) + t * ab;
                A[p * L + p] = app;
                A[q * L + q] = aqq;
                A[p * L + q] = 0.0;
                A[q * L + p] = 0.0;
                for (int32_t r = 0; r < L; ++r) {
                    cplx vrp = V[r * L + p], vrq = V[r * L + q];
                    V[r * L + p] = c * vrp - s * conj(e) * vrq;
                    V[r * L + q] = s * e * vrp + c * vrq;
                }
            }
    }
    for (int32_t j = 0; j < L; ++j) evals[j] = creal(A[j * L + j]);
    return converged ? sweeps : -1;
}

/* ---------------------------------------------------------------------------------
 * Step 6 -- root-MUSIC polynomial (Sec. 3, Eq. 12-14): with model order 1 the noise
 * subspace projector is U_n U_n^H = C = I - u1 u1^H. On the unit circle
 * u(z)^H C u(z) = sum_{m,l} z^-m C[m][l] z^l = sum_k c_k z^k, c_k = sum_{l-m=k} C[m][l].
 * Multiplying by z^(L-1) gives Q(z) = sum_i q_i z^i, q_i = c_{i-(L-1)}, i = 0..2L-2.
 * u must have unit norm. q has 2L-1 entries, q[i] multiplies z^i.
 * ------------------------------------------------------------------------------- */
void orc_music_poly(const cplx* u, int32_t L, cplx* q) {
    for (int32_t i = 0; i < 2 * L - 1; ++i) q[i] = 0.0;
    for (int32_t m = 0; m < L; ++m)
        for (int32_t l = 0; l < L; ++l) {
            cplx Cml = (m == l ? 1.0 : 0.0) - u[m] * conj(u[l]);
            q[(l - m) + (L - 1)] += Cml;
        }
}

/* ---------------------------------------------------------------------------------
 * Step 7 -- all roots of Q (Sec. 3: the paper takes the eigenvalues of the companion
 * matrix; any method that returns all roots gives the same set). Simultaneous
 * Aberth-Ehrlich iteration in FP64: z_i <- z_i - w_i, w_i = N_i / (1 - N_i S_i),
 * N_i = Q(z_i)/Q'(z_i), S_i = sum_{j != i} 1/(z_i - z_j), updated in place. A root is
 * accepted once |Q(z_i)| <= 1e-14 sum_k |q_k| |z_i|^k (the value is at the rounding
 * level), and two closing sweeps refine all roots together. Exact zero leading coefficients
 * (roots at infinity) are dropped; exact zero trailing coefficients give roots at 0.
 * q[0..deg] ascending powers. Writes the finite roots to roots[] and returns their
 * count; *not_conv is set when 500 iterations did not settle every root.
 * ------------------------------------------------------------------------------- */
static void orc_horner(const cplx* q, int32_t deg, cplx z, cplx* p, cplx* dp, double* bound) {
    cplx pv = q[deg], dv = 0.0;
    double b = cabs(q[deg]);
    double az = cabs(z);
    for (int32_t i = deg - 1; i >= 0; --i) {
        dv = dv * z + pv;
        pv = pv * z + q[i];
        b = b * az + cabs(q[i]);
    }
    *p = pv;
    *dp = dv;
    *bound = b;
}

int orc_poly_roots(const cplx* q_in, int32_t deg, cplx* roots, int32_t* not_conv) {
    cplx q[2 * ORC_MAXL];
    *not_conv = 0;
    while (deg > 0 && q_in[deg] == 0.0) --deg; /* roots at infinity */
    int32_t nzero = 0;
    while (nzero < deg && q_in[nzero] == 0.0) ++nzero; /* roots at the origin */
    int32_t n = deg - nzero;
    for (int32_t i = 0; i <= n; ++i) q[i] = q_in[i + nzero];
    for (int32_t i = 0; i < nzero; ++i) roots[i] = 0.0;
    cplx* z = roots + nzero;
    if (n <= 0) return nzero;
    /* Initial guesses on the circle of radius |q0/qn|^(1/n), the geometric mean of the
       root moduli, at angles offset from the real axis. */
    double r0 = pow(cabs(q[0]) / cabs(q[n]), 1.0 / (double)n);
    for (int32_t i = 0; i < n; ++i) {
        double a = 2.0 * ORC_PI * (double)i / (double)n + 0.7;
        z[i] = r0 * (cos(a) + I * sin(a));
    }
    int done[2 * ORC_MAXL];
    for (int32_t i = 0; i < n; ++i) done[i] = 0;
    int it;
    for (it = 0; it < 500; ++it) {
        int active = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (done[i]) continue;
            cplx p, dp;
            double b;
            orc_horner(q, n, z[i], &p, &dp, &b);
            if (cabs(p) <= 1e-14 * b) { done[i] = 1; continue; }
            active = 1;
            if (dp == 0.0) { z[i] *= (1.0 + 1e-7 * I); continue; }
            cplx Ni = p / dp;
            cplx Si = 0.0;
            for (int32_t j = 0; j < n; ++j)
                if (j != i) Si += 1.0 / (z[i] - z[j]);
            z[i] -= Ni / (1.0 - Ni * Si);
        }
        if (!active) break;
    }
    if (it == 500) *not_conv = 1;
    /* The residual test accepts a root once its backward error is at the rounding level; for
       a simple root lying close to another one (a pair z, 1/conj(z) near the circle) the
       forward error can still be ~1e-9. Two more Aberth sweeps, whose corrections account for
       the neighbouring roots, bring such roots to the accuracy the double-precision
       coefficients allow. Roots with another root within 1e-6 (one double root split by
       rounding, resolved in the selection step) are left as they are, and a correction is
       kept only if it lowers |Q|. */
    for (int sweep = 0; sweep < 2; ++sweep)
        for (int32_t i = 0; i < n; ++i) {
            double near = INFINITY;
            for (int32_t j = 0; j < n; ++j)
                if (j != i && cabs(z[i] - z[j]) < near) near = cabs(z[i] - z[j]);
            if (!(near >= 1e-6)) continue;
            cplx p, dp;
            double b;
            orc_horner(q, n, z[i], &p, &dp, &b);
            if (p == 0.0 || dp == 0.0) continue;
            cplx Ni = p / dp;
            cplx Si = 0.0;
            for (int32_t j = 0; j < n; ++j)
                if (j != i) Si += 1.0 / (z[i] - z[j]);
            cplx w = Ni / (1.0 - Ni * Si);
            if (!(isfinite(creal(w)) && isfinite(cimag(w)))) continue;
            cplx p2, dp2;
            double b2;
            orc_horner(q, n, z[i] - w, &p2, &dp2, &b2);
            if (cabs(p2) < cabs(p)) z[i] -= w;
        }
    return n + nzero;
}

/* ---------------------------------------------------------------------------------
 * Step 8 -- root selection (Sec. 3 and Algorithm 1: the root closest to the unit circle
 * with magnitude less than one). Candidates: |z| <= 1 + 1e-9 (so that a double root lying
 * on the circle, split by rounding, still qualifies). The candidate with the smallest
 * ||z| - 1| wins; exact ties go to the smaller |wrap(arg z - omega_ref)|.
 * A noise-free window makes the winner a double root (Eq. 7-8: R_s has rank one, so the
 * polynomial touches zero on the circle). Rounding splits a double root into two roots
 * about sqrt(eps) apart whose positions are only accurate to that level, so when another
 * root lies within 1e-6 of the winner the pair is taken as one double root and located as
 * the root of Q' between them (Newton on Q' from the pair's mean). Returns 0, or -1 if no
 * candidate exists. q[0..deg] are Q's coefficients, ascending.
 * ------------------------------------------------------------------------------- */
static double orc_wrap(double a) {
    while (a > ORC_PI) a -= 2.0 * ORC_PI;
    while (a <= -ORC_PI) a += 2.0 * ORC_PI;
    return a;
}

/* Q'(z) and Q''(z) by Horner's rule. */
static void orc_horner_d12(const cplx* q, int32_t deg, cplx z, cplx* d1, cplx* d2) {
    cplx p = q[deg], a1 = 0.0, a2 = 0.0;
    for (int32_t i = deg - 1; i >= 0; --i) {
        a2 = a2 * z + a1;
        a1 = a1 * z + p;
        p = p * z + q[i];
    }
    *d1 = a1;
    *d2 = 2.0 * a2;
}

int orc_select_root(const cplx* q, int32_t deg, const cplx* roots, int32_t n, double omega_ref,
                    cplx* zsel) {
    int32_t best = -1;
    double bestd = INFINITY, bestt = INFINITY;
    for (int32_t i = 0; i < n; ++i) {
        double r = cabs(roots[i]);
        if (!(r <= 1.0 + 1e-9)) continue;
        double d = fabs(r - 1.0);
        double t = fabs(orc_wrap(carg(roots[i]) - omega_ref));
        if (d < bestd || (d == bestd && t < bestt)) { best = i; bestd = d; bestt = t; }
    }
    if (best < 0) return -1;
    int32_t near = -1;
    double neard = INFINITY;
    for (int32_t j = 0; j < n; ++j) {
        if (j == best) continue;
        double d = cabs(roots[j] - roots[best]);
        if (d < neard) { neard = d; near = j; }
    }
    if (near < 0 || !(neard < 1e-6)) {
        *zsel = roots[best];
        return 0;
    }
    cplx z = 0.5 * (roots[best] + roots[near]);
    for (int it = 0; it < 16; ++it) {
        cplx d1, d2;
        orc_horner_d12(q, deg, z, &d1, &d2);
        if (d2 == 0.0) break;
        cplx step = d1 / d2;
        z -= step;
        if (cabs(step) <= 1e-16 * cabs(z)) break;
    }
    /* keep the polished point only if it stayed inside the cluster */
    if (cabs(z - roots[best]) <= 2.0 * neard)
        *zsel = z;
    else
        *zsel = 0.5 * (roots[best] + roots[near]);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Step 5 with model order one (Sec. 3, Eq. 9-11): the unit-norm eigenvector u of the
 * largest eigenvalue of the Hermitian L x L matrix R spans the signal subspace. Returns
 * ORC_OK, ORC_NOT_CONVERGED (the Jacobi sweeps did not settle) or ORC_DEGENERATE (R = 0,
 * or lambda1 - lambda2 <= 1e-12 lambda1: no unique signal subspace).
 * ------------------------------------------------------------------------------- */
static int orc_principal_vector(const cplx* R, int32_t L, cplx* u) {
    cplx V[ORC_MAXL * ORC_MAXL];
    double ev[ORC_MAXL];
    double normR = 0.0;
    for (int32_t i = 0; i < L * L; ++i) normR += creal(R[i] * conj(R[i]));
    if (!(normR > 0.0)) return ORC_DEGENERATE;
    int sweeps = orc_eig_hermitian(R, L, ev, V);
    int status = sweeps < 0 ? ORC_NOT_CONVERGED : ORC_OK;
    /* largest and second largest eigenvalue */
    int32_t j1 = 0;
    for (int32_t j = 1; j < L; ++j)
        if (ev[j] > ev[j1]) j1 = j;
    double l2 = -INFINITY;
    for (int32_t j = 0; j < L; ++j)
        if (j != j1 && ev[j] > l2) l2 = ev[j];
    if (!(ev[j1] - l2 > 1e-12 * ev[j1])) return ORC_DEGENERATE;
    double nu = 0.0;
    for (int32_t m = 0; m < L; ++m) nu += creal(V[m * L + j1] * conj(V[m * L + j1]));
    nu = sqrt(nu);
    for (int32_t m = 0; m < L; ++m) u[m] = V[m * L + j1] / nu;
    return status;
}

/* ---------------------------------------------------------------------------------
 * Steps 4-9 for one window w[0..N-1] of the analytic signal. omega_ref is the carrier
 * phase step removed from the angle (2 pi f0 when the window runs along the carrier,
 * else 0). Writes the derivative wrap(arg z - omega_ref) (Sec. 3, Eq. 15) and returns the
 * status. Optional outputs (may be NULL): u1 (L), q (2L-1), roots (2L-2), zsel (1).
 * ------------------------------------------------------------------------------- */
int orc_window_derivative(const cplx* w, int32_t N, int32_t L, int32_t fb, double omega_ref,
                          double* deriv, cplx* u1_out, cplx* q_out, cplx* roots_out,
                          int32_t* nroots_out, cplx* zsel_out) {
    cplx R[ORC_MAXL * ORC_MAXL], u[ORC_MAXL], q[2 * ORC_MAXL];
    cplx roots[2 * ORC_MAXL];
    *deriv = NAN;
    if (L < 2 || L > ORC_MAXL || N < L) return ORC_DEGENERATE;
    orc_covariance(w, N, L, fb, R);
    int status = orc_principal_vector(R, L, u);
    if (status == ORC_DEGENERATE) return ORC_DEGENERATE;
    orc_music_poly(u, L, q);
    int32_t nc = 0;
    int32_t nr = orc_poly_roots(q, 2 * L - 2, roots, &nc);
    if (nc) status = ORC_NOT_CONVERGED;
    cplx z;
    if (orc_select_root(q, 2 * L - 2, roots, nr, omega_ref, &z) != 0) return ORC_DEGENERATE;
    *deriv = orc_wrap(carg(z) - omega_ref);
    if (u1_out) memcpy(u1_out, u, sizeof(cplx) * (size_t)L);
    if (q_out) memcpy(q_out, q, sizeof(cplx) * (size_t)(2 * L - 1));
    if (roots_out) memcpy(roots_out, roots, sizeof(cplx) * (size_t)nr);
    if (nroots_out) *nroots_out = nr;
    if (zsel_out) *zsel_out = z;
    return status;
}

/* ctypes-friendly form of the above: complex arrays interleaved (re, im). */
int orc_window_derivative_ri(const double* w_ri, int32_t N, int32_t L, int32_t fb,
                             double omega_ref, double* deriv, double* u1_ri, double* q_ri,
                             double* roots_ri, int32_t* nroots, double* zsel_ri) {
    cplx w[4096];
    if (N > 4096) return ORC_DEGENERATE;
    for (int32_t i = 0; i < N; ++i) w[i] = w_ri[2 * i] + I * w_ri[2 * i + 1];
    cplx u[ORC_MAXL], q[2 * ORC_MAXL], r[2 * ORC_MAXL], z = 0.0;
    int32_t nr = 0;
    int st = orc_window_derivative(w, N, L, fb, omega_ref, deriv, u, q, r, &nr, &z);
    if (u1_ri) for (int32_t i = 0; i < L; ++i) { u1_ri[2 * i] = creal(u[i]); u1_ri[2 * i + 1] = cimag(u[i]); }
    if (q_ri) for (int32_t i = 0; i < 2 * L - 1; ++i) { q_ri[2 * i] = creal(q[i]); q_ri[2 * i + 1] = cimag(q[i]); }
    if (roots_ri) for (int32_t i = 0; i < nr; ++i) { roots_ri[2 * i] = creal(r[i]); roots_ri[2 * i + 1] = cimag(r[i]); }
    if (nroots) *nroots = nr;
    if (zsel_ri) { zsel_ri[0] = creal(z); zsel_ri[1] = cimag(z); }
    return st;
}

/* ---------------------------------------------------------------------------------
 * Model order p > 1 (Sec. 3 with p exponentials per window instead of one: a real fringe
 * without the analytic step carries the two exponentials exp(+-j omega) of its cosine, plus one
 * at zero frequency for a local offset). Step 5 keeps the p largest eigenvalues' eigenvectors:
 * the noise projector is C = I - sum_{i<p} u_i u_i^H (degenerate if lambda_p - lambda_{p+1}
 * <= 1e-12 lambda_1); step 6 forms the polynomial from C; step 8 takes the p candidate roots
 * nearest the unit circle (a split double root counted once) and, among them, the one whose
 * angle is nearest omega_ref (the expected angle: the carrier's along the carrier axis), then
 * applies the split-double-root rule to it.
 * ------------------------------------------------------------------------------- */
static int orc_noise_projector(const cplx* R, int32_t L, int32_t p, cplx* C) {
    cplx V[ORC_MAXL * ORC_MAXL];
    double ev[ORC_MAXL];
    int32_t order[ORC_MAXL];
    double normR = 0.0;
    for (int32_t i = 0; i < L * L; ++i) normR += creal(R[i] * conj(R[i]));
    if (!(normR > 0.0) || p < 1 || p >= L) return ORC_DEGENERATE;
    int sweeps = orc_eig_hermitian(R, L, ev, V);
    int status = sweeps < 0 ? ORC_NOT_CONVERGED : ORC_OK;
    /* eigenvalue indices by decreasing eigenvalue (insertion sort, stable) */
    for (int32_t j = 0; j < L; ++j) {
        int32_t t = j;
        while (t > 0 && ev[order[t - 1]] < ev[j]) { order[t] = order[t - 1]; --t; }
        order[t] = j;
    }
    if (!(ev[order[p - 1]] - ev[order[p]] > 1e-12 * ev[order[0]])) return ORC_DEGENERATE;
    for (int32_t m = 0; m < L; ++m)
        for (int32_t l = 0; l < L; ++l) C[m * L + l] = (m == l) ? 1.0 : 0.0;
    for (int32_t i = 0; i < p; ++i) {
        int32_t j = order[i];
        double nu = 0.0;
        for (int32_t m = 0; m < L; ++m) nu += creal(V[m * L + j] * conj(V[m * L + j]));
        for (int32_t m = 0; m < L; ++m)
            for (int32_t l = 0; l < L; ++l) C[m * L + l] -= V[m * L + j] * conj(V[l * L + j]) / nu;
    }
    return status;
}

/* Step 6 from a projector C: c_k = sum_{l-m=k} C[m][l], q[i] = c_{i-(L-1)}. */
static void orc_music_poly_C(const cplx* C, int32_t L, cplx* q) {
    for (int32_t i = 0; i < 2 * L - 1; ++i) q[i] = 0.0;
    for (int32_t m = 0; m < L; ++m)
        for (int32_t l = 0; l < L; ++l) q[(l - m) + (L - 1)] += C[m * L + l];
}

int orc_select_root_p(const cplx* q, int32_t deg, const cplx* roots, int32_t n, int32_t p,
                      double omega_ref, cplx* zsel) {
    int32_t near_idx[3] = {-1, -1, -1};
    double near_d[3] = {INFINITY, INFINITY, INFINITY};
    if (p < 1 || p > 3) return -1;
    /* the p candidates nearest the circle, taken by increasing distance (earlier index first on
       equal distance); a root within 1e-6 of one already taken is the other half of a split
       double root and is not counted again */
    for (int32_t t = 0; t < p; ++t) {
        for (int32_t i = 0; i < n; ++i) {
            double r = cabs(roots[i]);
            if (!(r <= 1.0 + 1e-9)) continue;
            double d = fabs(r - 1.0);
            int taken = 0;
            for (int32_t u = 0; u < t; ++u)
                if (i == near_idx[u] || cabs(roots[i] - roots[near_idx[u]]) < 1e-6) taken = 1;
            if (!taken && d < near_d[t]) { near_d[t] = d; near_idx[t] = i; }
        }
    }
    int32_t best = -1;
    double bestt = INFINITY;
    for (int32_t t = 0; t < p; ++t) {
        if (near_idx[t] < 0) continue;
        double a = fabs(orc_wrap(carg(roots[near_idx[t]]) - omega_ref));
        if (a < bestt) { bestt = a; best = near_idx[t]; }
    }
    if (best < 0) return -1;
    /* the split-double-root rule of step 8 for the chosen root */
    int32_t nb = -1;
    double nd = INFINITY;
    for (int32_t j = 0; j < n; ++j) {
        if (j == best) continue;
        double d = cabs(roots[j] - roots[best]);
        if (d < nd) { nd = d; nb = j; }
    }
    if (nb < 0 || !(nd < 1e-6)) { *zsel = roots[best]; return 0; }
    cplx z = 0.5 * (roots[best] + roots[nb]);
    for (int it = 0; it < 16; ++it) {
        cplx d1, d2;
        orc_horner_d12(q, deg, z, &d1, &d2);
        if (d2 == 0.0) break;
        cplx step = d1 / d2;
        z -= step;
        if (cabs(step) <= 1e-16 * cabs(z)) break;
    }
    *zsel = cabs(z - roots[best]) <= 2.0 * nd ? z : 0.5 * (roots[best] + roots[nb]);
    return 0;
}

/* Steps 4-9 with model order p (p = 1 is orc_window_derivative). */
int orc_window_derivative_p(const cplx* w, int32_t N, int32_t L, int32_t fb, int32_t p,
                            double omega_ref, double* deriv, cplx* zsel_out) {
    if (p == 1) return orc_window_derivative(w, N, L, fb, omega_ref, deriv, NULL, NULL, NULL, NULL, zsel_out);
    cplx R[ORC_MAXL * ORC_MAXL], C[ORC_MAXL * ORC_MAXL], q[2 * ORC_MAXL], roots[2 * ORC_MAXL];
    *deriv = NAN;
    if (L < 2 || L > ORC_MAXL || N < L || p < 1 || p > 3 || p >= L) return ORC_DEGENERATE;
    orc_covariance(w, N, L, fb, R);
    int status = orc_noise_projector(R, L, p, C);
    if (status == ORC_DEGENERATE) return ORC_DEGENERATE;
    orc_music_poly_C(C, L, q);
    int32_t nc = 0;
    int32_t nr = orc_poly_roots(q, 2 * L - 2, roots, &nc);
    if (nc) status = ORC_NOT_CONVERGED;
    cplx z;
    if (orc_select_root_p(q, 2 * L - 2, roots, nr, p, omega_ref, &z) != 0) return ORC_DEGENERATE;
    *deriv = orc_wrap(carg(z) - omega_ref);
    if (zsel_out) *zsel_out = z;
    return status;
}

int orc_window_derivative_p_ri(const double* w_ri, int32_t N, int32_t L, int32_t fb, int32_t p,
                               double omega_ref, double* deriv, double* zsel_ri) {
    cplx w[4096], z = 0.0;
    if (N > 4096) return ORC_DEGENERATE;
    for (int32_t i = 0; i < N; ++i) w[i] = w_ri[2 * i] + I * w_ri[2 * i + 1];
    int st = orc_window_derivative_p(w, N, L, fb, p, omega_ref, deriv, &z);
    zsel_ri[0] = creal(z);
    zsel_ri[1] = cimag(z);
    return st;
}

/* ctypes-friendly wrappers for the individual steps (used by the pin tests). */
void orc_covariance_ri(const double* w_ri, int32_t N, int32_t L, int32_t fb, double* R_ri) {
    cplx w[4096], R[ORC_MAXL * ORC_MAXL];
    for (int32_t i = 0; i < N && i < 4096; ++i) w[i] = w_ri[2 * i] + I * w_ri[2 * i + 1];
    orc_covariance(w, N, L, fb, R);
    for (int32_t i = 0; i < L * L; ++i) { R_ri[2 * i] = creal(R[i]); R_ri[2 * i + 1] = cimag(R[i]); }
}

int orc_eig_hermitian_ri(const double* R_ri, int32_t L, double* evals, double* V_ri) {
    cplx R[ORC_MAXL * ORC_MAXL], V[ORC_MAXL * ORC_MAXL];
    for (int32_t i = 0; i < L * L; ++i) R[i] = R_ri[2 * i] + I * R_ri[2 * i + 1];
    int s = orc_eig_hermitian(R, L, evals, V);
    for (int32_t i = 0; i < L * L; ++i) { V_ri[2 * i] = creal(V[i]); V_ri[2 * i + 1] = cimag(V[i]); }
    return s;
}

void orc_music_poly_ri(const double* u_ri, int32_t L, double* q_ri) {
    cplx u[ORC_MAXL], q[2 * ORC_MAXL];
    for (int32_t i = 0; i < L; ++i) u[i] = u_ri[2 * i] + I * u_ri[2 * i + 1];
    orc_music_poly(u, L, q);
    for (int32_t i = 0; i < 2 * L - 1; ++i) { q_ri[2 * i] = creal(q[i]); q_ri[2 * i + 1] = cimag(q[i]); }
}

int orc_poly_roots_ri(const double* q_ri, int32_t deg, double* roots_ri, int32_t* not_conv) {
    cplx q[2 * ORC_MAXL], r[2 * ORC_MAXL];
    if (deg >= 2 * ORC_MAXL) return -1;
    for (int32_t i = 0; i <= deg; ++i) q[i] = q_ri[2 * i] + I * q_ri[2 * i + 1];
    int32_t n = orc_poly_roots(q, deg, r, not_conv);
    for (int32_t i = 0; i < n; ++i) { roots_ri[2 * i] = creal(r[i]); roots_ri[2 * i + 1] = cimag(r[i]); }
    return n;
}

int orc_select_root_ri(const double* q_ri, int32_t deg, const double* roots_ri, int32_t n,
                       double omega_ref, double* zsel_ri) {
    cplx q[2 * ORC_MAXL], r[2 * ORC_MAXL], z = 0.0;
    if (deg >= 2 * ORC_MAXL || n > 2 * ORC_MAXL) return -1;
    for (int32_t i = 0; i <= deg; ++i) q[i] = q_ri[2 * i] + I * q_ri[2 * i + 1];
    for (int32_t i = 0; i < n; ++i) r[i] = roots_ri[2 * i] + I * roots_ri[2 * i + 1];
    int s = orc_select_root(q, deg, r, n, omega_ref, &z);
    zsel_ri[0] = creal(z);
    zsel_ri[1] = cimag(z);
    return s;
}

/* ---------------------------------------------------------------------------------
 * Step 3 plus steps 4-9 over the pixels of one frame whose analytic signal gamma (H*W
 * interleaved complex, row-major) is given. The window of the pixel at position n of its
 * line along the derivative axis covers n - floor(N/2) .. n - floor(N/2) + N - 1; if that
 * leaves the line the pixel is a border pixel (Sec. 4: border pixels are neglected).
 * ------------------------------------------------------------------------------- */
static int orc_pixel(const double* gamma, int32_t H, int32_t W, const orc_params* p,
                     int32_t y, int32_t x, double* out) {
    int32_t N = p->window_len;
    int32_t len = p->deriv_axis == 0 ? W : H;
    int32_t n = p->deriv_axis == 0 ? x : y;
    int32_t start = n - N / 2;
    *out = NAN;
    if (start < 0 || start + N - 1 > len - 1) return ORC_BORDER;
    if (p->model_order < 1 || p->model_order > 3) return ORC_DEGENERATE;
    cplx w[4096];
    if (N > 4096) return ORC_DEGENERATE;
    for (int32_t i = 0; i < N; ++i) {
        size_t idx = p->deriv_axis == 0 ? (size_t)y * W + (size_t)(start + i)
                                        : (size_t)(start + i) * W + (size_t)x;
        w[i] = gamma[2 * idx] + I * gamma[2 * idx + 1];
    }
    double omega_ref = p->deriv_axis == p->carrier_axis ? 2.0 * ORC_PI * p->carrier_freq : 0.0;
    return orc_window_derivative_p(w, N, p->cov_order, p->forward_backward, p->model_order, omega_ref, out,
                                   NULL);
}

/* Whole-frame demodulation: derivative map out[H*W] (NaN where undefined) and status[H*W]
   (may be NULL). nthreads > 0 sets the OpenMP thread count. Returns the thread count
   used, or a negative value on error. */
int orc_demodulate(const void* frame, int32_t dtype, int32_t H, int32_t W, const orc_params* p,
                   double* out, uint8_t* status, int32_t nthreads) {
    if (H <= 0 || W <= 0 || p->window_len < 2 || p->cov_order < 2 ||
        p->cov_order > ORC_MAXL || p->cov_order > p->window_len)
        return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    double* gamma = (double*)malloc(sizeof(double) * 2 * (size_t)H * W);
    if (!gamma) return -2;
    int err = orc_gamma_of(frame, dtype, H, W, p, gamma);
    if (err) { free(gamma); return err; }
    int used = 1;
#pragma omp parallel for schedule(dynamic)
    for (int32_t y = 0; y < H; ++y) {
#ifdef _OPENMP
        if (y == 0) used = omp_get_num_threads();
#endif
        for (int32_t x = 0; x < W; ++x) {
            double d;
            int st = orc_pixel(gamma, H, W, p, y, x, &d);
            out[(size_t)y * W + x] = d;
            if (status) status[(size_t)y * W + x] = (uint8_t)st;
        }
    }
    free(gamma);
    return used;
}

/* Step 2 for the carrier lines marked in need[] only (the other lines of gamma are left
   untouched); a complex frame is copied whole. Returns the OpenMP thread count used. */
static int orc_gamma_lines(const void* frame, int32_t dtype, int32_t H, int32_t W, int32_t ca,
                           double f0, double B, const uint8_t* need, double* gamma) {
    if (dtype == ORC_C64 || dtype == ORC_C128) {
        orc_analytic_frame(frame, dtype, H, W, ca, f0, B, gamma);
        return 1;
    }
    int32_t nlines = ca == 0 ? H : W;
    int32_t len = ca == 0 ? W : H;
    int used = 1;
#pragma omp parallel for schedule(dynamic)
    for (int32_t li = 0; li < nlines; ++li) {
#ifdef _OPENMP
        if (li == 0) used = omp_get_num_threads();
#endif
        if (!need[li]) continue;
        double* v = (double*)malloc(sizeof(double) * (size_t)len);
        double* g = (double*)malloc(sizeof(double) * 2 * (size_t)len);
        if (!v || !g) { free(v); free(g); continue; }
        for (int32_t n = 0; n < len; ++n) {
            size_t idx = ca == 0 ? (size_t)li * W + n : (size_t)n * W + li;
            v[n] = orc_sample(frame, dtype, idx);
        }
        orc_analytic_line(v, len, f0, B, g);
        for (int32_t n = 0; n < len; ++n) {
            size_t idx = ca == 0 ? (size_t)li * W + n : (size_t)n * W + li;
            gamma[2 * idx] = g[2 * n];
            gamma[2 * idx + 1] = g[2 * n + 1];
        }
        free(v);
        free(g);
    }
    return used;
}

/* Sampled demodulation: only the listed pixels (ys[i], xs[i]) are computed. Only the
   lines the samples need are band-passed. Returns the thread count used, or < 0. */
int orc_demodulate_pixels(const void* frame, int32_t dtype, int32_t H, int32_t W,
                          const orc_params* p, int32_t npix, const int32_t* ys,
                          const int32_t* xs, double* out, uint8_t* status, int32_t nthreads) {
    if (H <= 0 || W <= 0 || p->window_len < 2 || p->cov_order < 2 ||
        p->cov_order > ORC_MAXL || p->cov_order > p->window_len)
        return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int32_t ca = p->carrier_axis;
    int32_t nlines = ca == 0 ? H : W;
    double B = p->band_halfwidth > 0 ? p->band_halfwidth : 0.5 * p->carrier_freq;
    /* mark the carrier lines every sample's window touches */
    uint8_t* need = (uint8_t*)calloc((size_t)nlines, 1);
    double* gamma = (double*)calloc(2 * (size_t)H * W, sizeof(double));
    if (!need || !gamma) { free(need); free(gamma); return -2; }
    int32_t N = p->window_len;
    for (int32_t i = 0; i < npix; ++i) {
        int32_t y = ys[i], x = xs[i];
        if (y < 0 || y >= H || x < 0 || x >= W) { free(need); free(gamma); return -1; }
        for (int32_t k = -N; k <= N; ++k) {
            /* lines crossed by the window: along the derivative axis when it differs
               from the carrier axis, otherwise the sample's own line */
            int32_t li;
            if (p->deriv_axis == ca) li = ca == 0 ? y : x;
            else li = (ca == 0 ? y : x) + k;
            if (li >= 0 && li < nlines) need[li] = 1;
        }
    }
    int used = 1;
    if (p->band_cross > 0.0 || p->raw_input) {
        /* the cross band mixes all lines (and the raw signal is cheap): the whole frame */
        int err = orc_gamma_of(frame, dtype, H, W, p, gamma);
        if (err) { free(need); free(gamma); return err; }
    } else {
        used = orc_gamma_lines(frame, dtype, H, W, ca, p->carrier_freq, B, need, gamma);
    }
#pragma omp parallel for schedule(dynamic)
    for (int32_t i = 0; i < npix; ++i) {
        double d;
        int st = orc_pixel(gamma, H, W, p, ys[i], xs[i], &d);
        out[i] = d;
        if (status) status[i] = (uint8_t)st;
    }
    free(need);
    free(gamma);
    return used;
}

/* =================================================================================
 * The paper's own geometry (Sec. 3, Eq. 4-15; Algorithm 1): a square block Gamma_w of
 * M x M samples, M = 2 Lp + 1, centred on the pixel. Its columns are the snapshots of
 * the y analysis and its conjugated rows those of the x analysis; both angles and the
 * local phase alpha come out of one block.
 * ================================================================================= */

/* ---------------------------------------------------------------------------------
 * One block G (row-major M x M; row r is the y offset r - Lp, column c the x offset
 * c - Lp). Following Sec. 3:
 *   R_y = (1/M) G G^H       (Eq. 4-5: E{Gamma_w Gamma_w^H}, columns as snapshots),
 *   R_x = (1/M) G^H G       (the x analysis: E{Gamma_w^H Gamma_w}, conjugated rows),
 *   u1, v1 = principal unit eigenvectors of R_y, R_x         (Eq. 9-11; the paper takes
 *            them from the SVD of Gamma_w, which gives the same vectors),
 *   Q_y, Q_x = root-MUSIC polynomials of u1, v1 (Eq. 12, Eq. 13; the construction of
 *            step 6 with L = M), all roots, and the root closest to the unit circle of
 *            magnitude below one (Algorithm 1),
 *   omega_y = arg z_y,  omega_x = -arg z_x                   (Eq. 15, rows 1-2),
 *   alpha   = angle of the block mean of G[r][c] exp(-j(omega_x (c-Lp) + omega_y (r-Lp)))
 *                                                            (Eq. 15, row 3).
 * ref_x and ref_y are the angles expected without modulation (the carrier's 2 pi f0 on
 * its axis, else 0); they only break exact ties in the selection (z_x is compared with
 * -ref_x). Outputs are the raw angles, carrier included. Optional outputs (may be NULL):
 * u1, v1 (M each), zx, zy (1 each).
 * ------------------------------------------------------------------------------- */
int orc_square_window(const cplx* G, int32_t Lp, double ref_x, double ref_y, double* wx,
                      double* wy, double* alpha, cplx* u1_out, cplx* v1_out, cplx* zx_out,
                      cplx* zy_out) {
    int32_t M = 2 * Lp + 1;
    *wx = NAN;
    *wy = NAN;
    *alpha = NAN;
    if (Lp < 1 || M > ORC_MAXL) return ORC_DEGENERATE;
    cplx Ry[ORC_MAXL * ORC_MAXL], Rx[ORC_MAXL * ORC_MAXL], u[ORC_MAXL], v[ORC_MAXL];
    cplx qy[2 * ORC_MAXL], qx[2 * ORC_MAXL], ry[2 * ORC_MAXL], rx[2 * ORC_MAXL];
    for (int32_t m = 0; m < M; ++m)
        for (int32_t l = 0; l < M; ++l) {
            cplx acc = 0.0;
            for (int32_t c = 0; c < M; ++c) acc += G[m * M + c] * conj(G[l * M + c]);
            Ry[m * M + l] = acc / (double)M;
        }
    for (int32_t a = 0; a < M; ++a)
        for (int32_t b = 0; b < M; ++b) {
            cplx acc = 0.0;
            for (int32_t r = 0; r < M; ++r) acc += conj(G[r * M + a]) * G[r * M + b];
            Rx[a * M + b] = acc / (double)M;
        }
    int sy = orc_principal_vector(Ry, M, u);
    int sx = orc_principal_vector(Rx, M, v);
    if (sy == ORC_DEGENERATE || sx == ORC_DEGENERATE) return ORC_DEGENERATE;
    int status = (sy != ORC_OK || sx != ORC_OK) ? ORC_NOT_CONVERGED : ORC_OK;
    orc_music_poly(u, M, qy);
    orc_music_poly(v, M, qx);
    int32_t ncy = 0, ncx = 0;
    int32_t nry = orc_poly_roots(qy, 2 * M - 2, ry, &ncy);
    int32_t nrx = orc_poly_roots(qx, 2 * M - 2, rx, &ncx);
    if (ncy || ncx) status = ORC_NOT_CONVERGED;
    cplx zy, zx;
    if (orc_select_root(qy, 2 * M - 2, ry, nry, ref_y, &zy) != 0) return ORC_DEGENERATE;
    if (orc_select_root(qx, 2 * M - 2, rx, nrx, -ref_x, &zx) != 0) return ORC_DEGENERATE;
    double oy = carg(zy);
    double ox = -carg(zx);
    cplx acc = 0.0;
    for (int32_t r = 0; r < M; ++r)
        for (int32_t c = 0; c < M; ++c)
            acc += G[r * M + c] * cexp(-I * (ox * (double)(c - Lp) + oy * (double)(r - Lp)));
    acc /= (double)(M * M);
    *wx = ox;
    *wy = oy;
    *alpha = carg(acc);
    if (u1_out) memcpy(u1_out, u, sizeof(cplx) * (size_t)M);
    if (v1_out) memcpy(v1_out, v, sizeof(cplx) * (size_t)M);
    if (zx_out) *zx_out = zx;
    if (zy_out) *zy_out = zy;
    return status;
}

/* ctypes-friendly form of orc_square_window: complex arrays interleaved (re, im);
   out3 receives (omega_x, omega_y, alpha), u1/v1 M entries, z2 (zx, zy). */
int orc_square_window_ri(const double* G_ri, int32_t Lp, double ref_x, double ref_y,
                         double* out3, double* u1_ri, double* v1_ri, double* z2_ri) {
    int32_t M = 2 * Lp + 1;
    if (Lp < 1 || M > ORC_MAXL) return ORC_DEGENERATE;
    cplx G[ORC_MAXL * ORC_MAXL], u[ORC_MAXL], v[ORC_MAXL], zx = 0.0, zy = 0.0;
    for (int32_t i = 0; i < M * M; ++i) G[i] = G_ri[2 * i] + I * G_ri[2 * i + 1];
    int st = orc_square_window(G, Lp, ref_x, ref_y, &out3[0], &out3[1], &out3[2], u, v, &zx, &zy);
    for (int32_t i = 0; i < M; ++i) {
        u1_ri[2 * i] = creal(u[i]);
        u1_ri[2 * i + 1] = cimag(u[i]);
        v1_ri[2 * i] = creal(v[i]);
        v1_ri[2 * i + 1] = cimag(v[i]);
    }
    z2_ri[0] = creal(zx);
    z2_ri[1] = cimag(zx);
    z2_ri[2] = creal(zy);
    z2_ri[3] = cimag(zy);
    return st;
}

/* ---------------------------------------------------------------------------------
 * One pixel of the paper geometry on a frame's analytic signal gamma (H*W interleaved
 * complex, row-major). The block covers rows y-Lp..y+Lp and columns x-Lp..x+Lp; a pixel
 * whose block leaves the frame is a border pixel (Sec. 4). The carrier is removed after
 * the angles (a modulation exp(j 2 pi f0 X) along the carrier axis X adds 2 pi f0 to that
 * axis' angle and 2 pi f0 X to alpha, exactly): dx, dy are the local phase derivatives
 * and alpha the local phase with the carrier's phase 2 pi f0 X at the pixel subtracted,
 * all wrapped to (-pi, pi].
 * ------------------------------------------------------------------------------- */
static int orc_square_pixel(const double* gamma, int32_t H, int32_t W, const orc_params* p,
                            int32_t Lp, int32_t y, int32_t x, double* dx, double* dy,
                            double* alpha) {
    int32_t M = 2 * Lp + 1;
    *dx = NAN;
    *dy = NAN;
    *alpha = NAN;
    if (y - Lp < 0 || y + Lp > H - 1 || x - Lp < 0 || x + Lp > W - 1) return ORC_BORDER;
    if (p->model_order != 1 || Lp < 1 || M > ORC_MAXL) return ORC_DEGENERATE;
    cplx G[ORC_MAXL * ORC_MAXL];
    for (int32_t r = 0; r < M; ++r)
        for (int32_t c = 0; c < M; ++c) {
            size_t idx = (size_t)(y - Lp + r) * W + (size_t)(x - Lp + c);
            G[r * M + c] = gamma[2 * idx] + I * gamma[2 * idx + 1];
        }
    double w0 = 2.0 * ORC_PI * p->carrier_freq;
    double ref_x = p->carrier_axis == 0 ? w0 : 0.0;
    double ref_y = p->carrier_axis == 1 ? w0 : 0.0;
    double wx, wy, a;
    int st = orc_square_window(G, Lp, ref_x, ref_y, &wx, &wy, &a, NULL, NULL, NULL, NULL);
    if (st == ORC_DEGENERATE) return st;
    *dx = orc_wrap(wx - ref_x);
    *dy = orc_wrap(wy - ref_y);
    /* carrier phase at the pixel: 2 pi times the fractional part of f0 X */
    double t = p->carrier_freq * (double)(p->carrier_axis == 0 ? x : y);
    t -= floor(t);
    *alpha = orc_wrap(a - 2.0 * ORC_PI * t);
    return st;
}

/* Whole-frame paper geometry: maps dx, dy, alpha (H*W each, NaN where undefined) and
   status (may be NULL). Returns the OpenMP thread count used, or < 0 on error. */
int orc_square_demodulate(const void* frame, int32_t dtype, int32_t H, int32_t W,
                          const orc_params* p, int32_t Lp, double* dx, double* dy,
                          double* alpha, uint8_t* status, int32_t nthreads) {
    if (H <= 0 || W <= 0 || Lp < 1 || 2 * Lp + 1 > ORC_MAXL) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    double* gamma = (double*)malloc(sizeof(double) * 2 * (size_t)H * W);
    if (!gamma) return -2;
    int err = orc_gamma_of(frame, dtype, H, W, p, gamma);
    if (err) { free(gamma); return err; }
    int used = 1;
#pragma omp parallel for schedule(dynamic)
    for (int32_t y = 0; y < H; ++y) {
#ifdef _OPENMP
        if (y == 0) used = omp_get_num_threads();
#endif
        for (int32_t x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            int st = orc_square_pixel(gamma, H, W, p, Lp, y, x, &dx[i], &dy[i], &alpha[i]);
            if (status) status[i] = (uint8_t)st;
        }
    }
    free(gamma);
    return used;
}

/* Sampled paper geometry: only the pixels (ys[i], xs[i]); only the carrier lines their
   blocks cross are band-passed. Returns the thread count used, or < 0. */
int orc_square_demodulate_pixels(const void* frame, int32_t dtype, int32_t H, int32_t W,
                                 const orc_params* p, int32_t Lp, int32_t npix,
                                 const int32_t* ys, const int32_t* xs, double* dx, double* dy,
                                 double* alpha, uint8_t* status, int32_t nthreads) {
    if (H <= 0 || W <= 0 || Lp < 1 || 2 * Lp + 1 > ORC_MAXL) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int32_t ca = p->carrier_axis;
    int32_t nlines = ca == 0 ? H : W;
    double B = p->band_halfwidth > 0 ? p->band_halfwidth : 0.5 * p->carrier_freq;
    uint8_t* need = (uint8_t*)calloc((size_t)nlines, 1);
    double* gamma = (double*)calloc(2 * (size_t)H * W, sizeof(double));
    if (!need || !gamma) { free(need); free(gamma); return -2; }
    for (int32_t i = 0; i < npix; ++i) {
        int32_t y = ys[i], x = xs[i];
        if (y < 0 || y >= H || x < 0 || x >= W) { free(need); free(gamma); return -1; }
        for (int32_t k = -Lp; k <= Lp; ++k) {
            int32_t li = (ca == 0 ? y : x) + k;
            if (li >= 0 && li < nlines) need[li] = 1;
        }
    }
    int used = 1;
    if (p->band_cross > 0.0) {
        int err = orc_gamma_of(frame, dtype, H, W, p, gamma);
        if (err) { free(need); free(gamma); return err; }
    } else {
        used = orc_gamma_lines(frame, dtype, H, W, ca, p->carrier_freq, B, need, gamma);
    }
#pragma omp parallel for schedule(dynamic)
    for (int32_t i = 0; i < npix; ++i) {
        int st = orc_square_pixel(gamma, H, W, p, Lp, ys[i], xs[i], &dx[i], &dy[i], &alpha[i]);
        if (status) status[i] = (uint8_t)st;
    }
    free(need);
    free(gamma);
    return used;
}

/* =================================================================================
 * Phase assembly (Sec. 3: the local phases alpha are followed by an unwrapping operation,
 * the reliability-sorting method of Herraez et al., Appl. Opt. 41, 7437 (2002), which the
 * paper cites). On a wrapped map phi (H x W, row-major; NaN = no value):
 *   - the wrap operator g(x) maps a difference of two wrapped values into (-pi, pi];
 *   - reliability of a pixel whose 8 neighbours all hold values: R = 1 / D with
 *       D^2 = H^2 + V^2 + D1^2 + D2^2, the second differences
 *       H  = g(phi[i][j-1] - phi[i][j]) - g(phi[i][j] - phi[i][j+1]),
 *       V  = g(phi[i-1][j] - phi[i][j]) - g(phi[i][j] - phi[i+1][j]),
 *       D1 = g(phi[i-1][j-1] - phi[i][j]) - g(phi[i][j] - phi[i+1][j+1]),
 *       D2 = g(phi[i-1][j+1] - phi[i][j]) - g(phi[i][j] - phi[i+1][j-1]);
 *     every other pixel with a value has R = 0 (reading: no second difference, least reliable);
 *   - an edge joins horizontally or vertically adjacent pixels that both hold values; its
 *     reliability is the sum of theirs; edges are taken from the most reliable down (equal
 *     reliabilities by edge index 2 (i W + j) + (0 right, 1 down), smaller first);
 *   - each pixel starts as its own group; an edge joining two groups shifts every pixel of the
 *     smaller group (the second endpoint's on equal sizes) by the multiple of 2 pi that makes the
 *     two endpoints differ by the wrapped difference g(phi_q - phi_p); the groups merge.
 * The reliabilities and the 2 pi jumps are decided in float32, the precision of the GPU path
 * whose result this is compared with (the wrapped input is float32 on both sides).
 * ================================================================================= */
#define ORC_PI_F 3.14159265358979f
#define ORC_TWO_PI_F 6.28318530717959f

static float orc_gam_f(float x) {
    if (x > ORC_PI_F) return x - ORC_TWO_PI_F;
    if (x <= -ORC_PI_F) return x + ORC_TWO_PI_F;
    return x;
}

/* Reliability map R[H*W] of a wrapped map (R = 0 where a neighbour is missing; NaN where
   phi itself has no value). */
void orc_unwrap_reliability(const float* phi, int32_t H, int32_t W, float* R) {
    for (int32_t i = 0; i < H; ++i)
        for (int32_t j = 0; j < W; ++j) {
            float c = phi[(size_t)i * W + j];
            if (isnan(c)) { R[(size_t)i * W + j] = NAN; continue; }
            int inner = i >= 1 && i + 1 < H && j >= 1 && j + 1 < W;
            if (inner)
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj)
                        if (isnan(phi[(size_t)(i + di) * W + (j + dj)])) inner = 0;
            if (!inner) { R[(size_t)i * W + j] = 0.0f; continue; }
#define PH(a, b) phi[(size_t)(i + (a)) * W + (j + (b))]
            float h = orc_gam_f(PH(0, -1) - c) - orc_gam_f(c - PH(0, 1));
            float v = orc_gam_f(PH(-1, 0) - c) - orc_gam_f(c - PH(1, 0));
            float d1 = orc_gam_f(PH(-1, -1) - c) - orc_gam_f(c - PH(1, 1));
            float d2 = orc_gam_f(PH(-1, 1) - c) - orc_gam_f(c - PH(1, -1));
#undef PH
            float hh = h * h;
            float vv = v * v;
            float aa = d1 * d1;
            float bb = d2 * d2;
            float d = sqrtf(((hh + vv) + aa) + bb);
            R[(size_t)i * W + j] = 1.0f / d;
        }
}

typedef struct {
    float w;
    int64_t e;
} orc_edge;

static int orc_edge_cmp(const void* a, const void* b) {
    const orc_edge* x = (const orc_edge*)a;
    const orc_edge* y = (const orc_edge*)b;
    if (x->w > y->w) return -1;
    if (x->w < y->w) return 1;
    return x->e < y->e ? -1 : (x->e > y->e ? 1 : 0);
}

/* Unwrap phi (H x W float32, NaN = no value) into out (double, NaN where phi is NaN) and the
   integer map k (out = phi + 2 pi k; 0 where NaN). Returns the number of groups left (the
   connected components of the pixels with values), or < 0 on allocation failure. */
int orc_unwrap(const float* phi, int32_t H, int32_t W, double* out, int32_t* k) {
    size_t n = (size_t)H * W;
    float* R = (float*)malloc(sizeof(float) * n);
    orc_edge* E = (orc_edge*)malloc(sizeof(orc_edge) * 2 * n + 1);
    int32_t* group = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * n);  /* member list of each group */
    int32_t* last = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* size = (int32_t*)malloc(sizeof(int32_t) * n);
    if (!R || !E || !group || !next || !last || !size) {
        free(R); free(E); free(group); free(next); free(last); free(size);
        return -2;
    }
    orc_unwrap_reliability(phi, H, W, R);
    size_t ne = 0;
    int ngroups = 0;
    for (int32_t i = 0; i < H; ++i)
        for (int32_t j = 0; j < W; ++j) {
            size_t p = (size_t)i * W + j;
            k[p] = 0;
            group[p] = (int32_t)p;
            next[p] = -1;
            last[p] = (int32_t)p;
            size[p] = 1;
            if (isnan(phi[p])) continue;
            ++ngroups;
            if (j + 1 < W && !isnan(phi[p + 1])) {
                E[ne].w = R[p] + R[p + 1];
                E[ne].e = 2 * (int64_t)p;
                ++ne;
            }
            if (i + 1 < H && !isnan(phi[p + W])) {
                E[ne].w = R[p] + R[p + W];
                E[ne].e = 2 * (int64_t)p + 1;
                ++ne;
            }
        }
    qsort(E, ne, sizeof(orc_edge), orc_edge_cmp);
    for (size_t t = 0; t < ne; ++t) {
        size_t p = (size_t)(E[t].e / 2);
        size_t q = (E[t].e % 2) ? p + W : p + 1;
        int32_t gp = group[p], gq = group[q];
        if (gp == gq) continue;
        /* k_q - k_p must equal the jump s of the wrapped difference phi_q - phi_p */
        float dq = phi[q] - phi[p];
        int32_t s = dq > ORC_PI_F ? -1 : (dq <= -ORC_PI_F ? 1 : 0);
        int32_t shift, from, into;
        if (size[gq] <= size[gp]) {
            shift = k[p] + s - k[q];  /* added to every pixel of q's group */
            from = gq;
            into = gp;
        } else {
            shift = k[q] - s - k[p];  /* added to every pixel of p's group */
            from = gp;
            into = gq;
        }
        for (int32_t m = from; m >= 0; m = next[m]) {
            k[m] += shift;
            group[m] = into;
        }
        next[last[into]] = from;
        last[into] = last[from];
        size[into] += size[from];
        --ngroups;
    }
    for (size_t p = 0; p < n; ++p)
        out[p] = isnan(phi[p]) ? NAN : (double)phi[p] + 2.0 * ORC_PI * (double)k[p];
    free(R); free(E); free(group); free(next); free(last); free(size);
    return ngroups;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
