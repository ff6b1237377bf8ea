"""Planted mistakes: each test copies the oracle's C source, plants one plausible error (a dropped
conjugate, a transposed operand, a wrong index or sign), compiles the copy on the CPU and checks
that the pins in test_oracle_pins.py, test_oracle_square.py, test_oracle_unwrap.py and
test_oracle_band2d.py, test_oracle_model_order.py reject it. This shows the pins constrain every step of the
oracle rather than only re-running it."""
import numpy as np
import pytest

import oracle as O
import test_oracle_pins as P
import test_oracle_square as S
import test_oracle_band2d as B2
import test_oracle_model_order as MO
import test_oracle_unwrap as U

MUTATIONS = {
    "band: negative side kept": ("fabs((double)k / (double)W - f0) < B", "fabs((double)k / (double)W + f0) < B"),
    "band: inverse kernel not conjugated": ("acc += X[k] * conj(tw[((int64_t)k * n) % W]);",
                                            "acc += X[k] * tw[((int64_t)k * n) % W];"),
    "band: 1/W dropped": ("acc /= (double)W;", "acc /= 1.0;"),
    "cov: conjugate dropped": ("acc += w[i + m] * conj(w[i + l]);", "acc += w[i + m] * w[i + l];"),
    "cov: operands transposed": ("acc += w[i + m] * conj(w[i + l]);", "acc += conj(w[i + m]) * w[i + l];"),
    "cov: last snapshot dropped": ("for (int32_t i = 0; i < K; ++i) acc +=", "for (int32_t i = 0; i < K - 1; ++i) acc +="),
    "cov: FB index not reversed": ("conj(Rf[(L - 1 - m) * L + (L - 1 - l)])", "conj(Rf[m * L + l])"),
    "eig: rotation phase not conjugated": ("A[r * L + p] = c * arp - s * conj(e) * arq;", "A[r * L + p] = c * arp - s * e * arq;"),
    "eig: eigenvector update sign": ("V[r * L + q] = s * e * vrp + c * vrq;", "V[r * L + q] = -s * e * vrp + c * vrq;"),
    "eig: diagonal update sign": ("double app = creal(A[p * L + p]) - t * ab;", "double app = creal(A[p * L + p]) + t * ab;"),
    "poly: lag index transposed": ("q[(l - m) + (L - 1)] += Cml;", "q[(m - l) + (L - 1)] += Cml;"),
    "poly: projector sign": ("cplx Cml = (m == l ? 1.0 : 0.0) - u[m] * conj(u[l]);", "cplx Cml = (m == l ? 1.0 : 0.0) + u[m] * conj(u[l]);"),
    "roots: Aberth sum sign": ("z[i] -= Ni / (1.0 - Ni * Si);", "z[i] -= Ni / (1.0 + Ni * Si);"),
    "roots: closing sweeps dropped": ("for (int sweep = 0; sweep < 2; ++sweep)", "for (int sweep = 0; sweep < 0; ++sweep)"),
    "select: outside roots": ("if (!(r <= 1.0 + 1e-9)) continue;", "if (!(r >= 1.0 - 1e-9)) continue;"),
    "select: farthest root": ("if (d < bestd || (d == bestd && t < bestt))", "if (-d < bestd || (d == bestd && t < bestt))"),
    "angle: carrier added": ("*deriv = orc_wrap(carg(z) - omega_ref);", "*deriv = orc_wrap(carg(z) + omega_ref);"),
    "window: off by one": ("int32_t start = n - N / 2;", "int32_t start = n - N / 2 + 1;"),
    "eig: smallest eigenvector": ("if (ev[j] > ev[j1]) j1 = j;", "if (ev[j] < ev[j1]) j1 = j;"),
    # the square block of the paper's geometry
    "square: R_y operands transposed": ("acc += G[m * M + c] * conj(G[l * M + c]);",
                                        "acc += conj(G[m * M + c]) * G[l * M + c];"),
    "square: R_x rows not conjugated": ("acc += conj(G[r * M + a]) * G[r * M + b];",
                                        "acc += G[r * M + a] * conj(G[r * M + b]);"),
    "square: x angle sign": ("double ox = -carg(zx);", "double ox = carg(zx);"),
    "square: u1 used for both axes": ("orc_music_poly(v, M, qx);", "orc_music_poly(u, M, qx);"),
    "square: alpha coordinates not centred": ("acc += G[r * M + c] * cexp(-I * (ox * (double)(c - Lp) + oy * (double)(r - Lp)));",
                                              "acc += G[r * M + c] * cexp(-I * (ox * (double)c + oy * (double)r));"),
    "square: alpha demodulation sign": ("acc += G[r * M + c] * cexp(-I * (ox", "acc += G[r * M + c] * cexp(I * (ox"),
    "square: carrier left in alpha": ("*alpha = orc_wrap(a - 2.0 * ORC_PI * t);", "*alpha = orc_wrap(a);"),
    "square: block read transposed": ("size_t idx = (size_t)(y - Lp + r) * W + (size_t)(x - Lp + c);",
                                      "size_t idx = (size_t)(y - Lp + c) * W + (size_t)(x - Lp + r);"),
    "square: carrier taken from the wrong axis": ("double t = p->carrier_freq * (double)(p->carrier_axis == 0 ? x : y);",
                                                  "double t = p->carrier_freq * (double)(p->carrier_axis == 0 ? y : x);"),
    # phase assembly (the reliability-sorting unwrapper)
    "unwrap: least reliable edge first": ("    if (x->w > y->w) return -1;\n    if (x->w < y->w) return 1;",
                                          "    if (x->w > y->w) return 1;\n    if (x->w < y->w) return -1;"),
    "unwrap: jump sign": ("int32_t s = dq > ORC_PI_F ? -1 : (dq <= -ORC_PI_F ? 1 : 0);",
                          "int32_t s = dq > ORC_PI_F ? 1 : (dq <= -ORC_PI_F ? -1 : 0);"),
    "unwrap: reliability not inverted": ("R[(size_t)i * W + j] = 1.0f / d;", "R[(size_t)i * W + j] = d;"),
    "unwrap: second difference sign": ("float h = orc_gam_f(PH(0, -1) - c) - orc_gam_f(c - PH(0, 1));",
                                       "float h = orc_gam_f(PH(0, -1) - c) + orc_gam_f(c - PH(0, 1));"),
    "unwrap: group shift sign": ("shift = k[p] + s - k[q];", "shift = k[q] + s - k[p];"),
    # the 2-D band-pass variant
    "band2d: one-sided cross band": ("int32_t ks = 2 * (int64_t)k < len ? k : k - len; /* signed bin */",
                                     "int32_t ks = k; /* signed bin */"),
    "band2d: 1/len dropped": ("            acc /= (double)len;\n            size_t idx = carrier_axis == 0 ? (size_t)n * W + li",
                              "            acc /= 1.0;\n            size_t idx = carrier_axis == 0 ? (size_t)n * W + li"),
    "band2d: along the carrier": ("    int32_t nlines = carrier_axis == 0 ? W : H;  /* lines across the carrier */",
                                  "    int32_t nlines = carrier_axis == 0 ? H : W;  /* lines across the carrier */"),
    # model order p > 1
    "p: projector keeps one eigenvector": ("    for (int32_t i = 0; i < p; ++i) {\n        int32_t j = order[i];",
                                           "    for (int32_t i = 0; i < 1; ++i) {\n        int32_t j = order[i];"),
    "p: expected angle ignored": ("if (a < bestt) { bestt = a; best = near_idx[t]; }",
                                  "if (best < 0) { bestt = a; best = near_idx[t]; }"),
    "p: split double root counted twice": ("if (i == near_idx[u] || cabs(roots[i] - roots[near_idx[u]]) < 1e-6) taken = 1;",
                                           "if (i == near_idx[u]) taken = 1;"),
    "raw: line mean kept": ("        mean /= (double)len;\n        for (int32_t n = 0; n < len; ++n) {",
                            "        mean = 0.0;\n        for (int32_t n = 0; n < len; ++n) {"),
}

PINS = [
    lambda: P.test_analytic_line_matches_fft_bandpass(128),
    P.test_analytic_line_closed_form_periodic_cosine,
    lambda: P.test_covariance_rank_one_for_exponential(32, 8, 0),
    lambda: P.test_covariance_rank_one_for_exponential(32, 8, 1),
    P.test_covariance_structure_noise,
    lambda: P.test_eig_matches_lapack(8),
    P.test_eig_eigenvalues_signal_plus_noise,
    lambda: P.test_music_poly_on_circle_equals_noise_projection(8),
    P.test_music_poly_closed_form_steering_vector,
    lambda: P.test_roots_match_companion_matrix(3),
    lambda: P.test_roots_near_pair_at_rounding_level(8),
    P.test_selection_hand_cases,
    lambda: P.test_p1_noise_free_linear_phase_exact(32, 8, 1),
    lambda: P.test_p2_order_two_is_pulse_pair(1),
    P.test_p4_carrier_rotation,
    P.test_p7_noisy_selection_by_enumeration,
    lambda: S.test_square_plane_wave_exact(3),
    lambda: S.test_square_real_fringe_with_carrier_exact(0),
    lambda: S.test_square_real_fringe_with_carrier_exact(1),
    lambda: S.test_square_eigenvectors_are_singular_vectors(3),
    lambda: S.test_square_angles_by_enumeration(2),
    S.test_square_alpha_is_least_squares_phase,
    lambda: U.test_unwrap_smooth_maps_exact(0),
    U.test_unwrap_single_row_is_numpy_unwrap,
    U.test_reliability_closed_form_quadratic,
    lambda: U.test_unwrap_is_max_spanning_tree_integration(0),
    lambda: B2.test_band2d_matches_fft2_rectangle(0),
    B2.test_band2d_plane_waves_inside_and_outside,
    lambda: MO.test_p2_noise_free_real_cosine_exact(8, 1),
    MO.test_p3_models_a_local_offset,
    lambda: MO.test_p_noisy_windows_by_enumeration(2),
]


def _failing_pins(first_only=False):
    failed = []
    for i, pin in enumerate(PINS):
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:  # an AssertionError, or a crash of the mutated code path
            failed.append(i)
            if first_only:
                break
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = O.source()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    path = O.compile_variant(src.replace(old, new), str(tmp_path / "liboracle_mut.so"))
    with O.use_library(path):
        failed = _failing_pins(first_only=True)
    assert failed, f"no pin rejects the planted mistake '{name}'"


def test_unmutated_copy_passes(tmp_path):
    path = O.compile_variant(O.source(), str(tmp_path / "liboracle_copy.so"))
    with O.use_library(path):
        assert _failing_pins() == []
