"""The oracle's pins catch plausible slips.

Each case plants one mistake in one oracle module -- a dropped term or
factor, a wrong sign, index, constant or comparison, a transposed or swapped
operand -- by editing one site of the module's source, executes the edited
source as a fresh module and puts it in place of the original wherever the
oracle package, the other oracle modules and the pin test modules refer to
it.  The pins named for the case then run against the mutant, and at least
one of them must fail (an assertion, or an error the pin would report).
The originals are restored after every case; the same pins pass on them in
their own test files.

A change that leaves the defined result unchanged is not a slip and is not
listed: for example the side on which the mean-shift step is applied moves
the iterates but not the fixed point (the weighted mean of the tangent
coordinates is zero), and a different tie rule between equal energies picks
an equal value.  Nor are choices the paper leaves open and that no closed
form decides (the order of the chain directions over the iterations): the
oracle fixes them and the GPU parity replays them.

The mistakes are planted in the oracle only, on the CPU; nothing here runs
the CUDA path.
"""
import inspect
import sys
import types

import numpy as np
import pytest

import oracle  # noqa: F401  (the package whose modules are replaced)
import test_cnn_oracle  # noqa: F401
import test_ka_oracle  # noqa: F401
import test_oracle_pins  # noqa: F401
import test_posecov_oracle  # noqa: F401
import test_vc_oracle  # noqa: F401

PINS = "test_oracle_pins"
PC = "test_posecov_oracle"
KA = "test_ka_oracle"
VC = "test_vc_oracle"
CNN = "test_cnn_oracle"

# (id, oracle module, source site, replacement, [(pin module, pin, args)])
MUTANTS = [
    # ---- Fisk residual model
    ("fisk-density-square-dropped", "fisk",
     "s ** (beta - 2.0) / (1.0 + s ** beta) ** 2", "s ** (beta - 2.0) / (1.0 + s ** beta)",
     [(PINS, "test_residual_density_is_a_planar_density", (0.5, 2.0)),
      (PINS, "test_inlier_energy_beta2_closed_form", ())]),
    ("fisk-density-2pi-to-pi", "fisk",
     "beta / (2.0 * math.pi * alpha * alpha)", "beta / (math.pi * alpha * alpha)",
     [(PINS, "test_residual_density_is_a_planar_density", (0.5, 2.0))]),
    ("fisk-energy-ratio-inverted", "fisk",
     "np.log1p(p0 / residual_density(r, alpha, beta))",
     "np.log1p(residual_density(r, alpha, beta) / p0)",
     [(PINS, "test_inlier_energy_beta2_closed_form", ())]),
    ("fisk-cdf-exponent-sign", "fisk", "** (-beta))", "** (beta))",
     [(PINS, "test_fisk_pdf_normalises_and_cdf_closed_form", (0.5, 2.0))]),
    ("fisk-pdf-exponent", "fisk", "z ** (beta - 1)", "z ** beta",
     [(PINS, "test_fisk_pdf_normalises_and_cdf_closed_form", (0.7, 1.5))]),
    ("fisk-posterior-numerator", "fisk", "return p1 / (p1 + p0)", "return p0 / (p1 + p0)",
     [(PINS, "test_inlier_energy_beta2_closed_form", ())]),
    # ---- forward-backward and confidence
    ("hmm-forward-wrong-emission", "hmm",
     "x0 = (a0[m - 1] * g + a1[m - 1] * h) * e0[m]", "x0 = (a0[m - 1] * g + a1[m - 1] * h) * e1[m]",
     [(PINS, "test_forward_backward_matches_enumeration", (5,))]),
    ("hmm-backward-transition-swapped", "hmm", "x0 = g * y0 + h * y1", "x0 = h * y0 + g * y1",
     [(PINS, "test_forward_backward_matches_enumeration", (5,))]),
    ("hmm-backward-emission-index", "hmm",
     "y1 = e1[m + 1] * b1[m + 1]", "y1 = e1[m] * b1[m + 1]",
     [(PINS, "test_forward_backward_matches_enumeration", (5,))]),
    ("hmm-posterior-mixed-states", "hmm", "p1 = a1 * b1", "p1 = a1 * b0",
     [(PINS, "test_forward_backward_matches_enumeration", (5,))]),
    ("hmm-initial-distribution", "hmm", "x0, x1 = 0.5 * e0[0], 0.5 * e1[0]",
     "x0, x1 = 0.5 * e0[0], 0.25 * e1[0]",
     [(PINS, "test_forward_backward_matches_enumeration", (5,))]),
    ("hmm-transition-swapped", "hmm", "g, h = gamma, 1.0 - gamma", "g, h = 1.0 - gamma, gamma",
     [(PINS, "test_forward_backward_matches_enumeration", (5,))]),
    ("hmm-confidence-denominator", "hmm",
     "C = q.astype(np.float64).sum(0) / P.N", "C = q.astype(np.float64).sum(0) / (P.N + 1)",
     [(PINS, "test_estep_moving_blobs_get_low_rigidness", ())]),
    # ---- geometry
    ("geometry-so3-sine-sign", "geometry", "np.eye(3) + math.sin(th) / th * Kx",
     "np.eye(3) - math.sin(th) / th * Kx",
     [(PINS, "test_se3_exp_log_roundtrip_and_compose", ())]),
    ("geometry-V-power", "geometry", "(np.eye(3) + (1 - math.cos(th)) / th ** 2 * Kx",
     "(np.eye(3) + (1 - math.cos(th)) / th * Kx",
     [(PINS, "test_se3_exp_equals_the_matrix_exponential", ())]),
    ("geometry-bilinear-weights", "geometry", "((1 - ax) * f00 + ax * f01)",
     "((1 - ay) * f00 + ay * f01)",
     [(PINS, "test_bilinear_reproduces_affine_fields_and_grid_values", ())]),
    ("geometry-bilinear-tap", "geometry", "f01 = F[y0, x0 + 1]", "f01 = F[y0 + 1, x0]",
     [(PINS, "test_bilinear_reproduces_affine_fields_and_grid_values", ())]),
    ("geometry-inside-last-column", "geometry", "(x <= W - 1)", "(x < W - 1)",
     [(PINS, "test_bilinear_reproduces_affine_fields_and_grid_values", ())]),
    ("geometry-projection-cx", "geometry", "fx * X[..., 0] + cx * X[..., 2]",
     "fx * X[..., 0] + cx * X[..., 0]",
     [(PINS, "test_energy_minimum_at_true_depth_noise_free", ())]),
    ("geometry-compose-order", "geometry", "(A[:, :3] @ B[:, 3] + A[:, 3])",
     "(B[:, :3] @ A[:, 3] + B[:, 3])",
     [(PINS, "test_meanshift_cases", ()),
      (PINS, "test_pose_step_recovers_first_pose_from_true_depth", ())]),
    # ---- Philox
    ("philox-multiplier", "philox", "M0 = np.uint64(0xD2511F53)", "M0 = np.uint64(0xD2511F55)",
     [(PINS, "test_philox_known_answers", ())]),
    ("philox-weyl-constant", "philox", "W1 = 0xBB67AE85", "W1 = 0xBB67AE86",
     [(PINS, "test_philox_known_answers", ())]),
    ("philox-halves-swapped", "philox",
     "(hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)",
     "(hi0 ^ c1 ^ np.uint64(k0), lo1, hi1 ^ c3 ^ np.uint64(k1), lo0)",
     [(PINS, "test_philox_known_answers", ())]),
    ("philox-u24-low-bits", "philox", "(x >> np.uint32(8))", "(x & np.uint32(0xFFFFFF))",
     [(PINS, "test_philox_u24_and_pick_are_exact", ())]),
    ("philox-pick-modulo", "philox",
     "(np.asarray(x, np.uint64) * np.uint64(n)) >> np.uint64(32)",
     "np.asarray(x, np.uint64) % np.uint64(n)",
     [(PINS, "test_philox_u24_and_pick_are_exact", ())]),
    # ---- per-pixel energy and priors
    ("model-flow-residual-sign", "model", "dx = F[..., 0] - (x - xp)", "dx = F[..., 0] + (x - xp)",
     [(PINS, "test_energy_minimum_at_true_depth_noise_free", ())]),
    ("model-prior-term-dropped", "model", "E = E + prior_weight(P, S, iu, iv) * lh", "E = E",
     [(PINS, "test_stereo_prior_optimum_is_the_prior", ())]),
    ("model-stereo-scale", "model", "rr = np.abs(d - float(P.fxb32) * rho)",
     "rr = np.abs(d - float(P.K[0]) * rho)",
     [(PINS, "test_stereo_prior_optimum_is_the_prior", ())]),
    ("model-rgbd-sigma-unscaled", "model", "sig = p.prior_c_sigma * rhat", "sig = p.prior_c_sigma",
     [(PINS, "test_rgbd_prior_closed_forms", ())]),
    ("model-rgbd-normaliser", "model",
     "logk = math.log(math.sqrt(2 * math.pi) * p.prior_c_sigma / p.prior_w_uniform)",
     "logk = math.log(2 * math.pi * p.prior_c_sigma / p.prior_w_uniform)",
     [(PINS, "test_rgbd_prior_closed_forms", ())]),
    ("model-rgbd-uniform-density", "model", "e0 = 1.0 / (p.prior_w_uniform * rhat)",
     "e0 = 1.0 / p.prior_w_uniform",
     [(PINS, "test_rgbd_prior_closed_forms", ())]),
    ("model-behind-camera-free", "model", "np.where(obs, fisk.L_BEHIND, 0.0)", "np.where(obs, 0.0, 0.0)",
     [(PINS, "test_behind_camera_and_unobserved_terms", ())]),
    ("model-unobserved-emission", "model", "np.where(obs, 0.0, p.outlier_density)",
     "np.where(obs, 0.0, 0.0)",
     [(PINS, "test_behind_camera_and_unobserved_terms", ())]),
    ("hmm-prior-rigidness-inverted", "hmm", "qh = np.where(valid, e1h / (e1h + e0h), 0.0)",
     "qh = np.where(valid, e0h / (e1h + e0h), 0.0)",
     [(PINS, "test_prior_rigidness_at_a_perfect_prior", ())]),
    ("em-initial-range", "em", "rho = rmin + np.float32(u * np.float32(rmax - rmin))",
     "rho = rmin + np.float32(u * rmax)",
     [(PINS, "test_initial_inverse_depth_is_uniform_in_range_or_the_prior", ())]),
    # ---- depth M-step
    ("depth-perturbation-scale", "depth", "0.5 * 2.0 ** (-it)", "0.5 * 2.0 ** (it)",
     [(PINS, "test_hypotheses_distribution_and_sharing", ())]),
    ("depth-perturbation-one-sided", "depth",
     "a = np.float32(np.float32(2.0) * u) - np.float32(1.0)", "a = u",
     [(PINS, "test_hypotheses_distribution_and_sharing", ())]),
    ("depth-uniform-range", "depth", "c = rmin + np.float32(u * rng)", "c = rmin + np.float32(u * rmax)",
     [(PINS, "test_hypotheses_distribution_and_sharing", ())]),
    ("depth-share-counter", "depth", "c0 = j - (iu % p.sample_share).astype(np.uint64)", "c0 = j",
     [(PINS, "test_hypotheses_distribution_and_sharing", ())]),
    ("depth-propagated-value-not-written", "depth", "        new[v, u] = cur\n",
     "        new[v, u] = rho_star[v, u]\n",
     [(PINS, "test_split_propagation_equals_naive_sequential", (0,))]),
    ("depth-hierarchical-coarse-test", "depth", "take = E_up < E_star", "take = E_up > E_star",
     [(PINS, "test_propagation_never_raises_a_pixels_energy", (0,))]),
    ("depth-argmin-keeps-first-slot", "depth", "best = np.where(take, cands[k], best)",
     "best = np.where(take & (k == 0), cands[k], best)",
     [(PINS, "test_argmin_finds_true_depth_among_candidates", ()),
      (PINS, "test_split_propagation_equals_naive_sequential", (0,))]),
    # ---- pose M-step
    ("pose-meanshift-weight-sign", "pose", "w = np.exp(-0.5 * np.sum(d * d * inv_var, axis=1))",
     "w = np.exp(0.5 * np.sum(d * d * inv_var, axis=1))",
     [(PINS, "test_meanshift_cases", ())]),
    ("pose-meanshift-stops-at-100-steps", "pose", "MS_MAX_ITERS = 100000", "MS_MAX_ITERS = 100",
     [(PINS, "test_meanshift_runs_to_the_mode_where_it_converges_slowly", ())]),
    ("pose-triplet-duplicates", "pose", "if len(set(idx)) == 3:", "if True:",
     [(PINS, "test_sample_triplets_are_distinct_indices", ())]),
    ("pose-kernel-widths-swapped", "pose",
     "inv_var = np.array([1 / p.pose_sigma_rot ** 2] * 3 + [1 / st ** 2] * 3)",
     "inv_var = np.array([1 / st ** 2] * 3 + [1 / p.pose_sigma_rot ** 2] * 3)",
     [(PINS, "test_meanshift_mode_on_one_rotation_axis_solves_the_scalar_equation", ())]),
    ("pose-rigid-threshold", "pose", "(S.q[t - 1] > np.float32(0.5))", "(S.q[t - 1] >= np.float32(0.0))",
     [(PINS, "test_pose_step_skips_degenerate_frame", ())]),
    ("pose-bearing-principal-point", "pose", "(xo[:, 0] - cx) / fx", "(xo[:, 0] - cy) / fx",
     [(PINS, "test_pose_step_recovers_first_pose_from_true_depth", ())]),
    ("pose-observation-flow-sign", "pose", "xp[vv, uu] + F[vv, uu, 0]", "xp[vv, uu] - F[vv, uu, 0]",
     [(PINS, "test_pose_step_recovers_first_pose_from_true_depth", ())]),
    # ---- P3P
    ("p3p-conic-sign", "p3p", "[c2 - b2, -2 * c2 * cb, c2]", "[c2 - b2, 2 * c2 * cb, c2]",
     [(PINS, "test_p3p_exact_correspondences", ())]),
    ("p3p-kabsch-reflection", "p3p",
     "D = np.diag([1.0, 1.0, np.sign(np.linalg.det(Vt.T @ U.T))])", "D = np.eye(3)",
     [(PINS, "test_p3p_exact_correspondences", ())]),
    ("p3p-resultant-sign", "p3p", "return s(m(A, A), m(B, C))", "return Pl.polyadd(m(A, A), m(B, C))",
     [(PINS, "test_p3p_exact_correspondences", ())]),
    # ---- 8-point bootstrap
    ("eightpoint-constraint-transposed", "eightpoint",
     "rows = (b[:, :, None] * a[:, None, :]).reshape(-1, 9)\n    f = np.sqrt",
     "rows = (a[:, :, None] * b[:, None, :]).reshape(-1, 9)\n    f = np.sqrt",
     [(PINS, "test_eight_point_noise_free_two_planes_is_exact", ())]),
    ("eightpoint-second-rotation", "eightpoint", "R2 = U @ WMAT.T @ Vt", "R2 = U @ WMAT @ Vt",
     [(PINS, "test_eight_point_noise_free_two_planes_is_exact", ())]),
    ("eightpoint-translation-column", "eightpoint", "t = U[:, 2]", "t = Vt[2]",
     [(PINS, "test_eight_point_noise_free_two_planes_is_exact", ())]),
    ("eightpoint-one-depth-test", "eightpoint", "return int(np.sum((la > 0) & (lb > 0)))",
     "return int(np.sum(la > 0))",
     [(PINS, "test_essential_decomposition_and_cheirality", ())]),
    ("eightpoint-improper-rotation", "eightpoint", "    if np.linalg.det(U) < 0:\n        U = -U\n",
     "",
     [(PINS, "test_essential_decomposition_and_cheirality", ())]),
    ("eightpoint-cheirality-sign", "eightpoint", "m12 = -np.sum(Ra * b, 1)", "m12 = np.sum(Ra * b, 1)",
     [(PINS, "test_eight_point_noise_free_two_planes_is_exact", ())]),
    # ---- pose covariance
    ("posecov-gate", "posecov", "inl = m <= 9.0", "inl = m <= 3.0",
     [(PC, "test_symmetric_star_closed_form", ()),
      (PC, "test_one_3_sigma_round_gives_the_truncated_chi2_moment", ())]),
    ("posecov-mad-constant", "posecov", "s = 1.4826 * np.median", "s = np.median",
     [(PC, "test_robust_start_is_the_gaussian_scale_and_ignores_outliers", ())]),
    ("posecov-unbiased-normalisation", "posecov", "dn.T @ dn / n_in", "dn.T @ dn / (n_in - 1)",
     [(PC, "test_symmetric_star_closed_form", ())]),
    ("posecov-start-mean", "posecov", "s = 1.4826 * np.median(np.abs(d), axis=0)",
     "s = 1.4826 * np.mean(np.abs(d), axis=0)",
     [(PC, "test_robust_start_is_the_gaussian_scale_and_ignores_outliers", ())]),
    ("posecov-six-samples", "posecov", "MIN_INLIERS = 7", "MIN_INLIERS = 6",
     [(PC, "test_six_samples_cannot_give_a_covariance", ())]),
    ("posecov-no-convergence-test", "posecov",
     "if prev is not None and np.array_equal(inl, prev):", "if False:",
     [(PC, "test_symmetric_star_closed_form", ())]),
    ("posecov-floor-min", "posecov", "np.maximum(w, eps)", "np.minimum(w, eps)",
     [(PC, "test_eigenvalue_floor_and_symmetry", ())]),
    ("posecov-coordinates-side", "posecov", "geometry.compose(mi, T)", "geometry.compose(T, mi)",
     [(PC, "test_symmetric_star_closed_form", ())]),
    # ---- VC score
    ("vc-cell-floor", "vc", "np.floor(x[vis] + np.float32(0.5))", "np.floor(x[vis])",
     [(VC, "test_sideways_translation_over_a_plane", (8,)),
      (VC, "test_two_projections_in_one_nearest_pixel_cell", ())]),
    ("vc-arithmetic-mean", "vc", "2.0 * v * c / (v + c)", "0.5 * (v + c)",
     [(VC, "test_harmonic_mean_stride_and_keyframe", ())]),
    ("vc-stride-boundary", "vc", "if s < tau_stride:", "if s <= tau_stride:",
     [(VC, "test_harmonic_mean_stride_and_keyframe", ())]),
    ("vc-coverage-over-depth-pixels", "vc", "c = n_cov / (W * H)", "c = n_cov / n_depth if n_depth else 0.0",
     [(VC, "test_coverage_is_a_fraction_of_the_image_not_of_the_depth_pixels", ())]),
    ("vc-invalid-depth-counted", "vc", "vis = valid & inside", "vis = inside",
     [(VC, "test_invalid_depths_are_not_depth_pixels", ())]),
    ("vc-inside-one-past", "vc", "(x <= f32(W - 1))", "(x <= f32(W))",
     [(VC, "test_direction_of_translation_and_rotation", ())]),
    # ---- keyframe alignment
    ("ka-residual-sign", "ka", "r = A / Z - B / (D * Z)", "r = B / (D * Z) - A / Z",
     [(KA, "test_jacobian_matches_finite_differences", ())]),
    ("ka-scale-jacobian-sign", "ka", "J[:, 6] = B / (D * Z)", "J[:, 6] = -B / (D * Z)",
     [(KA, "test_jacobian_matches_finite_differences", ())]),
    ("ka-normals-away-from-camera", "ka", "flip = np.sum(c * P[1:-1, 1:-1], axis=-1) > 0",
     "flip = np.sum(c * P[1:-1, 1:-1], axis=-1) < 0",
     [(KA, "test_normals_of_a_plane_face_the_camera", ())]),
    ("ka-step-acceptance", "ka", "if nn > 0 and En < E:", "if nn > 0 and En > E:",
     [(KA, "test_alignment_recovers_the_pose", ())]),
    ("ka-scale-dropped", "ka", "D = s * t1", "D = t1",
     [(KA, "test_alignment_recovers_the_scale", ())]),
    ("ka-kink-test-dropped", "ka", "ok_d[1:-1, 1:-1] & (nrm > 0) & smooth)",
     "ok_d[1:-1, 1:-1] & (nrm > 0))",
     [(KA, "test_alignment_recovers_the_pose", ()),
      (KA, "test_zero_residual_at_the_true_pose_on_plane_interiors", ())]),
    ("ka-occlusion-gate-dropped", "ka", "assoc = inside & ok1[li, lj] & valid_depth(th1) & agree",
     "assoc = inside & ok1[li, lj] & valid_depth(th1)",
     [(KA, "test_hidden_points_are_not_paired_with_the_occluder", ())]),
    ("ka-cauchy-weight", "ka", "w = C / (1.0 + (r / c) ** 2)", "w = C / (1.0 + np.abs(r / c))",
     [(KA, "test_robust_kernel_downweights_corrupted_depth", ()),
      (KA, "test_alignment_recovers_the_pose", ())]),
    # ---- learned initialiser
    ("cnn-kernel-flipped", "cnn",
     'z += np.einsum("oc,chw->ohw", W[:, ky, kx, :]', 'z += np.einsum("oc,chw->ohw", W[:, 2 - ky, 2 - kx, :]',
     [(CNN, "test_conv_equals_channel_sum_of_library_correlation", ())]),
    ("cnn-input-gradient-shift", "cnn", "dzp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + Wd]",
     "dzp[:, ky:ky + H, kx:kx + Wd]",
     [(CNN, "test_input_gradient_of_conv_matches_finite_differences", ())]),
    ("cnn-adam-bias-correction", "cnn", "mh = m / (1 - ADAM_B1 ** t)", "mh = m",
     [(CNN, "test_adam_first_step_closed_form", ())]),
    ("cnn-bf16-truncation", "cnn", "(u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u & 0xFFFF0000",
     [(CNN, "test_bf16_rounding_matches_torch_and_known_values", ())]),
    ("cnn-depth-head-sign", "cnn", "rho = np.clip(rho_c * np.exp(z[0]), rho_min, rho_max)",
     "rho = np.clip(rho_c * np.exp(-z[0]), rho_min, rho_max)",
     [(CNN, "test_heads_and_loss_closed_forms", ())]),
    ("cnn-loss-centre-sign", "cnn", "e = z[0] + 0.5 * np.log(rho_min * rho_max) - np.log(rho_t)",
     "e = z[0] - 0.5 * np.log(rho_min * rho_max) - np.log(rho_t)",
     [(CNN, "test_heads_and_loss_closed_forms", ())]),
    ("cnn-bias-dropped", "cnn",
     "z = np.broadcast_to(np.asarray(b, np.float64)[:, None, None], (W.shape[0], H, Wd)).copy()",
     "z = np.zeros((W.shape[0], H, Wd))",
     [(CNN, "test_conv_equals_channel_sum_of_library_correlation", ())]),
    ("cnn-adam-second-moment", "cnn", "v = ADAM_B2 * v + (1 - ADAM_B2) * g * g",
     "v = ADAM_B2 * v + (1 - ADAM_B2) * np.abs(g)",
     [(CNN, "test_adam_first_step_closed_form", ())]),
    ("cnn-bce-gradient-sign", "cnn", "dz[1:] = w_q * m * (q - q_t) / (nq * nm)",
     "dz[1:] = w_q * m * (q_t - q) / (nq * nm)",
     [(CNN, "test_backward_matches_finite_differences", ())]),
]


def _mutant(mod, site, repl):
    src = inspect.getsource(mod)
    assert src.count(site) == 1, f"{mod.__name__}: the site must occur exactly once: {site!r}"
    m = types.ModuleType(mod.__name__)
    m.__file__ = mod.__file__
    m.__package__ = mod.__package__
    exec(compile(src.replace(site, repl), mod.__file__, "exec"), m.__dict__)
    return m


def _install(monkeypatch, orig, mut):
    """Replace every reference to the module orig by mut (restored by monkeypatch)."""
    monkeypatch.setitem(sys.modules, orig.__name__, mut)
    for name, m in list(sys.modules.items()):
        if m is None or not (name == "oracle" or name.startswith("oracle.") or
                             name.startswith("test_")):
            continue
        for attr, val in list(vars(m).items()):
            if val is orig:
                monkeypatch.setattr(m, attr, mut)


def _fails(pin_mod, pin, args):
    try:
        getattr(sys.modules[pin_mod], pin)(*args)
    except Exception:   # noqa: BLE001 -- an assertion, or an error the pin reports
        return True
    return False


@pytest.mark.parametrize("case", MUTANTS, ids=[c[0] for c in MUTANTS])
def test_a_planted_slip_fails_a_pin(case, monkeypatch):
    _, modname, site, repl, pins = case
    orig = sys.modules["oracle." + modname]
    mut = _mutant(orig, site, repl)
    _install(monkeypatch, orig, mut)
    with np.errstate(all="ignore"):
        killed = [_fails(*p) for p in pins]
    assert any(killed), f"no pin fails with the slip {site!r} -> {repl!r}"


def test_mutant_ids_are_unique_and_every_oracle_module_is_covered():
    ids = [c[0] for c in MUTANTS]
    assert len(ids) == len(set(ids))
    covered = {c[1] for c in MUTANTS}
    assert covered >= {"fisk", "hmm", "geometry", "philox", "model", "depth", "pose", "p3p",
                       "eightpoint", "posecov", "vc", "ka", "cnn"}
