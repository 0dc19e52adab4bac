"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of an oracle function (a flipped sign, a dropped
term, a transposed operand, an off-by-one rule), patches it into the oracle for the duration
of the case, and checks that the pin named for that part of the method now fails. The
mistake is planted in the oracle's own source text, so each case is the oracle with exactly
one edit. Nothing here touches the GPU path.
"""
import importlib
import inspect
import textwrap

import pytest

import oracle
import oracle.fdgs_oracle as fo

# (oracle function, text in its source, replacement, pins that must catch it: a function of
# test_oracle_pins, or "module::function" for the pins kept beside another part)
MUTATIONS = {
    "conditional mean sign (Eq. 1)": (
        "condition_on_time",
        "mu3 = mean4[..., :3] + s_xt",
        "mu3 = mean4[..., :3] - s_xt",
        ["test_eq1_mean_maximises_the_4d_density"]),
    "conditional covariance without the Schur term (Eq. 1)": (
        "condition_on_time",
        "cov3 = cov4[..., :3, :3] - s_xt[..., :, None] * s_xt[..., None, :] / s_tt[..., None, None]",
        "cov3 = cov4[..., :3, :3]",
        ["test_eq1_matches_precision_schur_complement"]),
    "temporal weight without the 1/2 (Eq. 3)": (
        "condition_on_time",
        "p = torch.exp(-0.5 * dt * dt / s_tt)",
        "p = torch.exp(-dt * dt / s_tt)",
        ["test_zero_space_time_correlation_is_a_static_splat"]),
    "transposed rotation in the 4D covariance": (
        "covariance_4d",
        "return (R * s2[..., None, :]) @ R.transpose(-1, -2)",
        "return (R.transpose(-1, -2) * s2[..., None, :]) @ R",
        ["test_covariance_eigen_structure", "test_zero_space_time_correlation_is_a_static_splat"]),
    "right-quaternion matrix transposed": (
        "right_quat_matrix",
        "torch.stack([q1, p, s, -r], -1)",
        "torch.stack([q1, p, -s, r], -1)",
        ["test_rotation_identity_and_hamilton_products"]),
    "degree-1 SH basis sign": (
        "sh_basis",
        "out += [c1 * y, c1 * z, c1 * x]",
        "out += [-c1 * y, c1 * z, c1 * x]",
        ["test_sh_basis_matches_scipy"]),
    "stop rule blends the entry that crosses T < 1e-4 (Eq. 2 reading)": (
        "blend_tile",
        "blended = used & (pos < first_stop[:, None])",
        "blended = used & (pos <= first_stop[:, None])",
        ["test_two_gaussians_and_the_stop_rule"]),
    "power > 0 not skipped": (
        "blend_tile",
        "used = (power <= 0) & (alpha >= ALPHA_MIN)",
        "used = alpha >= ALPHA_MIN",
        ["test_positive_power_is_skipped"]),
    "variation factor without the 1/2 on tanh (Eq. 6)": (
        "variation_factor",
        "return 1.0 / (0.5 * torch.tanh(torch.abs(pk)) + 0.5)",
        "return 1.0 / (torch.tanh(torch.abs(pk)) + 0.5)",
        ["test_variation_factor_range_and_fixed_points"]),
    "first derivative of p(t) without its 1/Sigma_t (score variant d, Table 4)": (
        "temporal_first_derivative",
        "return -(dt / s_tt) * p",
        "return -dt * p",
        ["test_first_derivative_by_finite_differences_and_its_factor_range"]),
    "temporal-only score variant summed over the views (Table 4 c)": (
        "variation_scores",
        """            if variant == "temporal":
                S += f * gamma
                continue""",
        """            if variant == "temporal":
                S += f * gamma * max(len(cams), 1)
                continue""",
        ["test_score_variants_against_the_spatial_score_and_each_other"]),
    "Sigma_t variant with the temporal scale instead of its variance (Table 4 e)": (
        "variation_scores",
        "g_t = cov4[:, 3, 3] * gamma",
        "g_t = torch.sqrt(cov4[:, 3, 3]) * gamma",
        ["test_score_variants_against_the_spatial_score_and_each_other"]),
    "volume normalisation not clamped": (
        "volume_gamma",
        "return torch.clamp(V / p90, 0.0, 1.0) ** beta",
        "return (V / p90) ** beta",
        ["test_volume_gamma_range_and_percentile"]),
    "mask gate takes the intersection of the two key-frames (Sec. 4.2.2)": (
        "active_from_masks",
        "return ml | mr",
        "return ml & mr",
        ["test_mask_union_of_two_keyframes"]),
    "left key-frame taken as the first one after t (Sec. 4.2.2)": (
        "keyframe_pair",
        "if kt[i] <= t:",
        "if kt[i] < t:",
        ["test_keyframe_pair_cases"]),
    "EWA covariance without the 0.3 px^2 dilation": (
        "preprocess",
        "c00 = cov2[:, 0, 0] + COV2D_DILATION",
        "c00 = cov2[:, 0, 0]",
        ["test_single_gaussian_closed_form"]),
    "Jacobian off-diagonal sign": (
        "preprocess",
        "-fx * xz / zsafe",
        "fx * xz / zsafe",
        ["test_zero_space_time_correlation_is_a_static_splat"]),
    "conic off-diagonal sign": (
        "preprocess",
        "conA, conB, conC = c11 / detsafe, -c01 / detsafe, c00 / detsafe",
        "conA, conB, conC = c11 / detsafe, c01 / detsafe, c00 / detsafe",
        ["test_zero_space_time_correlation_is_a_static_splat"]),
    "2-sigma instead of 3-sigma radius": (
        "preprocess",
        "r3 = 3.0 * torch.sqrt",
        "r3 = 2.0 * torch.sqrt",
        ["test_zero_space_time_correlation_is_a_static_splat"]),
    "tile rectangle upper edge one pixel too far": (
        "preprocess",
        "xlo_f, xhi_f = u - radius, u + radius + (TILE - 1)",
        "xlo_f, xhi_f = u - radius, u + radius + TILE",
        ["test_tile_lists_match_brute_force_coverage"]),
    "SH direction from the mean to the camera": (
        "preprocess",
        "dvec = mu3 - eye",
        "dvec = eye - mu3",
        ["test_degree1_colour_follows_the_view_direction"]),
    "depth order reversed in a tile list (Eq. 2)": (
        "tile_list",
        "return ids[np.lexsort((ids, depth))]",
        "return ids[np.lexsort((ids, -depth))]",
        ["test_tile_lists_match_brute_force_coverage"]),
    "p'' with the wrong sign on 1 / Sigma_t (Eq. 5)": (
        "temporal_second_derivative",
        "return (dt * dt / (s_tt * s_tt) - 1.0 / s_tt) * p",
        "return (dt * dt / (s_tt * s_tt) + 1.0 / s_tt) * p",
        ["test_temporal_marginal_and_second_derivative_by_finite_differences"]),
    "volume percentile one rank low": (
        "volume_gamma",
        "p90 = srt[k - 1]",
        "p90 = srt[k - 2]",
        ["test_volume_gamma_range_and_percentile"]),
    "visibility mask without the entries that stop a pixel (Sec. 4.2.2 reading)": (
        "contributing",
        "mark[tl[s_[s_ < len(tl)]]] = True",
        "pass",
        ["test_oracle_masks::test_a_gaussian_that_only_stops_pixels_is_marked"]),
    "alpha-tight box without the float32 widening": (
        "tight_tile_rect",
        "Q = 2.0 * torch.log(255.0 * a) * 1.001 + 0.1",
        "Q = 2.0 * torch.log(255.0 * a) * 0.9",
        ["test_oracle_tight::test_tight_sets_keep_every_pixel_that_can_take_alpha"]),
    "keep-set ties broken by descending id": (
        "keep_set",
        "order = np.lexsort((np.arange(n), s))",
        "order = np.lexsort((-np.arange(n), s))",
        ["test_keep_set_ties_broken_by_id"]),
}


def _mutant(name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(fo, name)))
    assert src.count(old) >= 1, f"{name}: the text to mutate is not in the oracle"
    src = src.replace(old, new, 1)
    ns = dict(vars(fo))
    exec(compile(src, f"<mutant {name}>", "exec"), ns)
    return ns[name]


@pytest.mark.parametrize("label", list(MUTATIONS))
def test_pin_catches_planted_mistake(label, monkeypatch):
    name, old, new, catchers = MUTATIONS[label]
    mutant = _mutant(name, old, new)
    monkeypatch.setattr(fo, name, mutant)
    if hasattr(oracle, name):
        monkeypatch.setattr(oracle, name, mutant)
    for pin in catchers:
        mod, _, fn = pin.rpartition("::")
        with pytest.raises(AssertionError):
            getattr(importlib.import_module(mod or "test_oracle_pins"), fn)()
