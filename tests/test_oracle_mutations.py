"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign or factor, a
transposed operand, truncation instead of floor) in a copy of the oracle's
C++ source, builds that copy, and checks that at least one of the pins for
that step now fails.  The planted mistakes live only in temporary copies on
the CPU."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_activation as A
from tests import test_oracle_beta_ssi as Bs
from tests import test_oracle_crf_loss as Cl
from tests import test_oracle_eikonal as Ek
from tests import test_oracle_fusion as Fu
from tests import test_oracle_lattice as La
from tests import test_oracle_normal as Nm
from tests import test_oracle_render as R

MUTANTS = [
    ("laplace_factor", "? 0.5 * std::exp(s / beta) :", "? std::exp(s / beta) :",
     [R.test_laplace_density_closed_forms]),
    ("trilinear_swap", "(ex ? s.f[0] : 1.0 - s.f[0])", "(ex ? 1.0 - s.f[0] : s.f[0])",
     [R.test_trilinear_reproduces_linear_field]),
    ("bwd_drop_suffix", "* v[k] - suffix - R.TN * ubg;", "* v[k] - R.TN * ubg;",
     [lambda: R.test_backward_matches_central_differences(0, (0, 0, 0))]),
    ("bwd_bg_sign", "* v[k] - suffix - R.TN * ubg;", "* v[k] - suffix + R.TN * ubg;",
     [lambda: R.test_backward_matches_central_differences(4, (0.3, 0.6, 0.1))]),
    ("activation_trunc", "v[a] = ok ? (int64_t)std::floor(q) : 0;", "v[a] = ok ? (int64_t)q : 0;",
     [A.test_activation_floor_semantics_by_hand]),
    ("unproject_transpose", "float p1 = T[a * 4 + 1] * yc;", "float p1 = T[1 * 4 + a] * yc;",
     [A.test_unprojected_points_lie_on_the_surface]),
    ("last_delta", "(k + 1 < N ? R.smp[k + 1].s : R.S)", "(k + 1 < N ? R.smp[k + 1].s : sm.s)",
     [R.test_stratified_sampling_and_deltas]),
    ("inclusive_transmittance", "sm.T = std::exp(-cum);\n        sm.w", "sm.T = std::exp(-cum - sm.tau);\n        sm.w",
     [lambda: R.test_plane_depth_matches_quadrature_and_converges(0.01)]),
    ("adam_no_bias_correction", "double mh = m[i] / c1,", "double mh = m[i],",
     [R.test_adam_step_one_closed_form_and_torch]),
    ("traverse_start_point", "double tm = 0.5 * (ta + tb);", "double tm = ta;",
     [R.test_traversal_matches_dense_classification]),
    ("dilation_off_by_one", "b1[a] = floordiv(v[a] + r, 8);", "b1[a] = floordiv(v[a] + r - 1, 8);",
     [lambda: A.test_activation_matches_voxel_cube_enumeration(3)]),
    ("fusion_sdf_sign", "float o = D - c[2];", "float o = c[2] - D;", [Fu.test_plane_sdf_is_the_truncated_distance]),
    ("fusion_transpose", "float p1 = R[1 * 4 + j] * e[1];", "float p1 = R[j * 4 + 1] * e[1];",
     [Fu.test_plane_sdf_is_the_truncated_distance, Fu.test_two_views_agree_and_weights_count]),
    ("fusion_no_truncation", "float psi = std::min(o, mu);", "float psi = o;",
     [Fu.test_plane_sdf_is_the_truncated_distance]),
    ("fusion_keeps_occluded", "if (!(o >= -mu)) continue;", "",
     [Fu.test_plane_sdf_is_the_truncated_distance]),
    ("fusion_no_translation", "e[a] = x[a] - R[a * 4 + 3];", "e[a] = x[a];",
     [Fu.test_plane_sdf_is_the_truncated_distance]),
    ("fusion_pixel_rounding", "float fu = std::floor(pu), fv = std::floor(pv);",
     "float fu = std::floor(pu + 0.5f), fv = std::floor(pv + 0.5f);", [Fu.test_pixel_centre_convention]),
    ("fusion_unnormalised_logits", "? (ss[q] / n) / nn : 0.0;", "? (ss[q] / n) : 0.0;",
     [Fu.test_colour_is_the_mean_and_logits_are_normalised]),
    ("grad_no_inv_vs", "dfac[a] = (bit[a] ? 1.0 : -1.0) / vs;", "dfac[a] = (bit[a] ? 1.0 : -1.0);",
     [Ek.test_linear_field_gradient_and_eikonal_closed_forms]),
    ("grad_sign", "dfac[a] = (bit[a] ? 1.0 : -1.0) / vs;", "dfac[a] = (bit[a] ? -1.0 : 1.0) / vs;",
     [Ek.test_linear_field_gradient_and_eikonal_closed_forms]),
    ("grad_axis_swap", "dr[1] = fac[0] * dfac[1] * fac[2];", "dr[1] = fac[0] * fac[1] * dfac[2];",
     [Ek.test_gradient_equals_central_differences_of_the_interpolant]),
    ("eikonal_unnormalised", "* 2.0 * (norm - 1.0) / norm;", "* 2.0 * (norm - 1.0);",
     [Ek.test_eikonal_gradient_equals_central_differences_of_the_loss]),
    ("eikonal_no_factor_two", "* 2.0 * (norm - 1.0) / norm;", "* (norm - 1.0) / norm;",
     [Ek.test_eikonal_gradient_equals_central_differences_of_the_loss]),
    ("dbeta_front_sign", "if (d >= 0.0) return s * (d - beta) / (beta * beta);",
     "if (d >= 0.0) return s * (beta - d) / (beta * beta);",
     [lambda: Bs.test_beta_gradient_matches_central_differences((0, 0, 0))]),
    ("dbeta_behind_term", "return -s / beta + d * std::exp(d / beta) / (2.0 * beta * beta * beta);",
     "return -s / beta;", [lambda: Bs.test_beta_gradient_matches_central_differences((0, 0, 0))]),
    ("ssi_no_shift", "b = (sd - a * st) / nn;", "b = 0.0;", [Bs.test_ssi_loss_zero_for_affine_targets_and_invariant]),
    ("ssi_grad_factor", "g_depth[i] = 2.0 * lambda * r / nn;", "g_depth[i] = lambda * r / nn;",
     [Bs.test_ssi_gradient_matches_central_differences]),
    ("normal_drop_gradf_term", "grad_sdf[li] += s.w * (gn[0] * dr[0] + gn[1] * dr[1] + gn[2] * dr[2]);", "",
     [Nm.test_normal_backward_matches_central_differences]),
    ("normal_drop_weight_term", "for (int a = 0; a < 3; ++a) vk += g_normal[3 * i + a] * s.gf[a];", "",
     [Nm.test_normal_backward_matches_central_differences]),
    ("normal_swapped_axes", "for (int a = 0; a < 3; ++a) R.Nrm[a] += sm.w * sm.gf[a];",
     "for (int a = 0; a < 3; ++a) R.Nrm[a] += sm.w * sm.gf[(a + 1) % 3];",
     [Nm.test_linear_field_renders_opacity_times_normal]),
    ("crf_label_grad_sign", "gp_[c] = k * (std::exp(logp) - t[c]);", "gp_[c] = k * (t[c] - std::exp(logp));",
     [lambda: Cl.test_crf_loss_zero_at_target_and_matches_central_differences("label")]),
    ("crf_color_factor", "gp_[c] = 2.0 * k * (v - t[c]);", "gp_[c] = k * (v - t[c]);",
     [lambda: Cl.test_crf_loss_zero_at_target_and_matches_central_differences("color")]),
    ("crf_normal_axes", "g_out[st.lin[e]] += gp_[0] * dr[0] + gp_[1] * dr[1] + gp_[2] * dr[2];",
     "g_out[st.lin[e]] += gp_[0] * dr[0] + gp_[1] * dr[2] + gp_[2] * dr[1];",
     [lambda: Cl.test_crf_loss_zero_at_target_and_matches_central_differences("normal")]),
    ("lattice_blur_weight", "w[(size_t)m * cc + q] = 0.25 * s2;", "w[(size_t)m * cc + q] = 0.5 * s2;",
     [La.test_d1_filter_is_the_grid_filter]),
    ("lattice_no_excess_fix", "    if (excess > 0) {  // too high", "    if (excess > 0 && false) {  // too high",
     [lambda: La.test_simplex_is_the_enclosing_lattice_simplex(3)]),
    ("lattice_canonical_offset", "S.vert[j][k] = r[k] + (rank[k] < d1 - j ? j : j - d1);",
     "S.vert[j][k] = r[k] + (rank[k] <= d1 - j ? j : j - d1);",
     [lambda: La.test_simplex_is_the_enclosing_lattice_simplex(2)]),
    ("lattice_affine_row", "    rhs[d] = 1.0;\n", "    rhs[d] = 0.5;\n",
     [lambda: La.test_simplex_is_the_enclosing_lattice_simplex(2)]),
    ("lattice_fp64_elevation", "const double f = scd * pd[i - 1] / std::sqrt((double)i * (double)(i + 1));",
     "const double f = scd * pd[i - 1] / std::sqrt((double)i * (double)i);",
     [lambda: La.test_simplex_is_the_enclosing_lattice_simplex(4)]),
    ("lattice_neighbour_offset", "const int64_t o = k == dir ? d : -1;", "const int64_t o = k == dir ? d + 1 : -1;",
     [La.test_d1_filter_is_the_grid_filter]),
    ("meanfield_sign", "e[l] = unary[i * L + l] + w * (tot - qt);", "e[l] = unary[i * L + l] - w * (tot - qt);",
     [La.test_meanfield_update]),
    ("normal_loss_factor", "g_normal[i] = lambda * (double)((e > 0.0) - (e < 0.0)) / (3.0 * n);",
     "g_normal[i] = lambda * (double)((e > 0.0) - (e < 0.0)) / n;",
     [Nm.test_normal_loss_seeds_match_finite_differences]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, pins, tmp_path):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / f"{name}.cpp"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", str(mutated),
                           "-o", str(so)])
    with oracle.use_library(str(so)):
        caught = False
        for pin in pins:
            try:
                pin()
            except AssertionError:
                caught = True
        assert caught, f"no pin caught the planted mistake {name}"
