"""The oracle's pins have teeth: each planted mistake fails at least one.

A mutant is a copy of ``oracle/gs_oracle.c`` with one plausible mistake (a
dropped term, a wrong sign or index, a transposed operand, a missing rule),
built with gcc into a temporary library. The original snippet must occur
exactly once, so this test breaks loudly if the oracle source changes.
"""
from __future__ import annotations

import pytest

import oracle as O
import test_oracle_pins as P

MUTANTS = {
    "no_dilation": ("double a = cov[0] + prm[P_DIL], b = cov[1], cc = cov[3] + prm[P_DIL];",
                    "double a = cov[0], b = cov[1], cc = cov[3];"),
    "conic_B_sign": ("- r[R_CB] * dx * dy;", "+ r[R_CB] * dx * dy;"),
    "camera_R_transposed": (
        "c->R[3 * i] * mu[0] + c->R[3 * i + 1] * mu[1] + c->R[3 * i + 2] * mu[2] + c->t[i];",
        "c->R[i] * mu[0] + c->R[3 + i] * mu[1] + c->R[6 + i] * mu[2] + c->t[i];"),
    "sh_no_condon_shortley": ("pmm *= -odd * s;", "pmm *= odd * s;"),
    "no_termination": ("int stop = Tn < prm[P_TMIN];", "int stop = 0;"),
    "depth_descending": ("if (a->z < b->z) return -1;\n    if (a->z > b->z) return 1;",
                         "if (a->z < b->z) return 1;\n    if (a->z > b->z) return -1;"),
    "tie_index_descending": ("return (a->g > b->g) - (a->g < b->g);",
                             "return (a->g < b->g) - (a->g > b->g);"),
    "no_guard_clamp": ("double tx = xc * z, ty = yc * z;", "double tx = xz * z, ty = yc * z;"),
    "quat_sign": ("R[1] = 2.0 * (x * y - w * z);", "R[1] = 2.0 * (x * y + w * z);"),
    "no_alpha_max": ("double alpha = araw < prm[P_AMAX] ? araw : prm[P_AMAX];",
                     "double alpha = araw;"),
    "no_alpha_min_skip": ("int skip = araw < prm[P_AMIN];", "int skip = 0;"),
    "sh_dir_reversed": (
        "double d[3] = {mu[0] - c->cpos[0], mu[1] - c->cpos[1], mu[2] - c->cpos[2]};",
        "double d[3] = {c->cpos[0] - mu[0], c->cpos[1] - mu[1], c->cpos[2] - mu[2]};"),
    "pixel_centre_no_half": ("w.px = i + 0.5;", "w.px = i;"),
    "radius_lambda_min": ("double lmax = mid + sqrt(", "double lmax = mid - sqrt("),
    "depth_weight_T": ("D += wt * r[R_Z];", "D += T * r[R_Z];"),
    "camera_centre_sign": ("c->cpos[j] = -s;", "c->cpos[j] = s;"),
    "rect_ceil": ("int x0 = (int)floor(lo_x / ts)", "int x0 = (int)ceil(lo_x / ts)"),
    "sigmoid_sign": ("return 1.0 / (1.0 + exp(-x));", "return 1.0 / (1.0 + exp(x));"),
    "cov_R_transposed": ("M[3 * i + j] = R[3 * i + j] * exp(log_scale[j]);",
                         "M[3 * i + j] = R[3 * j + i] * exp(log_scale[j]);"),
    "jacobian_y_uses_fx": ("0.0, c->fy / z, -c->fy * ty / (z * z)};",
                           "0.0, c->fx / z, -c->fy * ty / (z * z)};"),
    "T_update_wrong": ("double Tn = T * (1.0 - alpha);", "double Tn = T * (1.0 - 0.5 * alpha);"),
    "sh_m_sign_swapped": ("v = sqrt(2.0) * K * cos(m * phi) * P;",
                          "v = sqrt(2.0) * K * sin(m * phi) * P;"),
}

PINS = [
    P.test_sh_matches_cartesian_table,
    P.test_sh_orthonormal_by_quadrature,
    P.test_quaternion_rotation_matches_library,
    P.test_cov3d_is_rotated_diag,
    lambda o: P.test_single_gaussian_closed_form(o, 2.0, 0.05, 0.7, (0.9, 0.4, 0.1)),
    lambda o: P.test_single_gaussian_closed_form(o, 0.8, 0.01, 0.3, (1.0, 1.0, 1.0)),
    P.test_sheared_footprint_pixels,
    lambda o: P.test_off_axis_anisotropic_jacobian(o, 50.0, 35.0),
    P.test_guard_band_clamp,
    P.test_two_gaussians_depth_order,
    P.test_termination_excludes_crossing_gaussian,
    P.test_alpha_threshold,
    P.test_sum_of_weights_plus_T_is_one,
    P.test_rigid_motion_invariance,
    P.test_sh_view_direction,
    P.test_near_plane_and_behind,
    P.test_tile_lists_sorted_and_complete,
    P.test_covering_all_tiles_and_partial_row,
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(O.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutant anchor for {name} not unique in the oracle source"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = O.build(str(msrc), str(tmp_path / "libmutant.so"), force=True)
    mut = O.Oracle(lib)
    caught = []
    for pin in PINS:
        try:
            pin(mut)
        except AssertionError:
            caught.append(getattr(pin, "__name__", "lambda"))
    assert caught, f"planted mistake {name!r} passed every pin"


def test_unmutated_source_passes_every_pin(tmp_path):
    lib = O.build(O.SRC, str(tmp_path / "libcopy.so"), force=True)
    o = O.Oracle(lib)
    for pin in PINS:
        pin(o)
