"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each case edits one line of a temporary copy of ``oracle/rogs_oracle.c`` (a
transposed operand, a dropped term, a wrong sign or index), builds it, and
runs the pins of ``test_oracle_pins`` against that build.  The committed
oracle is never modified.
"""
import os
import shutil
import tempfile

import pytest

import oracle
import test_oracle_box as box
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rogs_oracle.c")

MUTATIONS = {
    "transposed_world_to_camera": (
        "p[r] = c->R[3 * r] * x[0] + c->R[3 * r + 1] * x[1] + c->R[3 * r + 2] * x[2] + c->t[r];",
        "p[r] = c->R[r] * x[0] + c->R[3 + r] * x[1] + c->R[6 + r] * x[2] + c->t[r];"),
    "dropped_eps": ("s00 += cfg->eps; s11 += cfg->eps;", ""),
    "covariance_uses_normal_column": (
        "for (int r = 0; r < 3; ++r) { M[r][0] = Rq[3 * r] * sx; M[r][1] = Rq[3 * r + 1] * sy; }\n    double Sig",
        "for (int r = 0; r < 3; ++r) { M[r][0] = Rq[3 * r] * sx; M[r][1] = Rq[3 * r + 2] * sy; }\n    double Sig"),
    "back_to_front_sort": (
        "if (a->key < b->key) return -1;\n    if (a->key > b->key) return 1;\n    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);\n}\n\n/* Gather",
        "if (a->key < b->key) return 1;\n    if (a->key > b->key) return -1;\n    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);\n}\n\n/* Gather"),
    "ties_by_descending_index": (
        "return (a->idx < b->idx) ? -1 : (a->idx > b->idx);\n}\n\n/* Gather",
        "return (a->idx > b->idx) ? -1 : (a->idx < b->idx);\n}\n\n/* Gather"),
    "stop_keeps_crossing_surfel": (
        "if (Tn < cfg->t_min) break;\n        T = Tn;",
        "T = Tn;\n        if (Tn < cfg->t_min) { ++k; break; }"),
    "exposure_inside": ("o[ch] = ea * o[ch] + eb;", "o[ch] = ea * (o[ch] + eb);"),
    "mean_uses_cy": ("o->mu[0] = c->fx * p[0] / z + c->cx;", "o->mu[0] = c->fx * p[0] / z + c->cy;"),
    "suffix_sign": ("da += G[ch] * (T * f[ch] - S_suf[ch] / (1.0 - a));",
                    "da += G[ch] * (T * f[ch] + S_suf[ch] / (1.0 - a));"),
    "quat_derivative_sign": ("dqn[0] = 2 * (-z * dR[1]", "dqn[0] = 2 * (z * dR[1]"),
    "n3_as_row": ("double n31 = pv[3 + 2], n32 = pv[3 + 5], n33 = pv[3 + 8];",
                  "double n31 = pv[3 + 6], n32 = pv[3 + 7], n33 = pv[3 + 8];"),
    "conic_off_diagonal_sign": ("o->con[1] = -s01 / det;", "o->con[1] = s01 / det;"),
    "jacobian_depth_term_dropped": ("J[0][2] = -c->fx * u / z;", "J[0][2] = 0;"),
    "mean_gradient_missing_offdiag": ("gg[0] += dpow * (o->con[0] * dx + o->con[1] * dy);",
                                      "gg[0] += dpow * (o->con[0] * dx);"),
    # perspective box cull (supplementary "Perspective Rendering Acceleration")
    "box_axes_swapped": ("float l0 = dx * c->xh0;\n    float l1 = dy * c->xh1;",
                         "float l0 = dx * c->zh0;\n    float l1 = dy * c->zh1;"),
    "box_forward_sign": ("float fwd = f0 + f1;", "float fwd = -(f0 + f1);"),
    "box_sizes_swapped": ("(fabsf(lat) <= cfg->f_box_hx) && (fwd >= 0.0f) && (fwd <= cfg->f_box_d)",
                          "(fabsf(lat) <= cfg->f_box_d) && (fwd >= 0.0f) && (fwd <= cfg->f_box_hx)"),
    "box_forward_axis_unnormalised": ("c->zh0 = c->fR[6] / nz; c->zh1 = c->fR[7] / nz;",
                                      "c->zh0 = c->fR[6]; c->zh1 = c->fR[7];"),
    "box_lateral_axis_unnormalised": ("c->xh0 = c->fR[0] / nx; c->xh1 = c->fR[1] / nx;",
                                      "c->xh0 = c->fR[0]; c->xh1 = c->fR[1];"),
    "box_lateral_axis_from_column": ("c->xh0 = c->fR[0] / nx; c->xh1 = c->fR[1] / nx;",
                                     "c->xh0 = c->fR[0] / nx; c->xh1 = c->fR[3] / nx;"),
    "box_centre_sign": ("c->ox = -s;", "c->ox = s;"),
}

PIN_CALLS = [
    pins.test_fronto_parallel_surfel_closed_form,
    pins.test_tilted_surfel_uses_jacobian_third_column,
    pins.test_ortho_flat_road_closed_form,
    pins.test_projection_table_matches_closed_form,
    lambda: pins.test_two_surfel_compositing_closed_form((0, 1)),
    lambda: pins.test_two_surfel_compositing_closed_form((1, 0)),
    pins.test_equal_depth_breaks_ties_by_index,
    pins.test_early_stop_excludes_the_surfel_that_crosses_t_min,
    pins.test_exposure_is_affine_in_the_composite,
    pins.test_init_on_tilted_plane_is_exact,
    pins.test_init_yaw_only_and_small_roll_reading,
    pins.test_gradient_matches_central_differences,
    *[(lambda c=c: box.test_box_cull_keeps_exactly_the_hand_worked_box(c)) for c in box.CASES],
    box.test_box_cull_pitched_camera_needs_normalised_forward_axis,
    box.test_box_cull_rolled_camera_needs_normalised_lateral_axis,
]


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="orc_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmpdir_mod):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path_c = os.path.join(tmpdir_mod, f"{name}.c")
    path_so = os.path.join(tmpdir_mod, f"{name}.so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    oracle.build(force=True, src=path_c, out=path_so)
    failed = []
    with oracle.using(path_so):
        for call in PIN_CALLS:
            try:
                call()
            except AssertionError:
                failed.append(getattr(call, "__name__", "lambda"))
                break
    assert failed, f"no pin caught the planted mistake {name}"
