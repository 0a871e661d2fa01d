"""Planted mistakes in the oracle's two-view check, other minorants, optical
flow and research baselines: each is compiled into a copy of the oracle, the
copy replaces the oracle for the test, and at least one of the pins of that
part must fail.  A pin set that passes a plausible mistake would not be
pinning the oracle to the paper."""

import subprocess

import pytest

from oracle import oracle as O
import test_oracle_baselines as TB
import test_oracle_flow as TF
import test_oracle_lr as TLR
import test_oracle_minorants as TMIN

PINS = {
    "lr": [TLR.test_check_constant_disparity, TLR.test_check_two_planes_with_occlusion,
           TLR.test_check_rounds_half_to_even, TLR.test_check_threshold_is_inclusive_and_symmetric,
           TLR.test_check_borders_and_non_finite, lambda: TLR.test_right_cost_bruteforce(5),
           lambda: TLR.test_mirrored_pair_is_the_right_view((5, 17, 8))],
    "minorants": [lambda: TMIN.test_naive_is_min_marginals_over_n(4, 2),
                  lambda: TMIN.test_naive_is_min_marginals_over_n(3, 3),
                  lambda: TMIN.test_iterative_matches_its_definition_by_enumeration(3, (1, 4), 4, 2),
                  lambda: TMIN.test_iterative_matches_its_definition_by_enumeration(2, (1, 2), 5, 3),
                  lambda: TMIN.test_iterative_is_valid_and_maximal(3, (1, 4)),
                  lambda: TMIN.test_iterative_matches_its_definition_on_longer_chains(12, 5)],
    "flow": [lambda: TF.test_projected_costs_bruteforce(-2, 5, -1, 3),
             TF.test_data_term_is_bilinear_in_the_labels,
             lambda: TF.test_fit_is_exact_on_quadratics(1.0),
             TF.test_psd_part_is_the_eigenvalue_clamp, TF.test_prox_optimality_inside_the_box,
             TF.test_prox_with_diagonal_q_is_the_box_constrained_minimiser,
             TF.test_refine_without_regulariser_reaches_the_newton_point,
             TF.test_transposed_images_swap_the_components, TF.test_translation_is_recovered],
    "baselines": [lambda: TB.test_uniform_minorant_matches_exact_enumeration(3, 3),
                  lambda: TB.test_uniform_minorant_is_maximal_valid_and_above_m_over_n(4, 3),
                  TB.test_primal_mm_majorant_is_above_and_exact,
                  TB.test_primal_mm_is_monotone_and_above_the_minimum,
                  TB.test_primal_mm_keeps_a_global_minimiser,
                  TB.test_primal_mm_on_a_synthetic_frame_reaches_a_low_energy],
}

MUTATIONS = [
    ("check: counterpart on the wrong side", "lr",
     "const i64 xr = (i64)x - (i64)rintf(d);", "const i64 xr = (i64)x + (i64)rintf(d);"),
    ("check: rounding half up", "lr",
     "const i64 xr = (i64)x - (i64)rintf(d);", "const i64 xr = (i64)x - (i64)floorf(d + 0.5f);"),
    ("check: strict threshold", "lr", "pass = diff <= max_diff;", "pass = diff < max_diff;"),
    ("check: failing pixels keep their disparity", "lr",
     "out[i] = pass ? d : -1.0f;", "out[i] = d;"),
    ("right-view cost: images swapped", "lr",
     "if (x + l < W) v = popcount32(cr[y * W + x] ^ cl[y * W + x + l]);",
     "if (x + l < W) v = popcount32(cl[y * W + x] ^ cr[y * W + x + l]);"),
    ("naive: division toward zero", "minorants",
     "lam[e] = floor_div(lam[e], n);", "lam[e] = lam[e] / n;"),
    ("iterative: gamma < 1 on the last pass", "minorants",
     "const i64 num = s == max_pass ? 1 : gn, den = s == max_pass ? 1 : gd;",
     "const i64 num = gn, den = gd;"),
    ("iterative: forward message ignores the drained part", "minorants",
     "tmp[l] = theta[(i64)(i - 1) * K + l] - lam[(i64)(i - 1) * K + l] +",
     "tmp[l] = theta[(i64)(i - 1) * K + l] +"),
    ("iterative: the chain is never reversed", "minorants",
     "const int fwd = (s & 1) == 1;", "const int fwd = 1;"),
    ("flow: displacement sign", "flow",
     "int yy = y + d2, xx = x + d1;", "int yy = y - d2, xx = x - d1;"),
    ("flow: mixed second difference sign", "flow",
     "Q[1] = (S[2 * 3 + 2] - S[0 * 3 + 2] - S[2 * 3 + 0] + S[0 * 3 + 0]) / (4.0 * h * h);",
     "Q[1] = (S[2 * 3 + 2] + S[0 * 3 + 2] - S[2 * 3 + 0] - S[0 * 3 + 0]) / (4.0 * h * h);"),
    ("flow: gradient sign in the prox", "flow",
     "double r1 = uh1 + tau * (Q[0] * u01 + Q[1] * u02 - L[0]);",
     "double r1 = uh1 + tau * (Q[0] * u01 + Q[1] * u02 + L[0]);"),
    ("flow: negative curvature kept", "flow",
     "if (lp <= 0.0) { Q[0] = Q[1] = Q[2] = 0.0; return; }", "if (lp <= 0.0) return;"),
    ("flow: both components share the horizontal duals", "flow",
     "double* ph[2] = {D, D + 4 * N};", "double* ph[2] = {D, D};"),
    ("uniform: epsilon added to optimal labels too", "baselines",
     "            if (!O[e]) lam[e] += eps;", "            lam[e] += eps;"),
    ("primal_mm: majorant without the cap", "baselines",
     "bar[p * L + l] += 0.5 * cur + (l != a ? cap : 0.0);", "bar[p * L + l] += 0.5 * cur;"),
]


@pytest.mark.parametrize("name,group,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistakes(tmp_path, monkeypatch, name, group, old, new):
    src = open(O._SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"],
                   check=True)
    monkeypatch.setattr(O, "_lib", O.load(str(so)))
    caught = 0
    for pin in PINS[group]:
        try:
            pin()
        except Exception:      # a failed assertion, or the oracle refusing (no convergence)
            caught += 1
    assert caught > 0, f"planted mistake not caught: {name}"
