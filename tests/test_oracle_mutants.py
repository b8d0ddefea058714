"""Planted mistakes: every plausible slip in the oracle must trip a pin.

Each case edits one expression (every copy of it) of a copy of oracle/flock_oracle.c (on the
CPU, in a temporary directory), builds it, points the oracle loader at it and
runs the pins of tests/pins.py.  The test passes when at least one pin fails
for every mutant, i.e. the pins would have caught that mistake."""
import os

import numpy as np
import pytest

import flock_inputs as fi
import oracle
import pins

MUTANTS = {
    "no_x_wrap": ("if (dx > d->HL) dx = dx - d->L;", "if (0) dx = dx - d->L;"),
    "wrap_wrong_sign": ("else if (dy < -d->HL) dy = dy + d->L;",
                        "else if (dy < -d->HL) dy = dy - d->L;"),
    "range_not_strict": ("if (!(d2 < d->RV2)) continue;", "if (!(d2 <= d->RV2)) continue;"),
    "collision_not_strict": ("if (d2 < d->RC2) {", "if (d2 <= d->RC2) {"),
    "penalty_dropped": ("acc -= d->PK;", "(void)0;"),
    "ramp_upside_down": ("float t = (d->RV - dist) * d->INV_SPAN;",
                         "float t = dist * d->INV_SPAN;"),
    "ly_sign": ("float ly = dy * ux - dx * uy;", "float ly = dy * ux + dx * uy;"),
    "lx_transposed": ("float lx = dx * ux + dy * uy;", "float lx = dx * uy + dy * ux;"),
    "fov_start_turned_wrong_way": ("const float ux = c * d->CF + sn * d->SF;\n  const float uy = sn * d->CF - c * d->SF;",
                                   "const float ux = c * d->CF - sn * d->SF;\n  const float uy = sn * d->CF + c * d->SF;"),
    "quadrant_offset": ("if (x < 0.0f) return 2.0f + (-y) / (-x - y);",
                        "if (x < 0.0f) return 1.0f + (-y) / (-x - y);"),
    "sector_edge_off_by_one": ("for (int m = 1; m < v; ++m)", "for (int m = 2; m < v; ++m)"),
    "fov_test_dropped": ("if (!d->full && pa >= d->T[v]) continue;", "(void)0;"),
    "sincos_quadrant": ("case 1: *c_out = -sr; *s_out = cr; break;",
                        "case 1: *c_out = sr; *s_out = cr; break;"),
    "sincos_reduction_lo_dropped": ("float r = (th - qf * PIO2_HI) - qf * PIO2_LO;",
                                    "float r = (th - qf * PIO2_HI);"),
    "speed_formula_as_printed": ("if (s < d->SMIN) s = d->SMIN;\n  else if (s > d->SMAX) s = d->SMAX;",
                                 "s = s > d->SMAX ? s : d->SMAX;\n  s = d->SMIN < s ? d->SMIN : s;"),
    "heading_not_wrapped": ("else if (th < 0.0f) th = th + d->TWO_PI;", "else if (0) th = 0;"),
    "empty_sector_value": ("obs_row[2 * k] = cnt[k] ? sqrtf(mind2[k]) : d->RV;",
                           "obs_row[2 * k] = cnt[k] ? sqrtf(mind2[k]) : 0.0f;"),
    "count_includes_self": ("if (j == i) continue;", "if (j == i && 0) continue;"),
    "turn_table_swapped": ("d->DT[0] = -p->turn_step; d->DT[1] = 0.0f; d->DT[2] = p->turn_step;",
                           "d->DT[0] = p->turn_step; d->DT[1] = 0.0f; d->DT[2] = -p->turn_step;"),
    "cont_clamp_bound_swapped": ("if (acc < -amax) acc = -amax;", "if (acc < -amax) acc = amax;"),
    "cont_components_swapped": ("move_one(d, st, acc, rot);", "move_one(d, st, rot, acc);"),
    "cont_rotation_unclamped": ("else if (acc > amax) acc = amax;\n  if (rot < -tmax) rot = -tmax;\n  else if (rot > tmax) rot = tmax;",
                                "else if (acc > amax) acc = amax;\n  if (rot < -tmax) rot = -tmax;\n  else if (0) rot = tmax;"),
    "cont_nonfinite_kept": ("    acc = 0.0f;\n    *flags |= OR_FLAG_ACTION;", "    *flags |= OR_FLAG_ACTION;"),
    "layout1_counts_for_distances": ("o[k] = row[2 * k]; /* distances */",
                                     "o[k] = row[2 * k + 1]; /* distances */"),
    "layout1_heading_for_speed": ("o[v] = row[2 * v];                             /* speed */",
                                  "o[v] = row[2 * v + 1];                             /* speed */"),
    "gae_bootstrap_from_same_step": ("(reward[k] + gamma * value[k + n]) - value[k]",
                                     "(reward[k] + gamma * value[k]) - value[k]"),
    "gae_lambda_dropped": ("const float gl = gamma * lambda;", "const float gl = gamma;"),
    "gae_target_minus_value": ("ret[k] = a + value[k];", "ret[k] = a - value[k];"),
    "gae_forward_in_time": ("for (int t = T - 1; t >= 0; --t) {\n      const size_t k",
                            "for (int t = 0; t < T; ++t) {\n      const size_t k"),
    "tag_chaser_gets_ramp": ("    } else if (touch && tj == 0) {\n      acc += d->PK;",
                             "    } else if (touch && tj == 0) {\n      acc += d->PK;\n    } else if (tj == 0) {\n      acc += (int64_t)(((d->RV - sqrtf(d2)) * d->INV_SPAN) * scaleK);"),
    "tag_runner_ramp_from_chasers": ("      else if (tj == 0) {                    /* proximity to runners */",
                                     "      else {                                 /* proximity to runners */"),
    "tag_chaser_touch_chaser_rewarded": ("    } else if (touch && tj == 0) {", "    } else if (touch) {"),
    "tag_channels_swapped": ("k += tj * v; /* colour channel of the neighbour's type */",
                             "k += (1 - tj) * v; /* colour channel of the neighbour's type */"),
    "tag_speed_added": ("  st[3] = spd;\n  move_one(d, st, 0.0f, rot);", "  move_one(d, st, spd, rot);"),
    "exact_sum_resolution_one_short": ("int K = 24 - e;", "int K = 23 - e;"),
    "exact_sum_resolution_two_short": ("int K = 24 - e;", "int K = 22 - e;"),
    "move_before_turn": ("  float c, sn;\n  oracle_sincos(th, &c, &sn);\n  float x = st[0] + s * c;",
                         "  float c, sn;\n  oracle_sincos(st[2], &c, &sn);\n  float x = st[0] + s * c;"),
}


def _pins_fail():
    """Run the pins; return the name of the first one that fails, or None."""
    checks = [("golden", lambda: [pins.check_golden(p) for p in pins.golden_cases()]),
              ("sincos", pins.check_sincos),
              ("fp64", lambda: pins.check_fp64(*pins.random_case(400, fi.side_for(400, 0.3), 21))),
              ("fp64_full", lambda: pins.check_fp64(*pins.random_case(
                  400, fi.side_for(400, 0.3), 22, fov=fi.FULL_FOV))),
              ("translation", pins.check_translation),
              ("permutation", pins.check_permutation),
              ("statistics", lambda: pins.check_statistics(n=3000, threads=0)),
              ("cont_discrete", pins.check_cont_reduces_to_discrete),
              ("cont_clamp", pins.check_cont_clamp),
              ("cont_motion", pins.check_cont_motion),
              ("cont_nonfinite", pins.check_cont_nonfinite),
              ("layout_view_only", pins.check_layout_view_only),
              ("gae_hand", pins.check_gae_hand_worked),
              ("gae_special", pins.check_gae_special_cases),
              ("gae_fp64", pins.check_gae_fp64),
              ("tag_hand", pins.check_tag_hand_worked),
              ("tag_flock", pins.check_tag_all_runners_is_flock),
              ("tag_swap", pins.check_tag_channels_swap),
              ("tag_motion", pins.check_tag_motion),
              ("exact_sum", lambda: [pins.check_exact_reward_sum(o, n=200, side=30.0) for o in
                                     ({}, {"view_radius": 7.3}, {"agent_radius": 0.0})]),
              ("exact_sum_edge", lambda: [pins.check_exact_reward_edge_pairs(o) for o in
                                          ({}, {"view_radius": 7.3},
                                           {"view_radius": pins.odd_smallest_term_radius()})])]
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, ValueError):
            return name
    return None


def test_pins_pass_on_the_oracle():
    assert _pins_fail() is None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    # a formula written out in several places (the flock and tag loops) is
    # mutated in every copy, as a slip in a shared helper would be
    assert src.count(old) >= 1, "mutation anchor not found: %r" % old
    path = oracle.build_variant(src.replace(old, new), str(tmp_path / ("m_%s.so" % name)))
    prev = oracle.use_library(path)
    try:
        caught = _pins_fail()
    finally:
        oracle.use_library(prev)
    assert caught is not None, "planted mistake %s passed every pin" % name
