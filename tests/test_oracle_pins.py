"""Oracle pins (CPU only): the FP32 oracle against hand-derived cases, a float64
restatement, invariances and closed-form statistics.  See tests/pins.py."""
import math
import os

import numpy as np
import pytest

import flock_inputs as fi
import oracle
import pins


@pytest.mark.parametrize("path", pins.golden_cases(), ids=os.path.basename)
def test_golden(path):
    pins.check_golden(path)


def test_golden_present():
    assert len(pins.golden_cases()) >= 7


@pytest.mark.parametrize("over", [
    {},
    {"fov": fi.FULL_FOV},
    {"num_segments": 5},
    {"num_segments": 1, "fov": fi.FULL_FOV},
    {"num_segments": 16, "fov": float(np.float32(math.radians(120)))},
    {"agent_radius": 0.0},
], ids=lambda d: ",".join("%s=%s" % kv for kv in d.items()) or "default")
def test_fp64_reevaluation(over):
    n = 600
    side = fi.side_for(n, 0.3)  # denser than the benchmark: more pairs per agent
    p, st, act = pins.random_case(n, side, 21, **over)
    frac = pins.check_fp64(p, st, act)
    assert frac > 0.8


def test_fp64_reevaluation_small_side():
    # a square only just wider than 2 d_v: many pairs wrap
    p, st, act = pins.random_case(200, 11.0, 4)
    pins.check_fp64(p, st, act)


def test_translation_invariance():
    pins.check_translation()


def test_permutation_equivariance():
    pins.check_permutation()


def test_statistics_uniform():
    pins.check_statistics(threads=0)


def test_statistics_full_circle():
    pins.check_statistics(fov=fi.FULL_FOV, seed=12, threads=0)


def test_sincos_accuracy():
    pins.check_sincos()


def test_diamond_pseudo_angle():
    # quadrant anchors and monotonicity against the true angle
    assert oracle.diamond(1.0, 0.0) == 0.0
    assert oracle.diamond(1.0, 1.0) == 0.5
    assert oracle.diamond(0.0, 1.0) == 1.0
    assert oracle.diamond(-1.0, 0.0) == 2.0
    assert oracle.diamond(0.0, -1.0) == 3.0
    ang = np.linspace(0, 2 * math.pi, 2001)[:-1]
    vals = [oracle.diamond(float(np.float32(math.cos(a))), float(np.float32(math.sin(a))))
            for a in ang]
    assert all(b >= a for a, b in zip(vals, vals[1:]))


def test_derived_constants_full_circle():
    p = fi.default_params(100.0, fov=fi.FULL_FOV)
    d = oracle.derive(p)
    assert d["full"] == 1 and d["CF"] == -1.0 and d["SF"] == 0.0
    # edges every 45 degrees: pseudo-angles 0.5, 1, ..., 3.5
    assert d["T"][:7] == [0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5]
    assert d["K"] == 46 and d["PK"] == 2 ** 46
    assert d["RV2"] == 25.0 and d["RC2"] == 1.0 and d["INV_SPAN"] == 0.25


def test_empty_and_single():
    p = fi.default_params(100.0)
    st, obs, rew, coll, flags = oracle.step(p, np.zeros((0, 4), np.float32),
                                            np.zeros(0, np.int32))
    assert obs.shape == (0, 18) and flags == 0
    one = np.array([[10.0, 20.0, 1.0, 0.5]], np.float32)
    st, obs, rew, coll, flags = oracle.step(p, one, np.array([4], np.int32))
    assert rew[0] == 0.0 and coll[0] == 0
    assert np.all(obs[0, 0:16:2] == 5.0) and np.all(obs[0, 1:16:2] == 0.0)


def test_invalid_action_flag():
    p = fi.default_params(100.0)
    st = fi.initial_state(10, 100.0, 0)
    a = np.full(10, 4, np.int32)
    a[3] = 9
    a[5] = -1
    s1, _, _, _, flags = oracle.step(p, st, a)
    s2, _, _, _, flags2 = oracle.step(p, st, np.full(10, 4, np.int32))
    assert flags == oracle.FLAG_ACTION and flags2 == 0
    np.testing.assert_array_equal(s1, s2)


def test_state_range_flag():
    p = fi.default_params(100.0)
    st = fi.initial_state(4, 100.0, 0)
    st[2, 0] = 100.0  # x == L is outside [0, L)
    _, _, _, _, flags = oracle.step(p, st, None)
    assert flags == oracle.FLAG_STATE


def test_invalid_params():
    for bad in ({"view_radius": 0.0}, {"agent_radius": 3.0}, {"num_segments": 0},
                {"num_segments": 129}, {"fov": 7.0}, {"side": 9.0}, {"speed_max": -1.0}):
        assert not oracle.params_ok(dict(fi.default_params(100.0), **bad)), bad
    assert oracle.params_ok(fi.default_params(100.0))


def test_continuous_actions_reduce_to_discrete():
    pins.check_cont_reduces_to_discrete()


def test_continuous_actions_clamp():
    pins.check_cont_clamp()


def test_continuous_motion_closed_form():
    pins.check_cont_motion()


def test_continuous_nonfinite_action():
    pins.check_cont_nonfinite()


def test_view_only_layout():
    pins.check_layout_view_only()


def test_gae_hand_worked():
    pins.check_gae_hand_worked()


def test_gae_special_cases():
    pins.check_gae_special_cases()


def test_gae_against_float64():
    pins.check_gae_fp64()


def test_tag_hand_worked():
    pins.check_tag_hand_worked()


def test_tag_without_chasers_is_the_flock():
    pins.check_tag_all_runners_is_flock()


def test_tag_type_swap_swaps_channels():
    pins.check_tag_channels_swap()


def test_tag_motion_closed_form():
    pins.check_tag_motion()


def test_rounded_sqrt_is_monotone():
    """The identity the neighbour kernels rely on when they keep each sector's
    minimum as a distance: correctly rounded float32 sqrt is monotone, so the
    minimum of the rounded roots is the rounded root of the minimum d^2 (the
    observation's nearest distance).  Checked on every 61st float32 bit
    pattern in [0, 26) and on random sets of squared distances."""
    bits = np.arange(0, np.float32(26.0).view(np.uint32), 61, dtype=np.uint32)
    x = bits.view(np.float32)
    r = np.sqrt(x)
    assert r.dtype == np.float32 and np.all(np.diff(r) >= 0)
    rng = np.random.default_rng(5)
    for _ in range(200):
        d2 = (rng.random(rng.integers(1, 40)) * 25.0).astype(np.float32)
        assert np.sqrt(d2).min().view(np.uint32) == np.sqrt(d2.min()).view(np.uint32)


def test_fraction_rounding_helper():
    """fraction_to_f32 agrees with numpy's correctly rounded conversion where
    float64 holds the value exactly, and rounds ties to even."""
    from fractions import Fraction
    rng = np.random.default_rng(7)
    for v in rng.standard_normal(2000) * 10.0 ** rng.integers(-8, 8, 2000):
        assert pins.fraction_to_f32(Fraction(float(v))) == np.float32(v)
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 23)
    assert pins.fraction_to_f32(one + ulp / 2) == np.float32(1.0)  # tie to even (down)
    assert pins.fraction_to_f32(one + 3 * ulp / 2) == np.float32(1.0 + 2 * 2.0 ** -23)  # up
    assert pins.fraction_to_f32(one + ulp / 2 + Fraction(1, 2 ** 60)) == np.float32(1.0 + 2.0 ** -23)


def test_reward_is_the_exact_sum_for_several_resolutions():
    """Reading 15 against an independent exact sum (rationals, one rounding),
    on parameter sets whose fixed-point resolutions 2^-K differ: the
    defaults (K = 46), a view radius of 7.3 (47), a penalty of 0.375, agents
    of radius 0 (no collisions; ramp terms up to 1), a penalty of 3 * 2^-30
    (K set by the penalty, 52) and a view radius of 0.3 on a square of side 4
    (45)."""
    ks = set()
    for over, side in (({}, 40.0), ({"view_radius": 7.3}, 40.0),
                       ({"collision_penalty": 0.375}, 40.0), ({"agent_radius": 0.0}, 40.0),
                       ({"collision_penalty": 3.0 * 2.0 ** -30}, 40.0),
                       ({"view_radius": 0.3, "agent_radius": 0.1}, 4.0)):
        ks.add(pins.check_exact_reward_sum(over, side=side))
    assert len(ks) >= 4, ks


@pytest.mark.parametrize("over", [{}, {"view_radius": 7.3}, {"view_radius": 3.1},
                                  {"view_radius": 7.3, "agent_radius": 0.0}, "odd"])
def test_smallest_ramp_terms_are_exact(over):
    """Pairs just inside the view radius: each reward is the pair's own
    (smallest possible) ramp term, exactly.  "odd": a radius whose smallest
    term has an odd significand, where the resolution 2^-K must be exactly
    as fine as that term's last bit (and is: K is the least that holds it)."""
    if over == "odd":
        rv = pins.odd_smallest_term_radius()
        over = {"view_radius": rv}
        p = fi.default_params(200.0, **over)
        t = pins.smallest_term(p)
        K = oracle.derive(p)["K"]
        scaled = float(t) * 2.0 ** K
        assert scaled == int(scaled) and int(scaled) % 2 == 1, (rv, K)
    pins.check_exact_reward_edge_pairs(over)
