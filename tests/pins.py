"""Checks that pin the FP32 oracle to facts other than itself.

Each function raises AssertionError on a violation.  They are used directly
by test_oracle_pins.py and, against deliberately broken copies of the
oracle, by test_oracle_mutants.py (which requires that every planted mistake
trips at least one of them).

Pins (arXiv 2207.03945, Section 4.1, Eq. 1, Fig. 3, Fig. 4):
* hand-derived small cases in tests/golden/ (exact values);
* a float64 restatement with true angles and distances (oracle/fp64.py):
  every decision agrees away from boundaries;
* translation invariance on a dyadic grid (exact arithmetic);
* permutation equivariance (relabelling agents);
* closed-form statistics of uniform agents (Poisson neighbour counts);
* the deterministic sine/cosine against the library's float64 sin/cos.
"""
from __future__ import annotations

import glob
import json
import math
import os

import numpy as np

import fp64
import oracle
import flock_inputs as fi

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_cases():
    return sorted(glob.glob(os.path.join(GOLDEN, "*.json")))


def check_golden(path):
    fx = json.load(open(path))
    p = fx["params"]
    st = np.array(fx["state"], np.float32)
    act = np.array(fx["actions"], np.int32) if fx.get("actions") is not None else None
    st2, obs, rew, coll, flags = oracle.step(p, st, act)
    ex = fx["expect"]
    rows = ex.get("rows", list(range(len(st))))
    assert flags == 0, (fx["name"], flags)
    if "state" in ex:
        np.testing.assert_array_equal(st2, np.array(ex["state"], np.float32), err_msg=fx["name"])
    np.testing.assert_array_equal(rew[rows], np.array(ex["reward"], np.float32), err_msg=fx["name"])
    np.testing.assert_array_equal(coll[rows], np.array(ex["coll"], np.int32), err_msg=fx["name"])
    v = int(p["num_segments"])
    rv = np.float32(p["view_radius"])
    for r in rows:
        want = np.tile(np.array([rv, 0.0], np.float32), v)
        for k, c, d in ex.get("sectors", {}).get(str(r), []):
            want[2 * k] = np.float32(d)
            want[2 * k + 1] = np.float32(c)
        if str(r) in ex.get("sectors", {}):
            np.testing.assert_array_equal(obs[r, :2 * v], want, err_msg="%s row %d" % (fx["name"], r))
        np.testing.assert_array_equal(obs[r, 2 * v:], st2[r, [3, 2]], err_msg=fx["name"])


def random_case(n, side, seed, **over):
    p = fi.default_params(side, **over)
    st = fi.initial_state(n, side, seed)
    act = fi.random_actions(n, 1, seed)[0]
    return p, st, act


def check_fp64(p, st, act, tol_reward=1e-5):
    """Oracle step vs the float64 restatement: exact decisions away from edges."""
    st2, obs, rew, coll, flags = oracle.step(p, st, act)
    assert flags == 0
    # motion against float64 cos/sin: the FP32 path differs by rounding only
    ref_st = fp64.apply_fp64(p, st, act)
    L = float(np.float32(p["side"]))
    dxy = np.abs(st2[:, :2].astype(np.float64) - ref_st[:, :2])
    dxy = np.minimum(dxy, L - dxy)  # a wrap may land on either side of 0
    assert dxy.max() <= 8 * np.spacing(np.float32(L)), dxy.max()
    dth = np.abs(st2[:, 2] - ref_st[:, 2])
    dth = np.minimum(dth, 2 * math.pi - dth)
    assert dth.max() <= 1e-6, dth.max()
    np.testing.assert_array_equal(st2[:, 3], ref_st[:, 3].astype(np.float32))
    ref = fp64.reevaluate(p, st2)
    ok = ~ref["ambiguous"]
    assert ok.mean() > 0.5, ok.mean()
    v = int(p["num_segments"])
    cnt = obs[:, 1:2 * v:2].astype(np.int64)
    mind = obs[:, 0:2 * v:2].astype(np.float64)
    np.testing.assert_array_equal(coll[ok], ref["coll"][ok])
    np.testing.assert_array_equal(cnt[ok], ref["cnt"][ok])
    # rounding of d^2 and sqrt (relative), plus one rounding of x_j - x_i at
    # the magnitude of the side for pairs that wrap (absolute)
    tol_d = 4e-7 * np.maximum(ref["mind"][ok], 1.0) + 2 * float(np.spacing(np.float32(L)))
    assert np.all(np.abs(mind[ok] - ref["mind"][ok]) <= tol_d)
    err = np.abs(rew.astype(np.float64) - ref["reward"])
    bound = tol_reward * np.maximum(1.0, ref["absf"])
    assert np.all(err[ok] <= bound[ok]), float((err[ok] - bound[ok]).max())
    return ok.mean()


def check_translation(seed=3, n=400, side=64.0):
    """Dyadic positions (multiples of 1/8) shifted by a dyadic offset modulo
    the side: every difference is exact, so the outputs must be identical."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = fi.default_params(side)
    st = np.zeros((n, 4), np.float32)
    st[:, 0] = rng.integers(0, int(side * 8), n) / 8.0
    st[:, 1] = rng.integers(0, int(side * 8), n) / 8.0
    st[:, 2] = fi.initial_state(n, side, seed)[:, 2]
    st[:, 3] = 0.0
    act = np.full(n, 4, np.int32)
    _, obs0, rew0, coll0, _ = oracle.step(p, st, act)
    for ox, oy in ((13.25, 0.0), (0.0, 40.5), (63.875, 31.0)):
        st2 = st.copy()
        st2[:, 0] = np.mod(st[:, 0] + ox, side)
        st2[:, 1] = np.mod(st[:, 1] + oy, side)
        _, obs1, rew1, coll1, _ = oracle.step(p, st2, act)
        np.testing.assert_array_equal(obs1, obs0)
        np.testing.assert_array_equal(rew1, rew0)
        np.testing.assert_array_equal(coll1, coll0)


def check_permutation(seed=5, n=300):
    side = fi.side_for(n, 0.3)
    p, st, act = random_case(n, side, seed)
    _, obs0, rew0, coll0, _ = oracle.step(p, st, act)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
    _, obs1, rew1, coll1, _ = oracle.step(p, st[perm], act[perm])
    np.testing.assert_array_equal(obs1, obs0[perm])
    np.testing.assert_array_equal(rew1, rew0[perm])
    np.testing.assert_array_equal(coll1, coll0[perm])


def check_statistics(n=5000, seed=11, fov=None, threads=0):
    """Uniform agents at density rho: in-range neighbour counts are Poisson
    with mean rho*pi*d_v^2 (7.854), collisions rho*pi*(2 d_r)^2 (0.314), and
    each of the v sectors of a field of view fov holds mean rho*pi*d_v^2*fov/(2pi*v)."""
    side = fi.side_for(n)
    over = {} if fov is None else {"fov": fov}
    p = fi.default_params(side, **over)
    st = fi.initial_state(n, side, seed)
    _, obs, rew, coll, _ = oracle.step(p, st, None, threads=threads)
    rho = n / float(np.float32(side)) ** 2
    v = int(p["num_segments"])
    lam = rho * math.pi * 25.0
    lam_c = rho * math.pi * 1.0
    fovv = float(np.float32(p["fov"]))
    lam_k = lam * fovv / (2 * math.pi) / v
    cnt = obs[:, 1:2 * v:2]
    # neighbour counts of nearby agents are correlated (each pair counted
    # twice); 5 sigma of the per-agent Poisson spread, doubled, is generous
    def within(x, mean, var):
        return abs(float(np.mean(x)) - mean) <= 10 * math.sqrt(var / n)
    assert within(coll, lam_c, lam_c), (np.mean(coll), lam_c)
    assert within(cnt.sum(axis=1), lam * fovv / (2 * math.pi), lam), (cnt.sum(1).mean(), lam)
    for k in range(v):
        assert within(cnt[:, k], lam_k, lam_k), (k, cnt[:, k].mean(), lam_k)
    # reward mean: E[sum f] = rho * (-P * pi (2d_r)^2 + int_{2d_r}^{d_v} 2 pi r (d_v-r)/(d_v-2d_r) dr)
    ramp = 2 * math.pi * (5.0 * (25 - 1) / 2 - (125 - 1) / 3) / 4.0
    mean_r = rho * (-1.0 * math.pi * 1.0 + ramp)
    assert abs(float(np.mean(rew)) - mean_r) <= 10 * math.sqrt(lam / n), (np.mean(rew), mean_r)


def check_sincos():
    rng = np.random.Generator(np.random.PCG64(1))
    th = np.concatenate([rng.random(4000) * 2 * math.pi,
                         np.arange(0, 64) * (math.pi / 32)]).astype(np.float32)
    th = th[th < fi.TWO_PI_F32]
    worst = 0.0
    for t in th:
        c, s = oracle.sincos(float(t))
        worst = max(worst, abs(c - math.cos(float(t))), abs(s - math.sin(float(t))))
    assert worst <= 2e-7, worst
    assert oracle.sincos(0.0) == (1.0, 0.0)
