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

Pins of the paper's own flock variant (continuous two-dimensional actions,
the view-only observation of Section 4.1):
* continuous actions equal to the discrete steps {-a, 0, +a} x {-Delta, 0,
  +Delta} reproduce the pinned discrete update bit for bit;
* actions outside the ranges act as the clamped ones;
* one move against the closed form x + s cos(theta), y + s sin(theta) in
  float64 (to the FP32 rounding of the terms);
* a non-finite component acts as 0 and is flagged;
* the view-only layout holds exactly the distance columns and the speed of
  the pinned (distance, count) layout.
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


def check_cont_reduces_to_discrete(seed=31, n=500):
    """Continuous actions taken from the nine discrete ones give the discrete
    update: same state, observation, reward and collisions, bit for bit."""
    side = fi.side_for(n)
    p = fi.default_params(side)
    st = fi.initial_state(n, side, seed)
    a = fi.random_actions(n, 1, seed)[0]
    amax, tmax = np.float32(p["speed_step"]), np.float32(p["turn_step"])
    ds = np.array([-amax, 0.0, amax], np.float32)
    dt = np.array([-tmax, 0.0, tmax], np.float32)
    ca = np.stack([ds[a % 3], dt[a // 3]], axis=1).astype(np.float32)
    s1, o1, r1, c1, f1 = oracle.step(p, st, a, threads=0)
    s2, o2, r2, c2, f2 = oracle.step_cont(p, st, ca, layout=0, threads=0)
    for x, y, what in ((s1, s2, "state"), (o1, o2, "obs"), (r1, r2, "reward"), (c1, c2, "coll")):
        np.testing.assert_array_equal(x, y, err_msg="continuous vs discrete " + what)
    assert f1 == f2 == 0


def check_cont_clamp(seed=37, n=300):
    """Out-of-range actions act as the clamped ones."""
    side = fi.side_for(n)
    p = fi.default_params(side)
    st = fi.initial_state(n, side, seed)
    amax, tmax = np.float32(p["speed_step"]), np.float32(p["turn_step"])
    ca = fi.random_cont_actions(n, 1, seed, float(amax), float(tmax), over=3.0)[0]
    clipped = np.stack([np.clip(ca[:, 0], -amax, amax), np.clip(ca[:, 1], -tmax, tmax)],
                       axis=1).astype(np.float32)
    assert (np.abs(ca[:, 0]) > amax).any() and (np.abs(ca[:, 1]) > tmax).any()
    a = oracle.step_cont(p, st, ca, layout=1, threads=0)
    b = oracle.step_cont(p, st, clipped, layout=1, threads=0)
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y, err_msg="clamped actions")


def check_cont_motion():
    """One agent, no neighbours: speed and heading change by the action, the
    agent moves by s' (cos theta', sin theta') (float64 closed form)."""
    p = fi.default_params(100.0)
    cases = [((50.0, 50.0, 1.0, 0.5), (0.1, 0.2)),
             ((99.9, 0.05, 0.05, 0.75), (-0.2, -0.3)),   # heading wraps below 0, x and y wrap
             ((10.0, 20.0, 6.2, 0.9), (0.25, 0.3))]      # speed clamps at 1, heading wraps above 2 pi
    for st0, act in cases:
        st = np.array([st0], np.float32)
        s2, obs, _, _, flags = oracle.step_cont(p, st, np.array([act], np.float32), layout=1)
        assert flags == 0
        s = min(max(float(np.float32(np.float32(st0[3]) + np.float32(act[0]))), 0.0), 1.0)
        th = float(np.float32(np.float32(st0[2]) + np.float32(act[1])))
        two_pi = float(np.float32(2 * math.pi))
        if th < 0:
            th = float(np.float32(th + two_pi))
        elif th >= two_pi:
            th = float(np.float32(th - two_pi))
        x = (st0[0] + s * math.cos(th)) % 100.0
        y = (st0[1] + s * math.sin(th)) % 100.0
        assert abs(float(s2[0, 3]) - s) == 0.0 and abs(float(s2[0, 2]) - th) == 0.0
        assert abs(float(s2[0, 0]) - x) < 3e-5 and abs(float(s2[0, 1]) - y) < 3e-5, (s2, x, y)
        # view-only row: every sector empty (distance d_v), then the speed
        assert np.all(obs[0, :8] == np.float32(p["view_radius"])) and obs[0, 8] == s2[0, 3]


def check_cont_nonfinite():
    """A non-finite component acts as 0 and raises the action flag."""
    n = 50
    p = fi.default_params(40.0)
    st = fi.initial_state(n, 40.0, 41)
    ca = np.zeros((n, 2), np.float32)
    bad = ca.copy()
    bad[3, 0] = np.nan
    bad[7, 1] = np.inf
    a = oracle.step_cont(p, st, ca, layout=1)
    b = oracle.step_cont(p, st, bad, layout=1)
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)
    assert a[4] == 0 and b[4] == oracle.FLAG_ACTION


def check_layout_view_only(seed=43, n=600):
    """Layout 1 (the paper's 129-value observation for v = 128) holds the
    distance columns and the speed of layout 0."""
    p = fi.paper_params(n)
    st = fi.initial_state(n, p["side"], seed)
    ca = fi.random_cont_actions(n, 1, seed, p["speed_step"], p["turn_step"])[0]
    s0, o0, r0, c0, f0 = oracle.step_cont(p, st, ca, layout=0)
    s1, o1, r1, c1, f1 = oracle.step_cont(p, st, ca, layout=1)
    v = int(p["num_segments"])
    assert o1.shape == (n, v + 1) and o0.shape == (n, 2 * v + 2)
    np.testing.assert_array_equal(o1[:, :v], o0[:, 0:2 * v:2])
    np.testing.assert_array_equal(o1[:, v], o0[:, 2 * v])
    np.testing.assert_array_equal(o1[:, v], s1[:, 3])
    for x, y in ((s0, s1), (r0, r1), (c0, c1)):
        np.testing.assert_array_equal(x, y)
    # a tenth of the side: about 0.1 pi (L/10)^2 = pi n / 100 neighbours in range
    assert (o0[:, 1:2 * v:2].sum(axis=1) > 0).mean() > 0.9


# ---------------------------------------------------------------------------
# Advantages over a rollout (generalised advantage estimation, FP32)
# ---------------------------------------------------------------------------
def _gae64(r, v, gamma, lam):
    """The recursion in float64 (a second statement, for error bounds)."""
    T, n = r.shape
    r = r.astype(np.float64)
    v = v.astype(np.float64)
    adv = np.zeros((T, n))
    a = np.zeros(n)
    for t in range(T - 1, -1, -1):
        a = r[t] + gamma * v[t + 1] - v[t] + gamma * lam * a
        adv[t] = a
    return adv


def check_gae_hand_worked():
    """Reward 1 every step, values 0, gamma 1/2, lambda 1: the discounted sum
    of the remaining rewards, 1, 1.5, 1.75, ... exactly."""
    T, n = 6, 3
    r = np.ones((T, n), np.float32)
    v = np.zeros((T + 1, n), np.float32)
    adv, ret = oracle.gae(r, v, 0.5, 1.0)
    want = np.array([2.0 - 0.5 ** (T - 1 - t) for t in range(T)], np.float32)
    np.testing.assert_array_equal(adv, np.repeat(want[:, None], n, axis=1))
    np.testing.assert_array_equal(ret, adv)


def check_gae_special_cases(seed=61, T=64, n=200):
    """lambda = 0: the one-step TD error r_t + gamma v_{t+1} - v_t; gamma =
    lambda = 1: the sum of the remaining rewards plus v_T minus v_t
    (telescoping); both in float64 within the FP32 rounding of the terms."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.normal(0.0, 1.0, (T, n)).astype(np.float32)
    v = rng.normal(0.0, 5.0, (T + 1, n)).astype(np.float32)
    adv, _ = oracle.gae(r, v, 0.97, 0.0)
    td = r.astype(np.float64) + 0.97 * v[1:].astype(np.float64) - v[:-1].astype(np.float64)
    assert np.abs(adv - td).max() <= 1e-5 * (1.0 + np.abs(td).max())
    adv, ret = oracle.gae(r, v, 1.0, 1.0)
    tail = np.cumsum(r[::-1].astype(np.float64), axis=0)[::-1]
    want = tail + v[T].astype(np.float64) - v[:-1].astype(np.float64)
    assert np.abs(adv - want).max() <= 4 * T * 2.0 ** -24 * (np.abs(r).sum(axis=0).max() + 2 * np.abs(v).max())
    np.testing.assert_array_equal(ret, (adv + v[:-1]).astype(np.float32))


def check_gae_fp64(seed=67, T=128, n=300, gamma=0.99, lam=0.95):
    """General gamma, lambda: within the FP32 error bound of the float64
    recursion."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.normal(0.3, 1.0, (T, n)).astype(np.float32)
    v = rng.normal(0.0, 3.0, (T + 1, n)).astype(np.float32)
    adv, ret = oracle.gae(r, v, gamma, lam)
    ref = _gae64(r, v, gamma, lam)
    scale = np.abs(r).max() + 2 * np.abs(v).max()
    assert np.abs(adv - ref).max() <= 8 * T * 2.0 ** -24 * scale / (1 - gamma * lam) + 1e-7
    np.testing.assert_array_equal(ret, (adv + v[:-1]).astype(np.float32))


# ---------------------------------------------------------------------------
# Tag (Section 4.2): runners (type 0) and chasers (type 1)
# ---------------------------------------------------------------------------
TAG_CASE = {
    # hand-derived; full circle of view, 8 sectors, d_v 5, d_r 0.5, P 1, every
    # agent heading along +x, so a neighbour straight ahead is in sector 4 and
    # one straight behind in sector 0 (the full-circle sectors start behind)
    "state": [[50.0, 50.0, 0.0, 0.5],    # A runner
              [50.5, 50.0, 0.0, 0.5],    # B runner: touches A (0.5)
              [51.25, 50.0, 0.0, 0.5],   # C chaser: touches B (0.75), A at 1.25
              [51.75, 50.0, 0.0, 0.5],   # D chaser: touches C (0.5), B at 1.25, A at 1.75
              [46.0, 50.0, 0.0, 0.5]],   # E runner: A at 4, B at 4.5 (ramp 0.25, 0.125)
    "types": [0, 0, 1, 1, 0],
    # runner: -1 per touch, ramp from runners only; chaser: +1 per touched runner
    "reward": [-1.0 + 0.25, -2.0 + 0.125, 1.0, 0.0, 0.25 + 0.125],
    "coll": [1, 2, 2, 1, 0],
    # (agent, channel, sector, distance); every other entry is d_v
    "view": [(0, 0, 4, 0.5), (0, 1, 4, 1.25), (0, 0, 0, 4.0),
             (1, 0, 0, 0.5), (1, 1, 4, 0.75),
             (2, 0, 0, 0.75), (2, 1, 4, 0.5),
             (3, 0, 0, 1.25), (3, 1, 0, 0.5),
             (4, 0, 4, 4.0)],
}


def check_tag_hand_worked():
    p = fi.default_params(100.0, fov=fi.FULL_FOV)
    st = np.array(TAG_CASE["state"], np.float32)
    ty = np.array(TAG_CASE["types"], np.uint8)
    _, obs, rew, coll, flags = oracle.step_tag(p, st, ty, None)
    assert flags == 0
    np.testing.assert_array_equal(rew, np.array(TAG_CASE["reward"], np.float32))
    np.testing.assert_array_equal(coll, np.array(TAG_CASE["coll"], np.int32))
    want = np.full((5, 16), 5.0, np.float32)
    for i, ch, k, dist in TAG_CASE["view"]:
        want[i, 8 * ch + k] = dist
    np.testing.assert_array_equal(obs, want)


def check_tag_all_runners_is_flock(seed=81, n=700):
    """With no chasers the tag update is the flock update: the runner channel
    holds the flock's distances, the chaser channel is empty, rewards and
    collisions are the flock's."""
    side = fi.side_for(n)
    p = fi.default_params(side, num_segments=16)
    st = fi.initial_state(n, side, seed)
    _, o_t, r_t, c_t, _ = oracle.step_tag(p, st, np.zeros(n, np.uint8), None)
    _, o_f, r_f, c_f, _ = oracle.step_cont(p, st, None, layout=1)
    np.testing.assert_array_equal(o_t[:, :16], o_f[:, :16])
    assert np.all(o_t[:, 16:] == np.float32(p["view_radius"]))
    np.testing.assert_array_equal(r_t, r_f)
    np.testing.assert_array_equal(c_t, c_f)


def check_tag_channels_swap(seed=83, n=600):
    """Swapping every type swaps the two colour channels of every view."""
    side = fi.side_for(n)
    p = fi.default_params(side, num_segments=8)
    st = fi.initial_state(n, side, seed)
    ty = fi.tag_types(n, seed)
    _, o1, _, c1, _ = oracle.step_tag(p, st, ty, None)
    _, o2, _, c2, _ = oracle.step_tag(p, st, (1 - ty).astype(np.uint8), None)
    np.testing.assert_array_equal(o1[:, :8], o2[:, 8:])
    np.testing.assert_array_equal(o1[:, 8:], o2[:, :8])
    np.testing.assert_array_equal(c1, c2)


def check_tag_motion():
    """The tag action sets the speed (clamped) and turns the heading:
    float64 closed form of one move."""
    p = fi.default_params(100.0)
    for st0, act in (((50.0, 50.0, 1.0, 0.5), (0.8, 0.2)), ((20.0, 30.0, 3.0, 0.9), (1.7, -0.5))):
        st = np.array([st0], np.float32)
        s2, _, _, _, f = oracle.step_tag(p, st, np.zeros(1, np.uint8),
                                         np.array([act], np.float32))
        assert f == 0
        s = min(max(act[0], 0.0), 1.0)
        rot = max(-float(np.float32(p["turn_step"])), min(float(np.float32(p["turn_step"])), act[1]))
        th = float(np.float32(np.float32(st0[2]) + np.float32(rot)))
        assert float(s2[0, 3]) == float(np.float32(s)) and float(s2[0, 2]) == th
        assert abs(float(s2[0, 0]) - (st0[0] + s * math.cos(th))) < 3e-5
        assert abs(float(s2[0, 1]) - (st0[1] + s * math.sin(th))) < 3e-5


def fraction_to_f32(q):
    """The float32 nearest to the rational q (ties to even), by integer
    arithmetic on the exact value: no intermediate float64 rounding."""
    from fractions import Fraction
    q = Fraction(q)
    if q == 0:
        return np.float32(0.0)
    sign = -1.0 if q < 0 else 1.0
    a = abs(q)
    # e with 2^e <= a < 2^(e+1)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)  # subnormal range keeps the exponent of the smallest normal
    scaled = a * Fraction(2) ** (23 - e)  # the 24-bit significand, as a rational
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return np.float32(sign * math.ldexp(m, e - 23))  # exact: m <= 2^24


def exact_rewards(p, st):
    """Rewards of Eq. 1 (Fig. 4 shape, reading 2) for the agents of state st,
    summed exactly: each pair's FP32 term computed with numpy float32 (one
    rounding per operation, the specified formulas), then the terms of an
    agent added as exact rationals (fractions.Fraction) and the sum rounded
    once to float32.  Independent of the oracle's fixed-point accumulator."""
    from fractions import Fraction
    f = np.float32
    L = f(p["side"])
    HL = f(f(0.5) * L)
    rv = f(p["view_radius"])
    dr = f(p["agent_radius"])
    RV2 = f(rv * rv)
    two_dr = f(f(2.0) * dr)
    RC2 = f(two_dr * two_dr)
    inv_span = f(1.0 / (float(rv) - 2.0 * float(dr)))
    P = f(p["collision_penalty"])
    x = st[:, 0].astype(np.float32)
    y = st[:, 1].astype(np.float32)
    n = st.shape[0]
    out = np.zeros(n, np.float32)
    for i in range(n):
        dx = (x - x[i]).astype(np.float32)
        dy = (y - y[i]).astype(np.float32)
        dx = np.where(dx > HL, dx - L, np.where(dx < -HL, dx + L, dx)).astype(np.float32)
        dy = np.where(dy > HL, dy - L, np.where(dy < -HL, dy + L, dy)).astype(np.float32)
        d2 = (dx * dx + dy * dy).astype(np.float32)
        inr = d2 < RV2
        inr[i] = False
        coll = inr & (d2 < RC2)
        ramp = inr & ~coll
        t = ((rv - np.sqrt(d2[ramp])).astype(np.float32) * inv_span).astype(np.float32)
        s = sum((Fraction(float(v)) for v in t), Fraction(0))
        s -= int(coll.sum()) * Fraction(float(P))
        out[i] = fraction_to_f32(s)
    return out


def check_exact_reward_sum(over, n=360, side=40.0, seed=91):
    """The oracle's rewards equal the exact sums of exact_rewards bit for bit
    (reading 15: the exact sum of the FP32 terms, rounded once).  A
    fixed-point resolution 2^-K too coarse for some term, a truncated term or
    a penalty off the grid breaks the equality.  Returns the oracle's K."""
    p = fi.default_params(side, **over)
    st = fi.initial_state(n, side, seed)
    st2, obs, rew, coll, flags = oracle.step(p, st, None)
    assert flags == 0
    ref = exact_rewards(p, st2)
    bad = np.flatnonzero(rew.view(np.uint32) != ref.view(np.uint32))
    assert bad.size == 0, (over, bad[:5], rew[bad[:5]], ref[bad[:5]])
    # the case has terms of both kinds and cancellations near zero
    assert (coll > 0).any() or float(p["agent_radius"]) == 0.0
    return oracle.derive(p)["K"]


def edge_pairs_state(p, pairs=24):
    """Isolated pairs of agents whose distance is just below the view radius:
    pair j has one agent at x = 0 and the other at x = d_j = d_v - (j + 1)
    ulp(d_v) (a float32, so the offset is exactly d_j), in a row of its own,
    rows 3 d_v apart.  Each agent's reward is then one of the smallest ramp
    terms, those whose last bits set the fixed-point resolution."""
    f = np.float32
    rv = f(p["view_radius"])
    L = float(f(p["side"]))
    gap = 3.0 * float(rv)
    assert pairs * gap < L
    st = []
    d = rv
    for j in range(pairs):
        d = np.nextafter(d, f(0.0))
        y0 = f(gap * j + 0.5)
        st.append([0.0, y0, 0.0, 0.5])
        st.append([d, y0, 0.0, 0.5])
    return np.array(st, np.float32)


def smallest_term(p):
    """The ramp term of a neighbour at the largest float32 distance below d_v
    (FP32, the specified formula): the smallest term the sum can receive."""
    f = np.float32
    rv = f(p["view_radius"])
    dr = f(p["agent_radius"])
    inv_span = f(1.0 / (float(rv) - 2.0 * float(dr)))
    return f(f(rv - np.nextafter(rv, f(0.0))) * inv_span)


def odd_smallest_term_radius(lo=2.0, hi=9.0, step=0.1):
    """The first view radius in [lo, hi) (agent radius 0.5) whose smallest
    ramp term has an odd 24-bit significand: for it the resolution must be
    exactly fine enough for that last bit."""
    for k in range(int(round((hi - lo) / step))):
        rv = round(lo + k * step, 6)
        t = smallest_term({"view_radius": rv, "agent_radius": 0.5})
        if t.view(np.uint32) & 1:
            return rv
    raise AssertionError("no radius with an odd smallest term")


def check_exact_reward_edge_pairs(over, side=None):
    """The smallest ramp terms (pairs just inside the view radius) summed by
    the oracle equal their exact values: each agent's reward is its pair's
    term, bit for bit (a fixed-point resolution one bit too coarse truncates
    them).  Checked against exact_rewards."""
    rv = float(over.get("view_radius", 5.0))
    p = fi.default_params(side or max(200.0, 80.0 * rv), **over)
    st = edge_pairs_state(p)
    st2, obs, rew, coll, flags = oracle.step(p, st, None)
    assert flags == 0
    ref = exact_rewards(p, st2)
    # float32 positions round some offsets onto the range edge (no term)
    assert (ref > 0).mean() >= 0.5 and np.all(coll == 0)
    np.testing.assert_array_equal(rew.view(np.uint32), ref.view(np.uint32), err_msg=str(over))
