"""GPU parity of the paper's own flock variant (Section 4.1, Section 5):
continuous (acceleration, rotation) actions, 128 sectors, a view distance of
a tenth of the side, and the view-only observation (128 distances and the
speed).  Everything bit-exact against the oracle's continuous step."""
import numpy as np
import pytest

import flock_inputs as fi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402

DEV = torch.device("cuda:0")


def run_cont(p, st0, acts, tuning=None):
    n = st0.shape[0]
    env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    env.reset(torch.from_numpy(st0).to(DEV))
    out = []
    for a in acts:
        obs, rew, coll = env.step_continuous(torch.from_numpy(np.ascontiguousarray(a)).to(DEV))
        out.append((env.state().cpu().numpy(), obs.cpu().numpy().copy(),
                    rew.cpu().numpy().copy(), coll.cpu().numpy().copy()))
    err = env.error()
    env.close()
    return out, err


def oracle_cont(p, st0, acts, layout):
    st = st0
    out, flags = [], 0
    for a in acts:
        st, o, r, c, f = oracle.step_cont(p, st, a, layout=layout, threads=0)
        flags |= f
        out.append((st, o, r, c))
    return out, flags


def same(g, o, tag):
    for t, (gs, os_) in enumerate(zip(g, o)):
        for k, name in enumerate(("state", "obs", "reward", "coll")):
            if not np.array_equal(gs[k], os_[k]):
                bad = np.argwhere(gs[k] != os_[k])
                raise AssertionError("%s step %d %s differs at %d places, first %s: %s vs %s" % (
                    tag, t, name, len(bad), bad[0], gs[k][tuple(bad[0])], os_[k][tuple(bad[0])]))


@pytest.mark.parametrize("tuning", [None, {"mode": 2, "lanes": 1}, {"mode": 2, "lanes": 4},
                                    {"mode": 2, "lanes": 32},
                                    {"mode": 2, "stencil": 2, "lanes": 32},
                                    {"mode": 2, "stencil": 2}, {"mode": 1}],
                         ids=lambda d: "default" if d is None else "-".join(
                             "%s%s" % kv for kv in d.items()))
def test_paper_variant_trajectory(tuning):
    """2,000 agents, view L/10 (about 63 neighbours each), 128 sectors,
    continuous actions with some outside the ranges, 6 steps."""
    n, steps = 2000, 6
    p = fi.paper_params(n)
    st0 = fi.initial_state(n, p["side"], 51)
    acts = fi.random_cont_actions(n, steps, 51, p["speed_step"], p["turn_step"])
    g, err = run_cont(p, st0, acts, tuning)
    o, flags = oracle_cont(p, st0, acts, 1)
    same(g, o, "paper variant %s" % tuning)
    assert err == flags == 0


def test_paper_variant_full_size():
    """The benchmark's configuration: 16,000 agents (side 400, view 40, about
    500 neighbours in range), 2 steps, every output bit-exact."""
    n, steps = 16000, 2
    p = fi.paper_params(n)
    st0 = fi.initial_state(n, p["side"], 52)
    acts = fi.random_cont_actions(n, steps, 52, p["speed_step"], p["turn_step"])
    g, err = run_cont(p, st0, acts)
    o, _ = oracle_cont(p, st0, acts, 1)
    same(g, o, "16k")
    assert err == 0


def test_wide_view_gets_a_warp_per_agent():
    """The library's default launch shape for the paper's flock (about 1,800
    candidates per agent) gives each agent a whole warp."""
    p = fi.paper_params(16000)
    env = F.FlockEnv(p, 16000, device=DEV)
    assert env.tuning()["lanes"] == 32
    env.close()
    p = fi.default_params(fi.side_for(50000))
    env = F.FlockEnv(p, 50000, device=DEV)
    assert env.tuning()["lanes"] in (1, 2, 4)
    env.close()


def test_continuous_with_discrete_values_equals_discrete_step():
    n = 3000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 53)
    a = fi.random_actions(n, 1, 53)[0]
    amax, tmax = np.float32(p["speed_step"]), np.float32(p["turn_step"])
    ca = np.stack([np.array([-amax, 0, amax], np.float32)[a % 3],
                   np.array([-tmax, 0, tmax], np.float32)[a // 3]], axis=1)
    e1 = F.FlockEnv(p, n, device=DEV)
    e1.reset(torch.from_numpy(st0).to(DEV))
    o1, r1, c1 = (t.clone() for t in e1.step(torch.from_numpy(a).to(DEV)))
    e2 = F.FlockEnv(p, n, device=DEV)
    e2.reset(torch.from_numpy(st0).to(DEV))
    o2, r2, c2 = e2.step_continuous(torch.from_numpy(np.ascontiguousarray(ca)).to(DEV))
    assert torch.equal(o1, o2) and torch.equal(r1, r2) and torch.equal(c1, c2)
    assert torch.equal(e1.state(), e2.state())
    # and the same graph serves both kinds of step, in either order
    o3, _, _ = e1.step_continuous(torch.from_numpy(np.ascontiguousarray(ca)).to(DEV))
    o4, _, _ = e2.step(torch.from_numpy(a).to(DEV))
    assert torch.equal(o3, o4)
    e1.close()
    e2.close()


def test_nonfinite_continuous_action_is_flagged():
    n = 500
    p = fi.paper_params(n)
    st0 = fi.initial_state(n, p["side"], 54)
    ca = np.zeros((1, n, 2), np.float32)
    ca[0, 5, 0] = np.nan
    ca[0, 9, 1] = -np.inf
    g, err = run_cont(p, st0, ca)
    o, flags = oracle_cont(p, st0, ca, 1)
    same(g, o, "nonfinite")
    assert err == flags == F.FLOCK_ERR_ACTION


def test_view_only_layout_in_a_batch():
    """Instances of the batched kernel may use the view-only layout; with
    discrete actions their rows are the distance columns and the speed of the
    (distance, count) layout."""
    sizes = [700, 1500, 300]
    params = [fi.default_params(fi.side_for(k), num_segments=16, obs_layout=1) for k in sizes]
    total = sum(sizes)
    cells = sum(F.flock_instance_cells(q) for q in params)
    b = F.FlockBatch(len(sizes), total, cells, 17, device=DEV)
    states = [torch.from_numpy(fi.initial_state(k, fi.side_for(k), 60 + i)).to(DEV)
              for i, k in enumerate(sizes)]
    host0 = [s.cpu().numpy() for s in states]
    b.set(params, sizes, states, reset=[0] * len(sizes))
    a = fi.random_actions(total, 1, 60)[0]
    obs, rew, coll = b.step(torch.from_numpy(a).to(DEV))
    obs = obs.cpu().numpy().reshape(total, 17)
    off = 0
    for q, k, st in zip(params, sizes, host0):
        q0 = dict(q, obs_layout=0)
        s2, o, r, c, f = oracle.step(q0, st, a[off:off + k], threads=0)
        assert np.array_equal(obs[off:off + k, :16], o[:, 0:32:2])
        assert np.array_equal(obs[off:off + k, 16], o[:, 32])
        assert np.array_equal(rew.cpu().numpy()[off:off + k], r)
        off += k
    assert b.error() == 0
    b.close()


@pytest.mark.parametrize("batch", [False, True])
def test_view_only_layout_with_eight_sectors(batch):
    """Layout 1 with v = 8 runs the generic-sector kernels (the eight-sector
    kernels write layout 0 only): rows equal the oracle's view-only rows."""
    n = 2500
    side = fi.side_for(n)
    p = fi.default_params(side, obs_layout=1)
    st0 = fi.initial_state(n, side, 57)
    a = fi.random_actions(n, 1, 57)[0]
    q0 = dict(p, obs_layout=0)
    s2, o, r, c, _ = oracle.step(q0, st0, a, threads=0)
    want = np.concatenate([o[:, 0:16:2], o[:, 16:17]], axis=1)
    if batch:
        b = F.FlockBatch(1, n, F.flock_instance_cells(p), 9, device=DEV)
        b.set([p], [n], [torch.from_numpy(st0).to(DEV)], reset=[0])
        obs, rew, coll = b.step(torch.from_numpy(a).to(DEV))
        err = b.error()
        b.close()
    else:
        env = F.FlockEnv(p, n, device=DEV)
        env.reset(torch.from_numpy(st0).to(DEV))
        obs, rew, coll = env.step(torch.from_numpy(a).to(DEV))
        err = env.error()
        env.close()
    assert obs.shape == (n, 9)
    assert np.array_equal(obs.cpu().numpy(), want)
    assert np.array_equal(rew.cpu().numpy(), r) and err == 0
