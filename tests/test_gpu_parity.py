"""GPU parity: the CUDA library (through its C ABI) against the oracle.

Bit-exact for everything: the state along the trajectory, every observation
value, collision counts and rewards (the reward sum is evaluated exactly on
both sides, so the benchmark spec's 1e-5 relative allowance is not needed and the
tests use exact equality).  Inputs are the seeded workloads of
flock_inputs (uniform agents at density 0.1, random actions)."""
import math

import numpy as np
import pytest

import flock_inputs as fi
import oracle
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402

DEV = torch.device("cuda:0")


def gpu_run(p, st0, acts, tuning=None, check_state_each=True):
    """Reset, then len(acts) steps; returns per step (state, obs, reward, coll) and error bits."""
    n = st0.shape[0]
    env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    out = []
    obs, rew, coll = env.reset(torch.from_numpy(st0).to(DEV))
    out.append((env.state().cpu().numpy(), obs.cpu().numpy().copy(), rew.cpu().numpy().copy(),
                coll.cpu().numpy().copy()))
    for a in acts:
        obs, rew, coll = env.step(torch.from_numpy(np.ascontiguousarray(a)).to(DEV))
        st = env.state().cpu().numpy() if check_state_each else None
        out.append((st, obs.cpu().numpy().copy(), rew.cpu().numpy().copy(),
                    coll.cpu().numpy().copy()))
    err = env.error()
    tun = env.tuning()
    env.close()
    return out, err, tun


def oracle_run(p, st0, acts):
    out = []
    r = oracle.step(p, st0, None, threads=0)
    out.append(r[:4])
    st = r[0]
    flags = r[4]
    for a in acts:
        r = oracle.step(p, st, a, threads=0)
        st = r[0]
        flags |= r[4]
        out.append(r[:4])
    return out, flags


def assert_same(g, o, tag=""):
    for t, (gs, go) in enumerate(zip(g, o)):
        names = ("state", "obs", "reward", "coll")
        for k in range(4):
            if gs[k] is None:
                continue
            if not np.array_equal(gs[k], go[k]):
                bad = np.argwhere(gs[k] != go[k])
                raise AssertionError("%s step %d %s differs at %d places, first %s: gpu %s oracle %s"
                                     % (tag, t, names[k], len(bad), bad[0], gs[k][tuple(bad[0])],
                                        go[k][tuple(bad[0])]))


@pytest.mark.parametrize("path", pins.golden_cases(), ids=lambda s: s.rsplit("/", 1)[-1])
def test_golden_cases_on_gpu(path):
    import json
    fx = json.load(open(path))
    st = np.array(fx["state"], np.float32)
    acts = [np.array(fx["actions"], np.int32)]
    g, err, _ = gpu_run(fx["params"], st, acts)
    o, flags = oracle_run(fx["params"], st, acts)
    assert_same(g, o, fx["name"])
    assert err == flags == 0


def test_trajectory_1k_100_steps():
    """1,000 agents on a side of 100, 100 steps: every output of every step."""
    n, steps = 1000, 100
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 0)
    acts = fi.random_actions(n, steps, 0)
    g, err, _ = gpu_run(p, st0, acts)
    o, flags = oracle_run(p, st0, acts)
    assert_same(g, o, "1k")
    assert err == 0 and flags == 0


def test_trajectory_5k_20_steps():
    n, steps = 5000, 20
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 1)
    acts = fi.random_actions(n, steps, 1)
    g, err, _ = gpu_run(p, st0, acts)
    o, _ = oracle_run(p, st0, acts)
    assert_same(g, o, "5k")
    assert err == 0


@pytest.mark.parametrize("tuning", [{"mode": 1}, {"mode": 2}, {"mode": 2, "lanes": 2},
                                    {"mode": 2, "lanes": 4, "stencil": 2}],
                         ids=lambda d: "-".join("%s%s" % kv for kv in d.items()))
def test_50k_full_size_3_steps(tuning):
    """The benchmark's 50,000-agent configuration (side 707.1) in the launch
    shapes the autotuner picks from: three steps, all outputs, bit-exact."""
    n, steps = 50000, 3
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 2)
    acts = fi.random_actions(n, steps, 2)
    g, err, _ = gpu_run(p, st0, acts, tuning)
    o, _ = oracle_run(p, st0, acts)
    assert_same(g, o, "50k")
    assert err == 0


@pytest.mark.parametrize("over", [
    {"fov": fi.FULL_FOV},
    {"num_segments": 5},
    {"num_segments": 1, "fov": fi.FULL_FOV},
    {"num_segments": 32, "fov": 2.0},
    {"num_segments": 128, "fov": fi.FULL_FOV},
    {"agent_radius": 0.0},
    {"view_radius": 7.3, "collision_penalty": 0.375},
], ids=lambda d: ",".join("%s=%s" % kv for kv in d.items()))
def test_parameter_variants(over):
    n, steps = 3000, 4
    side = fi.side_for(n)
    p = fi.default_params(side, **over)
    st0 = fi.initial_state(n, side, 3)
    acts = fi.random_actions(n, steps, 3)
    g, _, _ = gpu_run(p, st0, acts)
    o, _ = oracle_run(p, st0, acts)
    assert_same(g, o, str(over))


@pytest.mark.parametrize("tuning", [
    {"mode": 1, "stencil": 1, "tile_w": 1, "tile_h": 1, "block": 64},
    {"mode": 1, "stencil": 1, "tile_w": 64, "tile_h": 8, "block": 512},
    {"mode": 1, "stencil": 1, "tile_w": 7, "tile_h": 3, "block": 96},
    {"mode": 1, "stencil": 2, "tile_w": 16, "tile_h": 4, "block": 128},
    {"mode": 1, "stencil": 2, "tile_w": 64, "tile_h": 1, "block": 256},
    {"mode": 2, "stencil": 1, "tile_w": 0, "tile_h": 0, "block": 64},
    {"mode": 2, "stencil": 1, "tile_w": 0, "tile_h": 0, "block": 512},
    {"mode": 2, "stencil": 2, "tile_w": 0, "tile_h": 0, "block": 128},
    {"mode": 2, "stencil": 2, "tile_w": 0, "tile_h": 0, "block": 256},
    {"mode": 2, "stencil": 1, "tile_w": 0, "tile_h": 0, "block": 64, "lanes": 2},
    {"mode": 2, "stencil": 1, "tile_w": 0, "tile_h": 0, "block": 512, "lanes": 4},
    {"mode": 2, "stencil": 2, "tile_w": 0, "tile_h": 0, "block": 128, "lanes": 4},
    {"mode": 2, "stencil": 2, "tile_w": 0, "tile_h": 0, "block": 256, "lanes": 2},
    {"mode": 2, "stencil": 1, "tile_w": 0, "tile_h": 0, "block": 128, "lanes": 32},
    {"mode": 2, "stencil": 2, "tile_w": 0, "tile_h": 0, "block": 64, "lanes": 32},
], ids=lambda d: "m%d-s%d-%dx%d-b%d-l%d" % (d["mode"], d["stencil"], d["tile_w"], d["tile_h"],
                                             d["block"], d.get("lanes", 1)))
def test_launch_shapes_are_bit_identical(tuning):
    """Every tuning the autotuner may pick gives the same bits."""
    n, steps = 4000, 3
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 4)
    acts = fi.random_actions(n, steps, 4)
    g, _, tun = gpu_run(p, st0, acts, tuning)
    assert tun["stencil"] == tuning["stencil"] and tun["mode"] == tuning["mode"]
    if "lanes" in tuning or tuning["mode"] == 1:
        assert tun["lanes"] == tuning.get("lanes", 1)
    o, _ = oracle_run(p, st0, acts)
    assert_same(g, o, str(tuning))


@pytest.mark.parametrize("mode", [1, 2, 4, 32])
@pytest.mark.parametrize("side,stencil", [(11.0, 1), (10.5, 1), (10.5, 2), (16.0, 1), (26.0, 2)])
def test_small_square_wraps_everywhere(side, stencil, mode):
    """mode 4 (32) here: the direct form (mode 2) with 4 (32) lanes per agent."""
    # squares only just wider than 2 d_v: one to five cells per axis, every
    # stencil wraps and some visit a cell twice under different shifts
    n, steps = 60, 10
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 5)
    acts = fi.random_actions(n, steps, 5)
    tun = ({"stencil": stencil, "mode": mode} if mode < 4 else
           {"stencil": stencil, "mode": 2, "lanes": mode})
    g, _, _ = gpu_run(p, st0, acts, tun)
    o, _ = oracle_run(p, st0, acts)
    assert_same(g, o, "side %g" % side)


@pytest.mark.parametrize("mode", [1, 2, 4, 32])
def test_dense_cluster_exceeds_shared_memory(mode):
    """6,000 agents packed into a 20 x 20 patch: in mode 1 tiles overflow the
    shared staging buffer and take the per-thread path; in mode 2 warps see
    hundreds of in-range neighbours per agent."""
    n = 6000
    rng = np.random.Generator(np.random.PCG64(6))
    st0 = fi.initial_state(n, 100.0, 6)
    st0[:, 0] = (40.0 + 20.0 * rng.random(n)).astype(np.float32)
    st0[:, 1] = (40.0 + 20.0 * rng.random(n)).astype(np.float32)
    p = fi.default_params(100.0)
    acts = fi.random_actions(n, 2, 6)
    tun = {"mode": mode} if mode < 4 else {"mode": 2, "lanes": mode}
    g, err, _ = gpu_run(p, st0, acts, tun)
    o, flags = oracle_run(p, st0, acts)
    assert_same(g, o, "cluster")
    assert err == flags == 0


def test_empty_and_tiny():
    for n in (0, 1, 2):
        p = fi.default_params(100.0)
        st0 = fi.initial_state(n, 100.0, 7)
        acts = fi.random_actions(n, 3, 7)
        g, err, _ = gpu_run(p, st0, acts)
        o, _ = oracle_run(p, st0, acts)
        assert_same(g, o, "n=%d" % n)
        assert err == 0


def test_invalid_actions_are_flagged_and_act_as_keep():
    n = 500
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 8)
    a = fi.random_actions(n, 1, 8)
    a[0, ::7] = 9
    a[0, ::11] = -3
    g, err, _ = gpu_run(p, st0, a)
    o, flags = oracle_run(p, st0, a)
    assert_same(g, o, "bad actions")
    assert err == F.FLOCK_ERR_ACTION == flags


def test_out_of_range_state_is_flagged():
    n = 100
    p = fi.default_params(100.0)
    st0 = fi.initial_state(n, 100.0, 9)
    st0[5, 3] = 2.0  # speed above speed_max
    _, err, _ = gpu_run(p, st0, [])
    assert err == F.FLOCK_ERR_STATE


def test_repeat_is_bitwise_deterministic():
    n = 20000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 10)
    acts = fi.random_actions(n, 3, 10)
    g1, _, _ = gpu_run(p, st0, acts)
    g2, _, _ = gpu_run(p, st0, acts)
    assert_same(g1, g2, "repeat")


def test_checkpoint_resume_is_identical():
    n = 3000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 11)
    acts = fi.random_actions(n, 6, 11)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st0).to(DEV))
    for a in acts[:3]:
        env.step(torch.from_numpy(a).to(DEV))
    ckpt = env.state().clone()
    for a in acts[3:]:
        obs, rew, coll = env.step(torch.from_numpy(a).to(DEV))
    ref = (obs.cpu().numpy().copy(), rew.cpu().numpy().copy(), env.state().cpu().numpy())
    env2 = F.FlockEnv(p, n, device=DEV)
    env2.set_state(ckpt)
    for a in acts[3:]:
        obs2, rew2, coll2 = env2.step(torch.from_numpy(a).to(DEV))
    assert np.array_equal(obs2.cpu().numpy(), ref[0])
    assert np.array_equal(rew2.cpu().numpy(), ref[1])
    assert np.array_equal(env2.state().cpu().numpy(), ref[2])
    env.close()
    env2.close()


@pytest.mark.parametrize("buffers", ["pinned", "pinned_offset", "pageable"])
def test_host_buffer_step_matches_device_step(buffers):
    """Host buffers: page-locked actions are read by the kernels in place
    (mapped host memory) and page-locked outputs written by the copy kernel
    (16-byte stores; 4-byte ones for buffers one element off a 16-byte
    boundary), captured with the step in one graph that is kept while the
    buffers are the same; pageable ones are copied in and out; the two host
    steps, then a device step, all match the oracle.  4,999 agents: no buffer
    is a whole number of 16-byte units."""
    n = 4999
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 12)
    acts = fi.random_actions(n, 3, 12)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st0).to(DEV))
    o, _ = oracle_run(p, st0, acts)
    k = 1 if buffers == "pinned_offset" else 0
    for t in range(2):
        # "pinned": the same buffers both times (the step's graph is kept);
        # "pinned_offset": new buffers each time (the graph is captured again)
        if buffers != "pageable" and (t == 0 or buffers == "pinned_offset"):
            obs_h = torch.empty(n * 18 + k, dtype=torch.float32).pin_memory()[k:].view(n, 18)
            rew_h = torch.empty(n + k, dtype=torch.float32).pin_memory()[k:]
            coll_h = torch.empty(n + k, dtype=torch.int32).pin_memory()[k:]
            act_h = torch.empty(n, dtype=torch.int32).pin_memory()
        if buffers != "pageable":
            act_h.copy_(torch.from_numpy(acts[t]))
            obs_h.fill_(-1.0)
            if t == 0:
                F.env_step_host(env.env, act_h, obs_h, rew_h, coll_h)
            else:  # the same call through buffers bound once
                F.env_step_host_bind(env.env, act_h, obs_h, rew_h, coll_h)()
            got = (obs_h.numpy(), rew_h.numpy(), coll_h.numpy())
        else:
            obs_n = np.zeros((n, 18), np.float32)
            rew_n = np.zeros(n, np.float32)
            coll_n = np.zeros(n, np.int32)
            F.env_step_host(env.env, np.ascontiguousarray(acts[t]), obs_n, rew_n, coll_n)
            got = (obs_n, rew_n, coll_n)
        assert np.array_equal(got[0], o[t + 1][1]), t
        assert np.array_equal(got[1], o[t + 1][2]), t
        assert np.array_equal(got[2], o[t + 1][3]), t
    obs, rew, coll = env.step(torch.from_numpy(acts[2]).to(DEV))
    assert np.array_equal(obs.cpu().numpy(), o[3][1])
    assert env.error() == 0
    env.close()


@pytest.mark.parametrize("n,tuning", [(20001, None), (20001, {"lanes": 1}), (20001, {"mode": 1}),
                                      (20001, {"lanes": 32}), (20001, {"stencil": 2}),
                                      (150001, {"lanes": 1}), (150001, {"lanes": 2})])
def test_host_buffer_step_forms_match_device_step(n, tuning):
    """The host-buffer step with page-locked buffers runs the neighbour scan
    in agent order and writes the outputs straight into the mapped buffers
    (3 x 3 cells, 4 lanes per agent up to 100,000 agents, else the tuning's
    1 or 2), or steps in the workspace and copies (32 lanes, 5 x 5 cells):
    either way the same bits as the device step, over three steps with the
    buffers kept (the graph reused).  20,001 and 150,001 agents: the last
    warp's block of rows is partial and of odd length."""
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 31)
    acts = fi.random_actions(n, 3, 31)
    dev_env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    host_env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    dev_env.reset(torch.from_numpy(st0).to(DEV))
    host_env.reset(torch.from_numpy(st0).to(DEV))
    obs_h = torch.empty((n, 18), dtype=torch.float32).pin_memory()
    rew_h = torch.empty(n, dtype=torch.float32).pin_memory()
    coll_h = torch.empty(n, dtype=torch.int32).pin_memory()
    act_h = torch.empty(n, dtype=torch.int32).pin_memory()
    step = F.env_step_host_bind(host_env.env, act_h, obs_h, rew_h, coll_h)
    for t in range(3):
        obs, rew, coll = dev_env.step(torch.from_numpy(acts[t]).to(DEV))
        act_h.copy_(torch.from_numpy(acts[t]))
        obs_h.fill_(-1.0)
        step()
        assert torch.equal(obs_h, obs.cpu()), (tuning, t)
        assert torch.equal(rew_h, rew.cpu()), (tuning, t)
        assert torch.equal(coll_h, coll.cpu()), (tuning, t)
        assert torch.equal(host_env.state(), dev_env.state()), (tuning, t)
    assert host_env.error() == 0 and dev_env.error() == 0
    dev_env.close()
    host_env.close()


def test_statistics_at_benchmark_density():
    """Sanity at 100,000 agents: mean in-range neighbours rho*pi*d_v^2 = 7.854,
    collisions rho*pi*(2 d_r)^2 = 0.314 (Poisson, well within 10 sigma)."""
    n = 100000
    side = fi.side_for(n)
    p = fi.default_params(side, fov=fi.FULL_FOV)
    st0 = fi.initial_state(n, side, 13)
    g, err, _ = gpu_run(p, st0, [])
    obs, coll = g[0][1], g[0][3]
    rho = n / float(np.float32(side)) ** 2
    lam = rho * math.pi * 25
    assert abs(obs[:, 1:16:2].sum(1).mean() - lam) < 10 * math.sqrt(lam / n)
    assert abs(coll.mean() - rho * math.pi) < 10 * math.sqrt(rho * math.pi / n)
    assert err == 0


def test_new_buffers_each_step_without_waiting():
    """Steps queued back to back, each with other action and output buffers
    (the step graph is updated in place while earlier steps may still run):
    the last two steps' outputs and the final state match the oracle."""
    n, steps = 3000, 8
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 11)
    acts = fi.random_actions(n, steps, 11)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st0).to(DEV))
    acts_d = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in acts]
    outs = [(torch.empty((n, env.obs_dim), dtype=torch.float32, device=DEV),
             torch.empty(n, dtype=torch.float32, device=DEV),
             torch.empty(n, dtype=torch.int32, device=DEV)) for _ in range(2)]
    torch.cuda.synchronize()
    for k in range(steps):
        F.env_step(env.env, acts_d[k], *outs[k % 2])
    torch.cuda.synchronize()
    o, _ = oracle_run(p, st0, acts)
    assert np.array_equal(env.state().cpu().numpy(), o[-1][0])
    for k in (steps - 2, steps - 1):
        obs, rew, coll = (t.cpu().numpy() for t in outs[k % 2])
        assert np.array_equal(obs, o[k + 1][1]) and np.array_equal(rew, o[k + 1][2])
        assert np.array_equal(coll, o[k + 1][3])
    assert env.error() == 0
    env.close()
