"""The FLOCK_DEBUG build (libflock_debug.so) on the GPU: the same kernels
with index checks on their scratch and output accesses, each failed check
latching FLOCK_ERR_BOUNDS instead of trapping.  Small cases of every launch
form (single environment: shared-memory tiles, the direct form with 1, 4 and
32 lanes per agent, both stencils, wrapping squares, a dense cluster, tag;
the policy step's scan with the network; the host-buffer step's agent-order
scan; the batch in all three forms; the allocation-free step) must give the
oracle's bits with no error bit latched."""
import numpy as np
import pytest

import flock_inputs as fi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402
from paper_2207_03945_gb300 import _abi  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture
def debug_lib():
    prev = _abi.use_library(_abi.DEBUG_LIB_PATH)
    try:
        yield
    finally:
        _abi.restore_library(prev)


def run_env(p, st0, acts, tuning):
    n = st0.shape[0]
    env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    out = [tuple(x.cpu().numpy().copy() for x in env.reset(torch.from_numpy(st0).to(DEV)))]
    for a in acts:
        out.append(tuple(x.cpu().numpy().copy() for x in env.step(torch.from_numpy(a).to(DEV))))
    state = env.state().cpu().numpy()
    err = env.error()
    env.close()
    return out, state, err


def oracle_run(p, st0, acts):
    st, o, r, c, _ = oracle.step(p, st0, None, threads=0)
    out = [(o, r, c)]
    for a in acts:
        st, o, r, c, _ = oracle.step(p, st, a, threads=0)
        out.append((o, r, c))
    return out, st


CASES = [
    ("tiles", 3000, None, {"mode": 1}),
    ("direct-l1", 3000, None, {"mode": 2, "lanes": 1}),
    ("direct-l4-5x5", 3000, None, {"mode": 2, "lanes": 4, "stencil": 2}),
    ("direct-l32", 3000, None, {"mode": 2, "lanes": 32}),
    ("wrapping-square", 60, 10.5, {"mode": 2, "lanes": 4}),
    ("generic-sectors", 2000, None, {"mode": 2, "lanes": 2}),
]


@pytest.mark.parametrize("name,n,side,tuning", CASES, ids=[c[0] for c in CASES])
def test_debug_build_single_environment(debug_lib, name, n, side, tuning):
    side = side or fi.side_for(n)
    over = {"num_segments": 5} if name == "generic-sectors" else {}
    p = fi.default_params(side, **over)
    st0 = fi.initial_state(n, side, 21)
    acts = fi.random_actions(n, 3, 21)
    got, state, err = run_env(p, st0, acts, tuning)
    ref, ref_state = oracle_run(p, st0, acts)
    assert err == 0, "latched bits %d" % err
    for t, (g, r) in enumerate(zip(got, ref)):
        for k in range(3):
            assert np.array_equal(g[k], r[k]), (name, t, k)
    assert np.array_equal(state, ref_state)


def test_debug_build_dense_cluster(debug_lib):
    n = 3000
    rng = np.random.Generator(np.random.PCG64(8))
    st0 = fi.initial_state(n, 100.0, 8)
    st0[:, 0] = (40.0 + 15.0 * rng.random(n)).astype(np.float32)
    st0[:, 1] = (40.0 + 15.0 * rng.random(n)).astype(np.float32)
    p = fi.default_params(100.0)
    acts = fi.random_actions(n, 1, 8)
    for tuning in ({"mode": 1}, {"mode": 2, "lanes": 1}, {"mode": 2, "lanes": 32}):
        got, _, err = run_env(p, st0, acts, tuning)
        ref, _ = oracle_run(p, st0, acts)
        assert err == 0, (tuning, err)
        for t, (g, r) in enumerate(zip(got, ref)):
            for k in range(3):
                assert np.array_equal(g[k], r[k]), (tuning, t, k)


def test_debug_build_tag(debug_lib):
    n = 2000
    p = fi.tag_params(n)
    st0 = fi.initial_state(n, p["side"], 23)
    ty = fi.tag_types(n, 23)
    acts = fi.tag_actions(n, 2, 23, p["speed_max"], p["turn_step"])
    for tuning in ({"mode": 2, "lanes": 4}, {"mode": 2, "lanes": 32}):
        env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
        env.set_types(torch.from_numpy(ty).to(DEV))
        env.reset(torch.from_numpy(st0).to(DEV))
        st = st0
        for a in acts:
            obs, rew, coll = env.step_continuous(torch.from_numpy(a).to(DEV))
            st, o, r, c, _ = oracle.step_tag(p, st, ty, a)
            assert np.array_equal(obs.cpu().numpy(), o) and np.array_equal(rew.cpu().numpy(), r)
            assert np.array_equal(coll.cpu().numpy(), c)
        assert env.error() == 0, tuning
        env.close()


@pytest.mark.parametrize("mode", [2, 3, 4])
def test_debug_build_batch(debug_lib, mode):
    sizes = [700, 0, 1, 2600, 45, 1900]
    params = [fi.default_params(max(fi.side_for(n), 12.0)) for n in sizes]
    tuning = {"mode": mode}
    cells = sum(F.flock_instance_cells(p, tuning) for p in params)
    b = F.FlockBatch(len(sizes), sum(sizes), cells, 18, device=DEV, tuning=tuning)
    host = [fi.initial_state(n, max(fi.side_for(n), 12.0), 30 + k) for k, n in enumerate(sizes)]
    states = [torch.from_numpy(h).to(DEV) for h in host]
    b.set(params, sizes, states, reset=[1] * len(sizes))
    b.step(torch.zeros(sum(sizes), dtype=torch.int32, device=DEV))
    a = fi.random_actions(sum(sizes), 1, 31)[0]
    obs, rew, coll = b.step(torch.from_numpy(a).to(DEV))
    torch.cuda.synchronize()
    for k, (p, n) in enumerate(zip(params, sizes)):
        off = b.offsets[k]
        _, o, r, c, _ = oracle.step(p, host[k], a[off:off + n])
        assert np.array_equal(obs[off:off + n].cpu().numpy(), o), (mode, k)
        assert np.array_equal(rew[off:off + n].cpu().numpy(), r), (mode, k)
    assert b.error() == 0
    b.close()


def test_debug_build_static_step(debug_lib):
    n = 2500
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 33)
    a = fi.random_actions(n, 1, 33)[0]
    state = torch.from_numpy(st0).to(DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    assert F.flock_step_static(p, state, torch.from_numpy(a).to(DEV), obs, rew, coll) == 0
    _, o, r, c, _ = oracle.step(p, st0, a, threads=0)
    assert np.array_equal(obs.cpu().numpy(), o) and np.array_equal(rew.cpu().numpy(), r)
    assert np.array_equal(coll.cpu().numpy(), c)


@pytest.mark.parametrize("lanes", [1, 2, 4, 32])
def test_debug_build_policy_step(debug_lib, lanes):
    """The policy step's scan with the network in its epilogue: the
    environment part gives the oracle's bits, the greedy actions are the
    argmax of the step's own logits, and no bit is latched."""
    n = 3000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 41)
    a0 = fi.random_actions(n, 1, 41)[0]
    w = fi.policy_weights(6)
    blob = torch.from_numpy(w["blob"].view(np.int16)).to(DEV)
    env = F.FlockEnv(p, n, device=DEV, tuning={"mode": 2, "lanes": lanes})
    env.reset(torch.from_numpy(st0).to(DEV))
    act = torch.from_numpy(a0).to(DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    logits = torch.empty((n, 9), dtype=torch.float32, device=DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    F.env_step_policy(env.env, blob, act, rew, coll, logits, obs)
    torch.cuda.synchronize()
    st, o, r, c, _ = oracle.step(p, st0, a0, threads=0)
    assert np.array_equal(obs.cpu().numpy(), o) and np.array_equal(rew.cpu().numpy(), r)
    assert np.array_equal(coll.cpu().numpy(), c)
    assert np.array_equal(env.state().cpu().numpy(), st)
    assert np.array_equal(act.cpu().numpy(), np.argmax(logits.cpu().numpy(), axis=1))
    assert env.error() == 0, "latched bits"
    env.close()


@pytest.mark.parametrize("n,tuning", [(3001, {"mode": 2, "lanes": 4}),
                                      (120001, {"mode": 2, "lanes": 1})])
def test_debug_build_host_step_agent_order(debug_lib, n, tuning):
    """The host-buffer step with page-locked buffers (the neighbour scan in
    agent order writing the mapped buffers): the oracle's bits, no bit
    latched.  3,001 agents with 4 lanes per agent; 120,001 with the tuning's
    one lane (past 100,000 agents the agent-order form keeps it)."""
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 43)
    a = fi.random_actions(n, 1, 43)[0]
    env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    env.reset(torch.from_numpy(st0).to(DEV))
    obs_h = torch.empty((n, 18), dtype=torch.float32).pin_memory()
    rew_h = torch.empty(n, dtype=torch.float32).pin_memory()
    coll_h = torch.empty(n, dtype=torch.int32).pin_memory()
    act_h = torch.from_numpy(a).pin_memory()
    F.env_step_host(env.env, act_h, obs_h, rew_h, coll_h)
    ref = F.FlockEnv(p, n, device=DEV, tuning=tuning)
    ref.reset(torch.from_numpy(st0).to(DEV))
    o, r, c = (x.cpu().numpy() for x in ref.step(torch.from_numpy(a).to(DEV)))
    if n <= 5000:  # small enough for the oracle too
        _, o2, r2, c2, _ = oracle.step(p, st0, a, threads=0)
        assert np.array_equal(o, o2) and np.array_equal(r, r2) and np.array_equal(c, c2)
    assert np.array_equal(obs_h.numpy(), o) and np.array_equal(rew_h.numpy(), r)
    assert np.array_equal(coll_h.numpy(), c)
    assert env.error() == 0 and ref.error() == 0, "latched bits"
    env.close()
    ref.close()
