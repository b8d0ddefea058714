"""GPU tests of the rollout (T steps in one graph launch) and of the
advantage kernel (generalised advantage estimation), against the oracle:
both bit-exact."""
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


def test_rollout_discrete_equals_oracle_trajectory():
    n, T = 3000, 16
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 71)
    acts = fi.random_actions(n, T, 71)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st0).to(DEV))
    obs, rew, coll = env.rollout(torch.from_numpy(acts).to(DEV))
    torch.cuda.synchronize()
    st = st0
    for t in range(T):
        st, o, r, c, _ = oracle.step(p, st, acts[t], threads=0)
        assert np.array_equal(obs[t].cpu().numpy(), o), t
        assert np.array_equal(rew[t].cpu().numpy(), r), t
        assert np.array_equal(coll[t].cpu().numpy(), c), t
    assert np.array_equal(env.state().cpu().numpy(), st)
    # a second rollout reuses the graph and continues from the new state
    obs2, rew2, _ = env.rollout(torch.from_numpy(acts[:4]).to(DEV))
    for t in range(4):
        st, o, r, c, _ = oracle.step(p, st, acts[t], threads=0)
        assert np.array_equal(obs2[t].cpu().numpy(), o)
    assert env.error() == 0
    env.close()


def test_rollout_continuous_paper_variant():
    n, T = 1500, 8
    p = fi.paper_params(n)
    st0 = fi.initial_state(n, p["side"], 72)
    acts = fi.random_cont_actions(n, T, 72, p["speed_step"], p["turn_step"])
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st0).to(DEV))
    obs, rew, coll = env.rollout(actions2=torch.from_numpy(acts).to(DEV))
    torch.cuda.synchronize()
    st = st0
    for t in range(T):
        st, o, r, c, _ = oracle.step_cont(p, st, acts[t], layout=1, threads=0)
        assert np.array_equal(obs[t].cpu().numpy(), o), t
        assert np.array_equal(rew[t].cpu().numpy(), r), t
    assert env.error() == 0
    env.close()


def test_rollout_argument_checks():
    p = fi.default_params(100.0)
    env = F.FlockEnv(p, 100, device=DEV)
    a = torch.zeros((2, 100), dtype=torch.int32, device=DEV)
    a2 = torch.zeros((2, 100, 2), dtype=torch.float32, device=DEV)
    obs = torch.empty((2, 100, 18), device=DEV)
    rew = torch.empty((2, 100), device=DEV)
    coll = torch.empty((2, 100), dtype=torch.int32, device=DEV)
    with pytest.raises(F.FlockError):  # both kinds of action
        F.env_rollout(env.env, a, obs, rew, coll, actions2=a2)
    F.env_rollout(env.env, a, obs, rew, coll)
    env.close()


@pytest.mark.parametrize("T,n,gamma,lam", [(128, 10000, 0.99, 0.95), (1, 37, 0.5, 1.0),
                                           (33, 1000, 1.0, 1.0), (64, 257, 0.9, 0.0),
                                           (0, 50, 0.99, 0.95), (16, 0, 0.99, 0.95)])
def test_gae_bit_exact(T, n, gamma, lam):
    rng = np.random.Generator(np.random.PCG64(T * 7 + n))
    r = rng.normal(0.2, 1.0, (T, n)).astype(np.float32)
    v = rng.normal(0.0, 3.0, (T + 1, n)).astype(np.float32)
    adv = torch.empty((T, n), device=DEV)
    ret = torch.empty((T, n), device=DEV)
    F.flock_gae(torch.from_numpy(r).to(DEV), torch.from_numpy(v).to(DEV), gamma, lam, adv, ret)
    torch.cuda.synchronize()
    if T and n:
        a0, r0 = oracle.gae(r, v, gamma, lam)
        assert np.array_equal(adv.cpu().numpy(), a0)
        assert np.array_equal(ret.cpu().numpy(), r0)


def test_gae_on_rollout_rewards():
    """The trajectory processing of one training step: rollout rewards,
    values from any critic (here seeded numbers), advantages on the GPU."""
    n, T = 2000, 32
    side = fi.side_for(n)
    p = fi.default_params(side)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(fi.initial_state(n, side, 73)).to(DEV))
    _, rew, _ = env.rollout(torch.from_numpy(fi.random_actions(n, T, 73)).to(DEV))
    v = torch.from_numpy(np.random.Generator(np.random.PCG64(74)).normal(
        0, 1, (T + 1, n)).astype(np.float32)).to(DEV)
    adv = torch.empty((T, n), device=DEV)
    ret = torch.empty((T, n), device=DEV)
    F.flock_gae(rew, v, 0.99, 0.95, adv, ret)
    a0, r0 = oracle.gae(rew.cpu().numpy(), v.cpu().numpy(), 0.99, 0.95)
    assert np.array_equal(adv.cpu().numpy(), a0) and np.array_equal(ret.cpu().numpy(), r0)
    env.close()
