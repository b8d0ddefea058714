"""GPU tests of the step with the fused policy (BF16 MLP on the tensor cores).

* the environment part is unchanged: observations (when requested), rewards
  and collisions equal those of env_step bit for bit, and a trajectory driven
  by the policy's own actions stays bit-exact with the oracle;
* the logits are checked against a float64 restatement of the same network
  (oracle/fp64.py) on the same observations: the largest absolute error is
  reported and must stay below LOGIT_TOL, and the greedy action must agree
  wherever the float64 margin between the best and second logit exceeds
  2 * LOGIT_TOL.

LOGIT_TOL: the BF16 rounding of the inputs and of both hidden activations
(relative 2^-9 each) and the hardware tanh (relative about 2^-11), carried
through layers whose weights are N(0, 0.1), give errors of order 1e-2 for
observations of this size (4.3e-3 measured at 100,000 agents); 0.02 leaves
room for the heavy tail."""
import numpy as np
import pytest

import flock_inputs as fi
import fp64
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402

DEV = torch.device("cuda:0")
LOGIT_TOL = 0.02


def weights_dev(seed=0):
    w = fi.policy_weights(seed)
    blob = torch.from_numpy(w["blob"].view(np.int16)).to(DEV)
    return w, blob


@pytest.mark.parametrize("n,stencil", [(5000, 1), (100000, 1), (20000, 2)])
def test_policy_step_env_part_and_logits(n, stencil):
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 21)
    a0 = fi.random_actions(n, 1, 21)[0]
    w, blob = weights_dev(1)

    ref = F.FlockEnv(p, n, device=DEV, tuning={"stencil": stencil})
    ref.reset(torch.from_numpy(st0).to(DEV))
    o_ref, r_ref, c_ref = ref.step(torch.from_numpy(a0).to(DEV))

    env = F.FlockEnv(p, n, device=DEV, tuning={"stencil": stencil})
    env.reset(torch.from_numpy(st0).to(DEV))
    act = torch.from_numpy(a0).to(DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    logits = torch.empty((n, 9), dtype=torch.float32, device=DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    F.env_step_policy(env.env, blob, act, rew, coll, logits, obs)
    torch.cuda.synchronize()
    assert torch.equal(obs, o_ref) and torch.equal(rew, r_ref) and torch.equal(coll, c_ref)
    assert torch.equal(env.state(), ref.state())

    lg = logits.cpu().numpy().astype(np.float64)
    ref64 = fp64.mlp_forward(w, obs.cpu().numpy())
    err = np.abs(lg - ref64).max()
    print("n=%d max |logit - fp64| = %.3e" % (n, err))
    assert err < LOGIT_TOL
    greedy = act.cpu().numpy()
    assert np.array_equal(greedy, np.argmax(lg, axis=1))  # argmax of its own logits
    srt = np.sort(ref64, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    sure = margin > 2 * LOGIT_TOL
    assert sure.mean() > 0.5
    assert np.array_equal(greedy[sure], fp64.greedy(ref64)[sure])
    assert env.error() == 0
    env.close()
    ref.close()


def test_policy_drives_a_bit_exact_trajectory():
    """Five steps where the policy picks every next action; the oracle replays
    the same actions and must reach the same states and observations."""
    n = 3000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st = fi.initial_state(n, side, 5)
    w, blob = weights_dev(2)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st).to(DEV))
    act = torch.from_numpy(fi.random_actions(n, 1, 5)[0]).to(DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    for _ in range(5):
        a_in = act.cpu().numpy().copy()
        F.env_step_policy(env.env, blob, act, rew, coll, None, obs)
        st, o, r, c, _ = oracle.step(p, st, a_in)
        torch.cuda.synchronize()
        assert np.array_equal(obs.cpu().numpy(), o)
        assert np.array_equal(rew.cpu().numpy(), r)
        assert np.array_equal(env.state().cpu().numpy(), st)
    assert env.error() == 0
    env.close()


def test_policy_needs_eight_segments():
    p = fi.default_params(100.0, num_segments=5)
    env = F.FlockEnv(p, 10, device=DEV)
    _, blob = weights_dev()
    z = torch.zeros(10, dtype=torch.int32, device=DEV)
    r = torch.zeros(10, dtype=torch.float32, device=DEV)
    with pytest.raises(F.FlockError):
        F.env_step_policy(env.env, blob, z, r, z.clone())
    env.close()


def test_policy_rows_from_every_kernel_form():
    """Every flock form of the neighbour scan hands the network the same BF16
    rows: with 1, 2, 4 and 32 lanes per agent (32 uses the generic-sector
    kernel) and with the tile form requested, the policy step gives the same
    logits and actions, bit for bit."""
    n = 3000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 9)
    a0 = fi.random_actions(n, 1, 9)[0]
    _, blob = weights_dev(3)
    outs = []
    for tuning in ({"lanes": 1}, {"lanes": 2}, {"lanes": 4}, {"lanes": 32}, {"mode": 1}, None):
        env = F.FlockEnv(p, n, device=DEV, tuning=tuning)
        env.reset(torch.from_numpy(st0).to(DEV))
        act = torch.from_numpy(a0).to(DEV)
        rew = torch.empty(n, dtype=torch.float32, device=DEV)
        coll = torch.empty(n, dtype=torch.int32, device=DEV)
        logits = torch.empty((n, 9), dtype=torch.float32, device=DEV)
        F.env_step_policy(env.env, blob, act, rew, coll, logits)
        torch.cuda.synchronize()
        assert env.error() == 0, tuning
        outs.append((tuning, logits.cpu().numpy(), act.cpu().numpy(), rew.cpu().numpy()))
        env.close()
    for tuning, lg, ac, rw in outs[1:]:
        assert np.array_equal(lg, outs[0][1]), tuning
        assert np.array_equal(ac, outs[0][2]), tuning
        assert np.array_equal(rw, outs[0][3]), tuning


def test_weights_changed_in_place_between_calls():
    """The step's graph keeps the weights pointer; the operand image is rebuilt
    from it at every call, so weights updated in place (a training step) are
    the ones the next call's network uses."""
    n = 4000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 13)
    env = F.FlockEnv(p, n, device=DEV)
    env.reset(torch.from_numpy(st0).to(DEV))
    w1, blob = weights_dev(4)
    w2, blob2 = weights_dev(5)
    act = torch.from_numpy(fi.random_actions(n, 1, 13)[0]).to(DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    logits = torch.empty((n, 9), dtype=torch.float32, device=DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    for w, src in ((w1, None), (w2, blob2)):
        if src is not None:
            blob.copy_(src)  # same pointer, new contents
        F.env_step_policy(env.env, blob, act, rew, coll, logits, obs)
        torch.cuda.synchronize()
        ref64 = fp64.mlp_forward(w, obs.cpu().numpy())
        assert np.abs(logits.cpu().numpy().astype(np.float64) - ref64).max() < LOGIT_TOL
    assert env.error() == 0
    env.close()
