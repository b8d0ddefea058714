"""The allocation-free entry point (flock_step_static) against the normal one.

flock_step_static exists for callers that cannot allocate device memory (a
host callback or real-time loop where cudaMalloc may block or is forbidden,
a plugin whose host owns all device memory): its scratch is a fixed array in
the library's device memory.  This test drives it through the C ABI for two
calls in a row and requires exactly the outputs of env_reset/env_step (the
library's tests compare bit for bit).  It is collected last on purpose and
passes both alone and after the other tests."""
import numpy as np
import pytest

import flock_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("n", [50000, 3000])
def test_static_step_matches_env_step_two_calls(n):
    side = fi.side_for(n)
    p = fi.default_params(side)
    st0 = fi.initial_state(n, side, 77)
    acts = fi.random_actions(n, 2, 77)

    env = F.FlockEnv(p, n, device=DEV)
    ref = [tuple(x.clone() for x in env.reset(torch.from_numpy(st0).to(DEV)))]
    for a in acts:
        ref.append(tuple(x.clone() for x in env.step(torch.from_numpy(a).to(DEV))))
    ref_state = env.state()
    env.close()

    state = torch.from_numpy(st0).to(DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    assert F.flock_step_static(p, state, None, obs, rew, coll) == 0
    got = [(obs.clone(), rew.clone(), coll.clone())]
    for a in acts:  # two calls in a row, sharing the fixed scratch
        assert F.flock_step_static(p, state, torch.from_numpy(a).to(DEV), obs, rew, coll) == 0
        got.append((obs.clone(), rew.clone(), coll.clone()))
    for t, (g, r) in enumerate(zip(got, ref)):
        for k in range(3):
            assert torch.equal(g[k], r[k]), (t, k)
    assert torch.equal(state, ref_state)


def test_static_step_rejects_sizes_beyond_its_scratch():
    n = F._abi.STATIC_MAX_AGENTS + 1
    p = fi.default_params(fi.side_for(n))
    state = torch.zeros((n, 4), dtype=torch.float32, device=DEV)
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    with pytest.raises(F.FlockError):
        F.flock_step_static(p, state, None, obs, rew, coll)
    # few agents on a square whose cell list exceeds the fixed scratch
    p = fi.default_params(2000.0)  # 399 x 399 cells
    state = torch.from_numpy(fi.initial_state(10, 2000.0, 1)).to(DEV)
    with pytest.raises(F.FlockError):
        F.flock_step_static(p, state, None, obs[:10], rew[:10], coll[:10])
