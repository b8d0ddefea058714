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


def test_static_step_view_only_layout_matches_env_step_and_oracle():
    """The paper's view-only observation (obs_layout 1, v + 1 values per row)
    with eight sectors: rows of 9 floats, written by the generic-sector kernel
    (the eight-sector kernel writes (distance, count) pairs only).  Compared
    bit for bit with env_reset/env_step of the same layout and with the
    oracle (discrete actions applied, then the view-only observation)."""
    oracle = pytest.importorskip("oracle")
    n = 3000
    side = fi.side_for(n)
    p = dict(fi.default_params(side), obs_layout=1)
    assert p["num_segments"] == 8 and F.flock_obs_dim(p) == 9
    st0 = fi.initial_state(n, side, 5)
    acts = fi.random_actions(n, 2, 5)

    env = F.FlockEnv(p, n, device=DEV)
    ref = [tuple(x.clone() for x in env.reset(torch.from_numpy(st0).to(DEV)))]
    for a in acts:
        ref.append(tuple(x.clone() for x in env.step(torch.from_numpy(a).to(DEV))))
    env.close()

    state = torch.from_numpy(st0).to(DEV)
    obs = torch.empty((n, 9), dtype=torch.float32, device=DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    st = st0
    for t in range(len(acts) + 1):
        a = None if t == 0 else acts[t - 1]
        assert F.flock_step_static(p, state, None if a is None else torch.from_numpy(a).to(DEV),
                                   obs, rew, coll) == 0
        if a is not None:
            st, _ = oracle.apply(p, st, a)
        o = oracle.step_cont(p, st, None, layout=1, threads=0)
        for k, g in enumerate((obs, rew, coll)):
            assert torch.equal(g, ref[t][k]), (t, k)
            assert np.array_equal(g.cpu().numpy(), o[k + 1]), (t, k)
        assert np.array_equal(state.cpu().numpy(), st), t


def test_static_step_refuses_a_stream_in_capture():
    """A call made while its stream is being captured returns FLOCK_EINVAL
    and enqueues nothing (the call copies from pageable host memory, which
    capture does not allow); the capture itself ends normally."""
    n = 1000
    p = fi.default_params(fi.side_for(n))
    state = torch.from_numpy(fi.initial_state(n, fi.side_for(n), 3)).to(DEV)
    before = state.clone()
    obs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    rew = torch.empty(n, dtype=torch.float32, device=DEV)
    coll = torch.empty(n, dtype=torch.int32, device=DEV)
    # the first call on this device (set-up) comes before any capture
    assert F.flock_step_static(p, state, None, obs, rew, coll) == 0
    s = torch.cuda.Stream(device=DEV)
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.stream(s):
        try:
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                try:
                    F.flock_step_static(p, state, None, obs, rew, coll, stream=s, wait=False)
                except F.FlockError as e:
                    code = e.code
                # give the capture one node so that it ends as a valid graph
                obs.add_(0.0)
        finally:
            torch.cuda.synchronize()
    assert code == F._abi.FLOCK_EINVAL
    assert torch.equal(state, before)
