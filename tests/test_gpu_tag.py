"""GPU parity of the tag environment (Section 4.2): runners and chasers, two
colour channels of sectors, type-dependent rewards; bit-exact against the
oracle's tag step (tests/pins.py pins that oracle by hand-derived values)."""
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


def tag_env(p, st0, types, tuning=None):
    env = F.FlockEnv(p, st0.shape[0], device=DEV, tuning=tuning)
    env.set_types(torch.from_numpy(types).to(DEV))
    obs, rew, coll = env.reset(torch.from_numpy(st0).to(DEV))
    return env, obs, rew, coll


def test_hand_worked_case_on_gpu():
    c = pins.TAG_CASE
    p = fi.default_params(100.0, fov=fi.FULL_FOV, kind=1)
    st = np.array(c["state"], np.float32)
    ty = np.array(c["types"], np.uint8)
    env, obs, rew, coll = tag_env(p, st, ty)
    _, o, r, cc, _ = oracle.step_tag(p, st, ty, None)
    assert np.array_equal(obs.cpu().numpy(), o)
    assert np.array_equal(rew.cpu().numpy(), np.array(c["reward"], np.float32))
    assert np.array_equal(coll.cpu().numpy(), np.array(c["coll"], np.int32))
    env.close()


@pytest.mark.parametrize("tuning", [None, {"mode": 2, "lanes": 1}, {"mode": 2, "lanes": 2},
                                    {"mode": 2, "stencil": 2, "lanes": 4},
                                    {"mode": 2, "lanes": 32}, {"mode": 2, "stencil": 2, "lanes": 32}],
                         ids=lambda d: "default" if d is None else "-".join(
                             "%s%s" % kv for kv in d.items()))
def test_tag_trajectory(tuning):
    n, steps = 3000, 6
    p = fi.tag_params(n)
    st0 = fi.initial_state(n, p["side"], 91)
    ty = fi.tag_types(n, 91)
    acts = fi.tag_actions(n, steps, 91, p["speed_max"], p["turn_step"])
    env, obs, rew, coll = tag_env(p, st0, ty, tuning)
    st, o, r, c, _ = oracle.step_tag(p, st0, ty, None)
    assert np.array_equal(obs.cpu().numpy(), o) and np.array_equal(rew.cpu().numpy(), r)
    for t in range(steps):
        obs, rew, coll = env.step_continuous(torch.from_numpy(acts[t]).to(DEV))
        st, o, r, c, f = oracle.step_tag(p, st, ty, acts[t])
        assert np.array_equal(env.state().cpu().numpy(), st), t
        assert np.array_equal(obs.cpu().numpy(), o), t
        assert np.array_equal(rew.cpu().numpy(), r), t
        assert np.array_equal(coll.cpu().numpy(), c), t
    assert env.error() == 0
    env.close()


def test_tag_full_size():
    """The paper's tag run size: 16,000 runners and 1,600 chasers (view a
    tenth of the side, 64 sectors per channel), 2 steps."""
    n = 17600
    p = fi.tag_params(n)
    st0 = fi.initial_state(n, p["side"], 92)
    ty = fi.tag_types(n, 92)
    acts = fi.tag_actions(n, 2, 92, p["speed_max"], p["turn_step"])
    env, _, _, _ = tag_env(p, st0, ty)
    st = st0
    for t in range(2):
        obs, rew, coll = env.step_continuous(torch.from_numpy(acts[t]).to(DEV))
        st, o, r, c, _ = oracle.step_tag(p, st, ty, acts[t])
        assert np.array_equal(obs.cpu().numpy(), o) and np.array_equal(rew.cpu().numpy(), r)
        assert np.array_equal(coll.cpu().numpy(), c)
    assert env.error() == 0
    env.close()


def test_tag_rejections():
    p = fi.tag_params(500)
    with pytest.raises(F.FlockError):  # tag needs the direct form
        F.FlockEnv(p, 500, device=DEV, tuning={"mode": 1})
    flock = F.FlockEnv(fi.default_params(100.0), 10, device=DEV)
    with pytest.raises(F.FlockError):  # types on a flock environment
        flock.set_types(torch.zeros(10, dtype=torch.uint8, device=DEV))
    flock.close()
    b = F.FlockBatch(2, 1000, 1000, 128, device=DEV)
    st = torch.from_numpy(fi.initial_state(500, p["side"], 1)).to(DEV)
    with pytest.raises(F.FlockError):  # the batch steps flock instances
        b.set([p], [500], [st])
    b.close()
