"""Continuous batching on the GPU: sessions join while others run, leave
when their episode ends (or when their client cancels), and every session's
result in the mix equals the same session run alone and the oracle's
(bit for bit: observations, rewards, collisions, and the session's state rows
of the server's arena after every step)."""
import numpy as np
import pytest

import flock_inputs as fi

oracle = pytest.importorskip("oracle")

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402
from paper_2207_03945_gb300 import serve  # noqa: E402

DEV = torch.device("cuda:0")


def actions_for(seed, step, n):
    return fi.random_actions(n, 1, seed * 1000 + step)[0]


@pytest.mark.parametrize("pipeline", [False, True])
def test_alone_equals_in_the_mix(pipeline):
    # (iteration it arrives at, agents, episode steps, seed)
    plan = [(0, 3000, 8, 1), (0, 700, 5, 2), (2, 5000, 6, 3), (3, 9000, 4, 4), (4, 150, 9, 5),
            (6, 2500, 3, 6)]
    # the budget holds the largest session (9,000 agents) but not it together
    # with the first ones: it has to wait until memory frees up
    p9 = F.flock_default_params(max(fi.side_for(9000), 12.0))
    budget = serve.session_bytes(9000, F.flock_instance_cells(p9)) + 2000
    rec = {}
    srv = None

    def on_step(s, obs, rew, coll):
        # pipelined, the arena rows may already hold the next issued step
        rows = None if pipeline else srv.arena[s.offset:s.offset + s.n].cpu().numpy().copy()
        rec.setdefault(s.sid, []).append((obs.cpu().numpy().copy(), rew.cpu().numpy().copy(),
                                          coll.cpu().numpy().copy(), rows))

    def action_fn(s, step, out):
        out.copy_(torch.from_numpy(actions_for(s.seed, step, s.n)))

    srv = serve.FlockServer(budget, state_fn=lambda s: fi.initial_state(s.n, s.params["side"],
                                                                         s.seed),
                            max_slots=8, arena_agents=40000, max_cells=40000, device=DEV,
                            action_fn=action_fn, pipeline=pipeline)
    srv.on_step = on_step
    sids = {}
    it = 0
    while it < 100:
        for (t, n, steps, seed) in plan:
            if t == it:
                s = srv.submit(n, steps, seed)
                assert s is not None
                sids[seed] = s
        stepped = srv.iteration()
        it += 1
        if stepped == 0 and not srv.sched.queue and it > 6:
            break
    srv.drain()
    st = srv.stats()
    assert st["sessions_finished"] == len(plan) and st["sessions_rejected"] == 0
    assert sids[4].t_admit > sids[3].t_admit  # admission waited for memory
    assert st["set_changes"] >= 4
    srv.close()

    # each session alone, same initial state and actions
    for (t, n, steps, seed) in plan:
        s = sids[seed]
        env = F.FlockEnv(s.params, n, device=DEV)
        got = rec[s.sid]
        assert len(got) == steps
        o, r, c = env.reset(torch.from_numpy(fi.initial_state(n, s.params["side"], seed)).to(DEV))
        assert np.array_equal(o.cpu().numpy(), got[0][0])
        for k in range(1, steps):
            # the server's step k applied the actions drawn for step k
            o, r, c = env.step(torch.from_numpy(actions_for(seed, k, n)).to(DEV))
            assert np.array_equal(o.cpu().numpy(), got[k][0]), (seed, k)
            assert np.array_equal(r.cpu().numpy(), got[k][1]), (seed, k)
            assert np.array_equal(c.cpu().numpy(), got[k][2]), (seed, k)
        env.close()
    # and against the oracle: the same session replayed from its initial
    # state with the same actions, step by step
    for (t, n, steps, seed) in plan:
        s = sids[seed]
        replay_against_oracle(s.params, fi.initial_state(n, s.params["side"], seed), seed,
                              rec[s.sid])


def replay_against_oracle(params, state0, seed, got):
    """got[k] = (obs, reward, coll, arena rows) the server recorded after its
    k-th step of a session (k = 0 observes the initial state)."""
    st = state0
    for k, (obs, rew, coll, rows) in enumerate(got):
        a = None if k == 0 else actions_for(seed, k, st.shape[0])
        st, o, r, c, flags = oracle.step(params, st, a, threads=0)
        assert flags == 0
        assert np.array_equal(obs, o), (seed, k)
        assert np.array_equal(rew, r), (seed, k)
        assert np.array_equal(coll, c), (seed, k)
        if rows is not None:
            assert np.array_equal(rows, st), (seed, k)


@pytest.mark.parametrize("pipeline", [False, True])
def test_cancelled_session_leaves_at_the_next_iteration(pipeline):
    """A client cancels its session mid-episode (from the step callback): the
    session takes no further step, its slot and arena rows are freed at the
    next iteration (a session waiting for them is admitted into the same
    rows), and every recorded step of every session, the cancelled one's
    included, equals the oracle's."""
    # (iteration it arrives at, agents, episode steps, seed)
    plan = [(0, 4000, 12, 11), (0, 1200, 6, 12), (1, 3500, 5, 13)]
    cancel_after = 3  # session 11 leaves after its third recorded step
    # room for two sessions at a time: the third waits for the cancellation
    p4 = F.flock_default_params(max(fi.side_for(4000), 12.0))
    budget = (serve.session_bytes(4000, F.flock_instance_cells(p4))
              + serve.session_bytes(1200, F.flock_instance_cells(
                  F.flock_default_params(max(fi.side_for(1200), 12.0)))) + 2000)
    rec = {}
    srv = None
    sids = {}

    def on_step(s, obs, rew, coll):
        rows = None if pipeline else srv.arena[s.offset:s.offset + s.n].cpu().numpy().copy()
        rec.setdefault(s.sid, []).append((obs.cpu().numpy().copy(), rew.cpu().numpy().copy(),
                                          coll.cpu().numpy().copy(), rows))
        if s.seed == 11 and len(rec[s.sid]) == cancel_after:
            srv.cancel(s)

    def action_fn(s, step, out):
        out.copy_(torch.from_numpy(actions_for(s.seed, step, s.n)))

    srv = serve.FlockServer(budget, state_fn=lambda s: fi.initial_state(s.n, s.params["side"],
                                                                         s.seed),
                            max_slots=2, arena_agents=5200, max_cells=40000, device=DEV,
                            action_fn=action_fn, pipeline=pipeline)
    srv.on_step = on_step
    offsets = {}
    for it in range(40):
        for (t, n, steps, seed) in plan:
            if t == it:
                s = srv.submit(n, steps, seed)
                assert s is not None
                sids[seed] = s
        stepped = srv.iteration()
        for s in srv.sched.active:
            offsets.setdefault(s.seed, s.offset)
        if stepped == 0 and not srv.sched.queue and it > 2:
            break
    srv.drain()
    st = srv.stats()
    assert st["sessions_cancelled"] == 1 and st["sessions_finished"] == 2
    assert len(rec[sids[11].sid]) == cancel_after
    assert sids[11].cancelled and not sids[12].cancelled and not sids[13].cancelled
    # session 13 waited for the cancelled session's slot and took its rows
    assert sids[13].t_admit >= sids[11].t_done
    assert offsets[13] == offsets[11]
    assert srv.batch.error() == 0
    srv.close()
    for (t, n, steps, seed) in plan:
        s = sids[seed]
        got = rec[s.sid]
        assert len(got) == (cancel_after if seed == 11 else steps)
        replay_against_oracle(s.params, fi.initial_state(n, s.params["side"], seed), seed, got)


def test_poisson_arrivals_short_run():
    arrivals = fi.session_stream(rate=200.0, duration=0.5, seed=3, n_lo=500, n_hi=20000,
                                 len_lo=5, len_hi=40)
    srv = serve.FlockServer(2 * 10 ** 9, state_fn=lambda s: fi.initial_state(
        s.n, s.params["side"], s.seed), max_slots=64, arena_agents=2_000_000,
        max_cells=2_000_000, device=DEV)
    st = srv.run(arrivals)
    assert st["sessions_finished"] == len(arrivals)
    assert st["step_latency_p99_ms"] is not None
    assert srv.batch.error() == 0
    srv.close()
