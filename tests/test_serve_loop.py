"""Host logic of FlockServer's iteration (no GPU): the batch is replaced by a
recorder, so the test checks what the server hands to the library -- which
sessions, at which arena rows, with which reset flags, how often the
descriptors are re-uploaded -- and its step accounting."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2207_03945_gb300 as F  # noqa: E402
from paper_2207_03945_gb300 import serve  # noqa: E402


class RecordingBatch:
    """Stand-in for FlockBatch: records set_rows calls and steps."""

    def __init__(self, max_instances, max_agents, max_cells, obs_dim, device=None, stream=None,
                 tuning=None):
        self.sets = []
        self.steps = []
        self.obs = torch.zeros((max_agents, obs_dim))
        self.reward = torch.zeros(max_agents)
        self.coll = torch.zeros(max_agents, dtype=torch.int32)
        self.offsets, self.n_total = [], 0

    def set_rows(self, params_c, n_agents, arena, rows, reset=None):
        self.sets.append((list(n_agents), list(rows), list(reset)))
        self.offsets = list(np.cumsum([0] + list(n_agents))[:-1])
        self.n_total = int(sum(n_agents))

    def step(self, actions):
        assert actions.shape[0] == self.n_total
        assert int(actions.min()) >= 0 and int(actions.max()) < 9
        self.steps.append(self.n_total)
        n = self.n_total
        return self.obs[:n], self.reward[:n], self.coll[:n]

    def error(self):
        return 0

    def close(self):
        pass


def make_server(monkeypatch, budget=10 ** 12, max_slots=8):
    monkeypatch.setattr(F, "FlockBatch", RecordingBatch)
    stream = types.SimpleNamespace(synchronize=lambda: None)
    return serve.FlockServer(budget, state_fn=lambda s: np.zeros((s.n, 4), np.float32),
                             max_slots=max_slots, arena_agents=100000, max_cells=100000,
                             device="cpu", stream=stream)


def test_every_session_steps_its_episode_once_per_iteration(monkeypatch):
    srv = make_server(monkeypatch)
    a = srv.submit(300, steps=3, seed=1)
    b = srv.submit(500, steps=5, seed=2)
    seen = []
    srv.on_step = lambda s, obs, rew, coll: seen.append((s.sid, obs.shape[0]))
    n_iter = 0
    while srv.sched.active or srv.sched.queue:
        srv.iteration()
        n_iter += 1
        assert n_iter < 50
    # five stepping iterations, then one that only retires b
    assert n_iter == 6 and srv.iterations == 5
    assert a.steps_done == 3 and b.steps_done == 5
    la, lb = srv.session_latencies(a), srv.session_latencies(b)
    assert len(la) == 3 and len(lb) == 5 and la == lb[:3] and all(x >= 0 for x in lb)
    st = srv.stats()
    assert st["step_latency_p50_ms"] is not None and st["agents_per_iteration"] == 3400 / 5
    assert srv.agent_steps == 3 * 300 + 5 * 500
    assert srv.batch.steps == [800, 800, 800, 500, 500]
    assert sorted(set(seen)) == [(a.sid, 300), (b.sid, 500)]
    assert srv.stats()["sessions_finished"] == 2


def test_descriptors_reset_then_cleared_and_not_re_uploaded_when_unchanged(monkeypatch):
    srv = make_server(monkeypatch)
    a = srv.submit(300, steps=4, seed=1)
    srv.iteration()            # admits a, uploads with reset
    srv.iteration()            # clears a's reset flag
    srv.iteration()            # nothing changed: no upload
    assert [s[2] for s in srv.batch.sets] == [[True], [False]]
    b = srv.submit(200, steps=2, seed=2)
    srv.iteration()            # admits b (reset), a keeps running
    srv.iteration()            # a retires after 4 steps; b's flag cleared
    sets = srv.batch.sets
    assert sets[2] == ([300, 200], [a.offset, b.offset], [False, True])
    assert sets[3] == ([200], [b.offset], [False])
    assert a.steps_done == 4 and b.steps_done == 2
    assert srv.set_changes == len(sets) == 4


def test_admission_waits_for_the_budget(monkeypatch):
    nbytes = serve.session_bytes(1000, 1000)
    srv = make_server(monkeypatch, budget=int(1.5 * nbytes))
    x = srv.submit(1000, steps=2, seed=1)
    y = srv.submit(1000, steps=2, seed=2)
    srv.iteration()
    assert [s.sid for s in srv.sched.active] == [x.sid] and y.steps_done == 0
    srv.iteration()
    srv.iteration()            # x retired, y admitted in its arena rows
    assert [s.sid for s in srv.sched.active] == [y.sid] and y.offset == x.offset
    assert y.steps_done == 1


def test_client_leaving_mid_episode(monkeypatch):
    """A client that disconnects during a step (from on_step): its session is
    not stepped again, its rows go to the next waiting session, the others
    run on; the descriptors are re-uploaded without it."""
    nbytes = serve.session_bytes(1000, 1000)
    srv = make_server(monkeypatch, budget=int(2.5 * nbytes))
    x = srv.submit(1000, steps=10, seed=1)
    y = srv.submit(1000, steps=3, seed=2)
    z = srv.submit(1000, steps=2, seed=3)     # waits for memory

    def on_step(s, obs, rew, coll):
        if s is x and s.steps_done == 1:      # x's client leaves after its second step
            srv.cancel(s)
    srv.on_step = on_step
    while srv.sched.active or srv.sched.queue:
        srv.iteration()
        assert srv.iterations < 20
    assert x.cancelled and x.steps_done == 2 and not y.cancelled and y.steps_done == 3
    assert z.steps_done == 2 and z.offset == x.offset   # admitted into x's rows
    st = srv.stats()
    assert st["sessions_cancelled"] == 1 and st["sessions_finished"] == 2
    assert all(x_ is not x for x_ in srv.sched.active)
    # the upload after the cancellation: y, then z in x's former rows, z resetting
    assert ([1000, 1000], [y.offset, z.offset], [False, True]) in srv.batch.sets
