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
                 tuning=None, out_buffers=1):
        self.sets = []
        self.steps = []
        self.bufs = []
        self.outs = [(torch.zeros((max_agents, obs_dim)), torch.zeros(max_agents),
                      torch.zeros(max_agents, dtype=torch.int32)) for _ in range(out_buffers)]
        self.offsets, self.n_total = [], 0

    def set_rows(self, params_c, n_agents, arena, rows, reset=None):
        self.sets.append((list(n_agents), list(rows), list(reset)))
        self.offsets = list(np.cumsum([0] + list(n_agents))[:-1])
        self.n_total = int(sum(n_agents))

    def step(self, actions, buf=0):
        assert actions.shape[0] == self.n_total
        assert int(actions.min()) >= 0 and int(actions.max()) < 9
        self.steps.append(self.n_total)
        self.bufs.append(buf)
        n = self.n_total
        obs, rew, coll = self.outs[buf]
        obs[:n] = len(self.steps)  # marks which step wrote the buffer
        return obs[:n], rew[:n], coll[:n]

    def error(self):
        return 0

    def close(self):
        pass


def make_server(monkeypatch, budget=10 ** 12, max_slots=8, pipeline=True):
    monkeypatch.setattr(F, "FlockBatch", RecordingBatch)
    stream = types.SimpleNamespace(synchronize=lambda: None)
    return serve.FlockServer(budget, state_fn=lambda s: np.zeros((s.n, 4), np.float32),
                             max_slots=max_slots, arena_agents=100000, max_cells=100000,
                             device="cpu", stream=stream, pipeline=pipeline)


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


@pytest.mark.parametrize("pipeline", [True, False])
def test_descriptors_uploaded_once_per_set_change(monkeypatch, pipeline):
    """A set change uploads the descriptors once: a new session's reset flag
    goes up with it and is cleared by the step that observes it (on the
    device, and in the host's copy when that step is issued), so no second
    upload follows."""
    srv = make_server(monkeypatch, pipeline=pipeline)
    a = srv.submit(300, steps=4, seed=1)
    srv.iteration()            # admits a, uploads with reset
    srv.iteration()            # nothing changed: no upload
    srv.iteration()
    assert [s[2] for s in srv.batch.sets] == [[True]]
    b = srv.submit(200, steps=2, seed=2)
    srv.iteration()            # admits b (reset), a issues its fourth step
    srv.iteration()            # a retired after 4 steps
    srv.drain()
    sets = srv.batch.sets
    assert sets[1] == ([300, 200], [a.offset, b.offset], [False, True])
    assert sets[2] == ([200], [b.offset], [False])
    assert a.steps_done == 4 and b.steps_done == 2
    assert srv.set_changes == len(sets) == 3


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
    assert y.steps_issued == 1


@pytest.mark.parametrize("pipeline", [True, False])
def test_client_leaving_mid_episode(monkeypatch, pipeline):
    """A client that disconnects during a step (from on_step): its session is
    not stepped again (pipelined, a step already issued has its results
    dropped), its rows go to the next waiting session, the others run on; the
    descriptors are re-uploaded without it."""
    nbytes = serve.session_bytes(1000, 1000)
    srv = make_server(monkeypatch, budget=int(2.5 * nbytes), pipeline=pipeline)
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
    assert x.steps_issued == (3 if pipeline else 2)
    if pipeline:
        # y's last step was issued with x's third: the upload after the
        # cancellation holds z alone, in x's former rows, resetting
        assert ([1000], [x.offset], [True]) in srv.batch.sets
    else:
        # the upload after the cancellation: y, then z in x's former rows
        assert ([1000, 1000], [y.offset, z.offset], [False, True]) in srv.batch.sets


def test_pipelined_results_arrive_one_iteration_later_from_alternating_buffers(monkeypatch):
    """Pipelined iterations: step i writes output buffer i % 2 and its results
    reach on_step during iteration i + 1 (after step i + 1 was issued, into the
    other buffer); drain() delivers the last one.  Without the pipeline every
    step is delivered in its own iteration from one buffer."""
    for pipeline in (True, False):
        srv = make_server(monkeypatch, pipeline=pipeline)
        a = srv.submit(100, steps=4, seed=1)
        got = []
        srv.on_step = lambda s, obs, rew, coll: got.append((srv.iterations, int(obs[0, 0])))
        for _ in range(4):
            srv.iteration()
        srv.drain()
        if pipeline:
            assert srv.batch.bufs == [0, 1, 0, 1]
            # (iterations issued when delivered, step that wrote the buffer)
            assert got == [(2, 1), (3, 2), (4, 3), (4, 4)]
        else:
            assert srv.batch.bufs == [0, 0, 0, 0]
            assert got == [(1, 1), (2, 2), (3, 3), (4, 4)]
        assert a.steps_done == 4 and a.steps_issued == 4


def test_device_tensor_initial_states(monkeypatch):
    """state_fn may return a tensor on the server's device: it is copied into
    the session's arena rows without staging (nothing waits on an upload
    event), and host arrays still go through the staging rows."""
    monkeypatch.setattr(F, "FlockBatch", RecordingBatch)
    stream = types.SimpleNamespace(synchronize=lambda: None)

    def state_fn(s):
        v = torch.full((s.n, 4), float(s.sid + 1))
        return v if s.sid % 2 == 0 else v.numpy()

    srv = serve.FlockServer(10 ** 12, state_fn=state_fn, max_slots=4, arena_agents=100000,
                            max_cells=100000, device="cpu", stream=stream)
    ss = [srv.submit(100 + 10 * k, steps=2, seed=k) for k in range(4)]
    srv.iteration()
    for s in ss:
        assert torch.equal(srv.arena[s.offset:s.offset + s.n], torch.full((s.n, 4), float(s.sid + 1)))
    while srv.sched.active or srv.sched.queue:
        srv.iteration()
    srv.close()
    assert all(s.steps_done == 2 for s in ss)
