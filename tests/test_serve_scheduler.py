"""Host logic of the serving loop (no GPU): admission by device-memory
budget and slots, first-arrived-first-admitted order, arena ranges that are
reused after sessions leave, rejection of sessions that can never fit."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location(
    "flock_serve", os.path.join(ROOT, "paper_2207_03945_gb300", "serve.py"))
serve = importlib.util.module_from_spec(_spec)
sys.modules["flock_serve"] = serve  # dataclasses look their module up
_spec.loader.exec_module(serve)


def sess(sid, n, steps=3, cells=None):
    return serve.Session(sid, n, cells if cells is not None else max(1, n // 2), steps, sid, 0.0)


def test_budget_and_slots_bind_and_order_is_fifo():
    b = serve.session_bytes(1000, 500)
    sc = serve.SessionScheduler(budget_bytes=2 * b + 10, max_slots=3, arena_agents=10000,
                                max_cells=100000)
    for k in range(4):
        assert sc.submit(sess(k, 1000))
    adm = sc.admit(0.0)
    assert [s.sid for s in adm] == [0, 1]  # the budget holds two
    assert sc.used_bytes == 2 * b
    # nothing more until one leaves
    assert sc.admit(0.1) == []
    sc.active[0].steps_issued = 3
    assert [s.sid for s in sc.retire(0.2)] == [0]
    assert [s.sid for s in sc.admit(0.3)] == [2]
    assert sc.admitted == 3 and sc.rejected == 0 and len(sc.queue) == 1


def test_slots_limit():
    sc = serve.SessionScheduler(budget_bytes=10 ** 12, max_slots=2, arena_agents=10 ** 6,
                                max_cells=10 ** 6)
    for k in range(5):
        sc.submit(sess(k, 10))
    assert len(sc.admit(0.0)) == 2


def test_never_fitting_sessions_are_rejected():
    sc = serve.SessionScheduler(budget_bytes=serve.session_bytes(100, 50), max_slots=4,
                                arena_agents=1000, max_cells=1000, queue_limit=2)
    assert not sc.submit(sess(0, 101))             # over the budget alone
    assert not sc.submit(sess(1, 50, cells=2000))  # over the cell capacity
    assert sc.submit(sess(2, 10)) and sc.submit(sess(3, 10))
    assert not sc.submit(sess(4, 10))              # queue full
    assert sc.rejected == 3


def test_arena_ranges_are_disjoint_and_reused():
    sc = serve.SessionScheduler(budget_bytes=10 ** 12, max_slots=16, arena_agents=1000,
                                max_cells=10 ** 6)
    for k, n in enumerate([300, 200, 400]):
        sc.submit(sess(k, n))
    sc.admit(0.0)
    ranges = sorted((s.offset, s.offset + s.n) for s in sc.active)
    assert all(a[1] <= b[0] for a, b in zip(ranges, ranges[1:]))
    assert ranges[-1][1] <= 1000
    # the middle one leaves; a session of 250 does not fit in the 200 hole
    # nor the 100 tail, one of 150 fits into the hole
    sc.active[1].steps_issued = 99
    sc.retire(1.0)
    sc.submit(sess(9, 250))
    assert sc.admit(1.1) == []
    sc.queue.clear()
    sc.submit(sess(10, 150))
    got = sc.admit(1.2)
    assert got and got[0].offset == 300
    # everything leaves: the arena is one free range again
    for s in sc.active:
        s.steps_issued = 99
    sc.retire(2.0)
    assert sc.free == [(0, 1000)] and sc.used_bytes == 0 and sc.used_cells == 0


def test_random_workload_keeps_invariants():
    import random
    rnd = random.Random(7)
    sc = serve.SessionScheduler(budget_bytes=serve.session_bytes(5000, 3000), max_slots=8,
                                arena_agents=6000, max_cells=4000)
    for it in range(2000):
        if rnd.random() < 0.3:
            sc.submit(sess(it, rnd.randint(1, 3000), steps=rnd.randint(1, 20),
                           cells=rnd.randint(1, 1500)))
        sc.admit(it)
        for s in sc.active:
            s.steps_issued += 1
        sc.retire(it)
        ranges = sorted((s.offset, s.offset + s.n) for s in sc.active)
        assert all(a[1] <= b[0] for a, b in zip(ranges, ranges[1:]))
        assert sc.used_bytes <= sc.budget and len(sc.active) <= sc.max_slots
        assert sc.used_cells <= sc.max_cells
        free = sum(l for _, l in sc.free) + sum(s.n for s in sc.active)
        assert free == sc.arena_agents


def test_version_changes_with_the_active_set_only():
    """The server re-uploads instance descriptors only when the scheduler's
    version moved: admissions and retirements bump it, idle calls do not."""
    sc = serve.SessionScheduler(budget_bytes=10 ** 12, max_slots=4, arena_agents=10 ** 6,
                                max_cells=10 ** 6)
    v0 = sc.version
    assert sc.admit(0.0) == [] and sc.retire(0.0) == [] and sc.version == v0
    sc.submit(sess(0, 100, steps=2))
    sc.submit(sess(1, 100, steps=5))
    sc.admit(0.0)
    v1 = sc.version
    assert v1 != v0
    for s in sc.active:
        s.steps_issued += 1
    assert sc.retire(0.1) == [] and sc.admit(0.1) == [] and sc.version == v1
    for s in sc.active:
        s.steps_issued += 1
    assert [s.sid for s in sc.retire(0.2)] == [0] and sc.version != v1


def test_cancel_waiting_and_running_sessions():
    """A client that leaves: a waiting session leaves the queue; a running
    one frees its slot, memory and arena rows at once, so the next waiting
    session is admitted into them; unknown or finished sessions are refused."""
    b = serve.session_bytes(1000, 500)
    sc = serve.SessionScheduler(budget_bytes=b + 10, max_slots=4, arena_agents=10000,
                                max_cells=100000)
    ss = [sess(k, 1000, steps=5) for k in range(3)]
    for s in ss:
        assert sc.submit(s)
    assert [s.sid for s in sc.admit(0.0)] == [0]  # the budget holds one
    assert sc.cancel(ss[2], 0.1) and [s.sid for s in sc.queue] == [1]
    v = sc.version
    assert sc.cancel(ss[0], 0.2)
    assert sc.version != v and sc.active == [] and sc.used_bytes == 0 and sc.used_cells == 0
    assert [s.sid for s in sc.admit(0.3)] == [1] and ss[1].offset == ss[0].offset
    assert not sc.cancel(ss[0], 0.4) and not sc.cancel(sess(9, 10), 0.4)
    assert [s.sid for s in sc.cancelled] == [2, 0] and all(s.cancelled for s in sc.cancelled)
    assert sc.finished == []
