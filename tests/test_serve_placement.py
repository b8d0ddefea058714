"""Host-side placement of serving sessions across GPUs (serve.SessionPlacer,
serve.place_sessions): every session goes to exactly one rank, the work
(agents x steps) stays balanced, and the placement depends only on the
arrival stream, so ranks that compute it independently agree.  Then two
gloo ranks, each running a server (the batch replaced by the recorder of
test_serve_loop) on its share of one arrival stream: together they serve
every session once, for its whole episode."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2207_03945_gb300 import serve  # noqa: E402


def stream(n_sessions, seed, steps_lo=100, steps_hi=2001):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_sessions):
        n = int(round(math.exp(math.log(500) + rng.random() * (math.log(50000) - math.log(500)))))
        out.append((float(rng.random() * 5.0), n, int(rng.integers(steps_lo, steps_hi)), 10 ** 6 + k))
    return sorted(out)


@pytest.mark.parametrize("n_ranks", [1, 2, 3, 4, 8])
def test_placement_covers_and_balances(n_ranks):
    arr = stream(500, 3)
    ranks = serve.place_sessions(arr, n_ranks)
    assert len(ranks) == len(arr) and set(ranks) <= set(range(n_ranks))
    work = np.zeros(n_ranks)
    for (_t, n, steps, _s), r in zip(arr, ranks):
        work[r] += n * steps
    biggest = max(n * steps for (_t, n, steps, _s) in arr)
    assert work.max() - work.min() <= biggest   # greedy least-loaded bound
    assert serve.place_sessions(arr, n_ranks) == ranks  # deterministic


def test_placement_rejects_no_ranks():
    with pytest.raises(ValueError):
        serve.SessionPlacer(0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import types

    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2207_03945_gb300 as F
    from paper_2207_03945_gb300 import serve as sv
    from test_serve_loop import RecordingBatch
    F.FlockBatch = RecordingBatch
    arr = [(0.0, n, steps, seed) for (_t, n, steps, seed) in stream(24, 7, 3, 12)]
    mine = [a for a, r in zip(arr, sv.place_sessions(arr, world)) if r == rank]
    srv = sv.FlockServer(10 ** 12, state_fn=lambda s: np.zeros((s.n, 4), np.float32),
                         max_slots=64, arena_agents=2_000_000, max_cells=2_000_000,
                         device="cpu", stream=types.SimpleNamespace(synchronize=lambda: None))
    sessions = {}
    for (_t, n, steps, seed) in mine:
        sessions[seed] = (srv.submit(n, steps, seed), steps)
    while srv.sched.active or srv.sched.queue:
        srv.iteration()
    srv.drain()
    done = {seed: (s.steps_done, steps) for seed, (s, steps) in sessions.items()}
    out = [None] * world
    dist.all_gather_object(out, (rank, done, srv.agent_steps))
    if rank == 0:
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_serve_every_session_once():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    arr = stream(24, 7, 3, 12)
    seen = {}
    total = 0
    for rank, done, agent_steps in out:
        total += agent_steps
        for seed, (steps_done, steps) in done.items():
            assert seed not in seen, "a session served by two ranks"
            seen[seed] = rank
            assert steps_done == steps
    assert sorted(seen) == sorted(seed for (_t, _n, _s, seed) in arr)
    assert total == sum(n * steps for (_t, n, steps, _seed) in arr)
    assert set(seen.values()) == {0, 1}
