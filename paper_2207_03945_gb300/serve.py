"""Serving loop with continuous batching for the flock environment.

Sessions (independent flock environments of different agent counts, the
environments of arXiv 2207.03945 Section 4.1) arrive over time.  The server
admits a waiting session as soon as a slot and enough of the device-memory
budget are free, keeps every admitted session's state resident in one device
arena, and advances ALL admitted sessions together, one step per iteration,
with the batched step (one CUDA graph launch per iteration).  A session
that arrives while others are running joins at the next iteration; a session
whose episode is over leaves and frees its slot and memory.  Nothing is
re-captured when the set changes: only the instance descriptors are
re-uploaded.

SessionScheduler is the host-side bookkeeping (queue, admission, arena
ranges) and needs no GPU; FlockServer runs it against the library.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

# Device bytes a session of n agents and c cells occupies while admitted:
# resident state (16/agent), the batch's per-agent scratch (cell and rank 8,
# sorted positions 8, sorted index 4), its rows of the flattened actions and
# outputs (4 + 72 + 4 + 4), per-cell scratch (counts, offsets, starts:
# 12/cell) and one descriptor.
BYTES_PER_AGENT = 16 + 8 + 8 + 4 + 4 + 72 + 4 + 4
BYTES_PER_CELL = 12
BYTES_PER_SESSION = 1024


def session_bytes(n_agents: int, n_cells: int) -> int:
    return BYTES_PER_AGENT * n_agents + BYTES_PER_CELL * n_cells + BYTES_PER_SESSION


class SessionPlacer:
    """Host-side placement of sessions across GPUs (one server per GPU, no
    collective): each arriving session goes to the rank with the least work
    placed so far (agents x episode steps), the lowest rank on ties.  The
    placement depends only on the sequence of sessions offered, so every rank
    computes the same one from the same arrival stream and serves its own
    share without any exchange."""

    def __init__(self, n_ranks: int):
        if n_ranks < 1:
            raise ValueError("n_ranks must be at least 1")
        self.load = [0] * n_ranks

    def place(self, n_agents: int, steps: int) -> int:
        r = min(range(len(self.load)), key=lambda k: (self.load[k], k))
        self.load[r] += int(n_agents) * int(steps)
        return r


def place_sessions(arrivals, n_ranks: int):
    """Rank of each (t, n, steps, seed) arrival, in the order given."""
    pl = SessionPlacer(n_ranks)
    return [pl.place(n, steps) for (_t, n, steps, _seed) in arrivals]


@dataclass
class Session:
    sid: int
    n: int
    cells: int
    steps: int
    seed: int
    t_arrival: float
    params: dict = None
    params_c: object = None   # the same as the library's struct, built once
    offset: int = -1          # first agent row of its state in the arena
    steps_done: int = 0       # steps whose results were delivered
    steps_issued: int = 0     # steps launched (one ahead of delivery when pipelined)
    t_admit: float = None
    t_done: float = None
    it0: int = -1             # the server's first iteration that stepped it
    reset: bool = True        # next step observes without moving
    cancelled: bool = False   # left before its episode ended

    @property
    def bytes(self):
        return session_bytes(self.n, self.cells)


class SessionScheduler:
    """Admission control and arena bookkeeping (host only).

    budget_bytes: device memory the admitted sessions may use in total;
    max_slots: sessions stepped together at most; arena_agents: agent rows of
    the state arena; max_cells: cells of all admitted sessions at most;
    queue_limit: waiting sessions beyond which arrivals are rejected."""

    def __init__(self, budget_bytes, max_slots, arena_agents, max_cells, queue_limit=100000):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.arena_agents = int(arena_agents)
        self.max_cells = int(max_cells)
        self.queue_limit = int(queue_limit)
        self.free = [(0, self.arena_agents)]  # free arena ranges (start, length), sorted
        self.queue = collections.deque()
        self.active = []
        self.used_bytes = 0
        self.used_cells = 0
        self.admitted = 0
        self.rejected = 0
        self.finished = []
        self.cancelled = []
        self.version = 0  # bumped whenever the active set changes

    # -- arena ranges: first fit, coalescing on free --
    def _alloc(self, n):
        for k, (s, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (s + n, l - n)
                return s
        return -1

    def _release(self, start, n):
        if n == 0:
            return
        self.free.append((start, n))
        self.free.sort()
        merged = []
        for s, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((s, l))
        self.free = merged

    def submit(self, sess: Session) -> bool:
        """Queue a session; False (rejected) if it can never fit or the queue is full."""
        if (sess.bytes > self.budget or sess.n > self.arena_agents or sess.cells > self.max_cells
                or len(self.queue) >= self.queue_limit):
            self.rejected += 1
            return False
        self.queue.append(sess)
        return True

    def admit(self, now):
        """Admit waiting sessions in arrival order while a slot, budget, cells
        and an arena range are free.  Returns the sessions admitted."""
        out = []
        while self.queue and len(self.active) < self.max_slots:
            s = self.queue[0]
            if (self.used_bytes + s.bytes > self.budget
                    or self.used_cells + s.cells > self.max_cells):
                break
            off = self._alloc(s.n) if s.n > 0 else 0
            if off < 0:
                break
            self.queue.popleft()
            s.offset = off
            s.t_admit = now
            s.reset = True
            self.used_bytes += s.bytes
            self.used_cells += s.cells
            self.active.append(s)
            self.admitted += 1
            out.append(s)
        if out:
            self.version += 1
        return out

    def cancel(self, sess: Session, now) -> bool:
        """Removes a session whose client left: from the queue, or from the
        running set, freeing its slot, memory and arena rows at once (call it
        between steps).  False if the session is neither waiting nor running."""
        if any(q is sess for q in self.queue):
            self.queue = collections.deque(q for q in self.queue if q is not sess)
        elif any(a is sess for a in self.active):
            self.active = [s for s in self.active if s is not sess]
            self._release(sess.offset, sess.n)
            self.used_bytes -= sess.bytes
            self.used_cells -= sess.cells
            self.version += 1
        else:
            return False
        sess.cancelled = True
        sess.t_done = now
        self.cancelled.append(sess)
        return True

    def retire(self, now):
        """Remove sessions whose episode's steps have all been issued (their
        rows may be reused: later uploads follow those steps in stream
        order); returns them."""
        done = [s for s in self.active if s.steps_issued >= s.steps]
        if done:
            self.version += 1
            self.active = [s for s in self.active if s.steps_issued < s.steps]
            for s in done:
                s.t_done = now
                self._release(s.offset, s.n)
                self.used_bytes -= s.bytes
                self.used_cells -= s.cells
                self.finished.append(s)
        return done


class FlockServer:
    """Runs a SessionScheduler against the batched kernel on one GPU.

    state_fn(session) -> (n, 4) float32 initial state of a session: a host
    array (the client's data, uploaded from page-locked staging) or a tensor
    on the server's device (drawn there, e.g. from the session's seed; copied
    into the arena in stream order, no host round trip); params_fn(n) -> parameter dict of a session of
    n agents (default: the library defaults on a square of side
    sqrt(n / 0.1), i.e. density 0.1); action_fn(session, step, out) fills the
    session's int32 actions for one step into the device tensor `out`
    (default: uniform random actions drawn on the device).

    pipeline=True overlaps the host's work for iteration i (retiring,
    admitting, uploading states and descriptors, drawing actions, launching)
    with the GPU's execution of iteration i - 1: the host waits on an event
    of the previous iteration instead of synchronising after each one, and
    the outputs alternate between two buffers so that a step never
    overwrites results not yet delivered.  Results (on_step) then arrive one
    iteration after their step was issued, and action_fn must be stream
    ordered (device work on the server's stream, as the default is): actions
    for step k + 1 are drawn before step k's results reach the host.  A
    session cancelled from on_step may have had one more step issued, whose
    results are dropped.  pipeline=False delivers every step before the next
    is issued."""

    def __init__(self, budget_bytes, state_fn, max_slots=256, arena_agents=2_000_000,
                 max_cells=1_000_000, device="cuda", stream=None, params_fn=None,
                 action_fn=None, queue_limit=100000, tuning=None, pipeline=True):
        import math

        import torch

        from . import FlockBatch, _abi, flock_default_params, flock_instance_cells
        self.torch = torch
        self._params_c = _abi.params_from_dict
        self.dev = torch.device(device)
        self.stream = stream
        self.tuning = tuning
        self.pipeline = bool(pipeline)
        self.params_fn = params_fn or (
            lambda n: flock_default_params(max(math.sqrt(max(n, 1) / 0.1), 12.0)))
        self.state_fn = state_fn
        self.action_fn = action_fn
        self.cells_fn = lambda p: flock_instance_cells(p, tuning)
        self.sched = SessionScheduler(budget_bytes, max_slots, arena_agents, max_cells,
                                      queue_limit)
        self.arena = torch.empty((arena_agents, 4), dtype=torch.float32, device=self.dev)
        self.batch = FlockBatch(max_slots, arena_agents, max_cells, 18, device=self.dev,
                                stream=stream, tuning=tuning,
                                out_buffers=2 if self.pipeline else 1)
        self.actions = torch.empty(arena_agents, dtype=torch.int32, device=self.dev)
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(12345)
        cuda = self.dev.type == "cuda"
        # page-locked staging of admitted sessions' initial states: a mirror
        # of the arena rows, so uploads of different sessions never share rows
        self._stage = torch.empty((arena_agents, 4), dtype=torch.float32,
                                  pin_memory=cuda)
        self._upload_ev = torch.cuda.Event() if cuda else None
        self._upload_pending = False
        self._events = [torch.cuda.Event() if cuda else None for _ in range(2)]
        self.next_sid = 0
        self.iterations = 0
        self.agent_steps = 0
        self.set_changes = 0
        self._version = None      # scheduler version of the uploaded set
        # per delivered iteration: latency (issue to results) and sessions
        # stepped (a session's step latencies are those of the iterations from
        # its it0 on)
        self.iter_lat = []
        self.iter_sessions = []
        self._inflight = None     # the issued iteration whose results are pending
        self._cancel = []         # cancellations taken at the next iteration
        self.on_step = None  # optional callback(session, obs, reward, coll) after each step

    def submit(self, n, steps, seed, t_arrival=None):
        p = self.params_fn(n)
        s = Session(self.next_sid, int(n), self.cells_fn(p), int(steps), int(seed),
                    time.perf_counter() if t_arrival is None else t_arrival, params=p,
                    params_c=self._params_c(p))
        self.next_sid += 1
        return s if self.sched.submit(s) else None

    def _sync_set(self):
        # re-upload the descriptors when the set changed; a session's reset
        # flag is cleared on the device by the step that observes it, and on
        # the host when that step is issued, so it needs no second upload
        if self.sched.version != self._version:
            act = self.sched.active
            self.batch.set_rows([s.params_c for s in act], [s.n for s in act], self.arena,
                                [s.offset for s in act], reset=[s.reset for s in act])
            self._version = self.sched.version
            self.set_changes += 1

    def iteration(self):
        """Deliver cancellations, retire, admit, issue one step of every
        admitted session, and deliver the results of the previous iteration
        (pipeline) or of this one.  Returns the number of sessions stepped."""
        with self.torch.cuda.stream(self.stream) if self.stream is not None else _null():
            return self._iteration()

    def cancel(self, sess):
        """A client left: its session stops before the next iteration (safe
        to call from on_step or between iterations)."""
        self._cancel.append(sess)

    def _upload_states(self, admitted):
        torch = self.torch
        if not admitted:
            return
        # staging rows may still feed the previous iteration's upload
        if self._upload_pending and self._upload_ev is not None:
            self._upload_ev.synchronize()
        staged = False
        for s in admitted:
            st = self.state_fn(s)
            if isinstance(st, torch.Tensor) and st.device == self.arena.device:
                # made on the device: copied in stream order, nothing staged
                self.arena[s.offset:s.offset + s.n].copy_(st.reshape(s.n, 4))
                continue
            st = np.ascontiguousarray(st, dtype=np.float32)
            self._stage[s.offset:s.offset + s.n].numpy()[...] = st
            self.arena[s.offset:s.offset + s.n].copy_(self._stage[s.offset:s.offset + s.n],
                                                      non_blocking=True)
            staged = True
        if staged and self._upload_ev is not None:
            self._upload_ev.record()
            self._upload_pending = True

    def _iteration(self):
        torch = self.torch
        now = time.perf_counter()
        if self._cancel:
            for s in self._cancel:
                self.sched.cancel(s, now)
            self._cancel = []
        self.sched.retire(now)
        admitted = self.sched.admit(now)
        for s in admitted:
            s.it0 = self.iterations
        self._upload_states(admitted)
        act = self.sched.active
        if not act:
            self._deliver_inflight()
            return 0
        t0 = time.perf_counter()
        self._sync_set()
        off = self.batch.n_total
        offsets = list(self.batch.offsets)
        if self.action_fn is not None:
            for s, o in zip(act, offsets):
                self.action_fn(s, s.steps_issued, self.actions[o:o + s.n])
        else:
            self.actions[:off].random_(0, 9, generator=self.gen)
        k = self.iterations % 2 if self.pipeline else 0
        obs, rew, coll = self.batch.step(self.actions[:off], buf=k)
        ev = self._events[k]
        if ev is not None:
            ev.record()
        for s in act:
            s.steps_issued += 1
            s.reset = False  # the device clears its copy in this step
        entry = (list(zip(act, offsets)), obs, rew, coll, ev, t0)
        self.iterations += 1
        self.agent_steps += off
        if self.pipeline:
            prev, self._inflight = self._inflight, entry
            if prev is not None:
                self._deliver(prev)
        else:
            self._deliver(entry)
        return len(act)

    def _deliver_inflight(self):
        if self._inflight is not None:
            prev, self._inflight = self._inflight, None
            self._deliver(prev)

    def _deliver(self, entry):
        members, obs, rew, coll, ev, t0 = entry
        if ev is not None:
            ev.synchronize()
        elif self.stream is not None:
            self.stream.synchronize()
        t1 = time.perf_counter()
        self.iter_lat.append(t1 - t0)
        self.iter_sessions.append(len(members))
        for s, o in members:
            if s.cancelled:
                continue  # issued before its client left: results dropped
            if self.on_step is not None:
                self.on_step(s, obs[o:o + s.n], rew[o:o + s.n], coll[o:o + s.n])
            s.steps_done += 1

    def drain(self):
        """Deliver the results of the last issued iteration."""
        with self.torch.cuda.stream(self.stream) if self.stream is not None else _null():
            self._deliver_inflight()

    def session_latencies(self, s):
        """Step latencies (seconds) of session s: those of the iterations it
        was stepped in, which are consecutive from its first."""
        return self.iter_lat[s.it0:s.it0 + s.steps_done] if s.it0 >= 0 else []

    def run(self, arrivals, duration=None, drain=True):
        """Replay `arrivals` = [(t, n, steps, seed), ...] in real time (t in
        seconds from now) and iterate until all sessions are done (or until
        `duration` seconds, when given).  Returns stats()."""
        t_start = time.perf_counter()
        pending = collections.deque(sorted(arrivals))
        while True:
            now = time.perf_counter() - t_start
            while pending and pending[0][0] <= now:
                t, n, steps, seed = pending.popleft()
                self.submit(n, steps, seed, t_arrival=t_start + t)
            if duration is not None and now >= duration:
                break
            if not self.sched.active and not self.sched.queue:
                self.drain()
                if not pending:
                    break
                time.sleep(min(0.001, max(0.0, pending[0][0] - now)))
                continue
            self.iteration()
        self.drain()
        self.wall = time.perf_counter() - t_start
        return self.stats()

    def stats(self):
        # every session stepped in an iteration saw that iteration's latency
        lat = np.repeat(np.asarray(self.iter_lat), np.asarray(self.iter_sessions, dtype=np.int64))
        waits = [s.t_admit - s.t_arrival
                 for s in self.sched.finished + self.sched.active + self.sched.cancelled
                 if s.t_admit is not None]
        wall = getattr(self, "wall", None)
        return {
            "sessions_admitted": self.sched.admitted, "sessions_rejected": self.sched.rejected,
            "sessions_finished": len(self.sched.finished),
            "sessions_cancelled": len(self.sched.cancelled),
            "sessions_waiting": len(self.sched.queue), "iterations": self.iterations,
            "agent_steps": self.agent_steps, "set_changes": self.set_changes,
            "pipeline": self.pipeline,
            "step_latency_p50_ms": 1e3 * float(np.percentile(lat, 50)) if lat.size else None,
            "step_latency_p99_ms": 1e3 * float(np.percentile(lat, 99)) if lat.size else None,
            "queue_wait_p50_ms": 1e3 * float(np.percentile(waits, 50)) if waits else None,
            "queue_wait_p99_ms": 1e3 * float(np.percentile(waits, 99)) if waits else None,
            "agent_steps_per_s": self.agent_steps / wall if wall else None,
            "agents_per_iteration": self.agent_steps / self.iterations if self.iterations else 0,
            "wall_s": wall,
        }

    def close(self):
        self.drain()
        self.batch.close()


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
