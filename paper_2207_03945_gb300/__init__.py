"""GB300 flock environment step (arXiv 2207.03945, Section 4.1).

Thin Python binding of ``libflock.so`` (C ABI declared in include/flock.h):
the functions below carry the C names and only marshal arguments -- tensors
become device pointers, dicts become ``flock_params`` -- so every step of the
environment runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing this package raises
if the library has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes

from . import _abi
from ._abi import (FLOCK_ERR_ACTION, FLOCK_ERR_BOUNDS, FLOCK_ERR_OVERFLOW, FLOCK_ERR_STATE,
                   FLOCK_ERR_TIMEOUT, FlockError)

__all__ = [
    "FlockError", "FLOCK_ERR_ACTION", "FLOCK_ERR_STATE", "FLOCK_ERR_TIMEOUT",
    "FLOCK_ERR_OVERFLOW", "FLOCK_ERR_BOUNDS", "flock_default_params", "flock_obs_dim",
    "flock_workspace_bytes",
    "flock_derive",
    "env_create", "env_reset", "env_step", "env_step_continuous", "env_rollout", "flock_gae",
    "flock_seed_states",
    "env_set_types",
    "env_step_host", "env_step_host_bind", "env_get_state", "env_set_state",
    "env_get_error", "env_get_derived", "env_get_tuning", "env_set_timing",
    "env_get_phase_times", "env_destroy", "FlockEnv", "lib_path", "flock_instance_cells",
    "env_step_policy",
    "flock_batch_workspace_bytes", "env_batch_create", "env_batch_set", "env_batch_step",
    "env_batch_set_rows", "env_batch_get_error", "env_batch_set_spin_limit", "env_batch_get_launch",
    "FlockSlab",
    "env_batch_set_timing", "env_batch_get_time", "env_batch_destroy", "FlockBatch",
    "flock_step_static",
]

lib_path = _abi.LIB_PATH


def _torch():
    import torch
    return torch


def _ptr(t, dtype, shape=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor of the given dtype/shape."""
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FlockError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise FlockError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise FlockError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise FlockError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def flock_default_params(side: float) -> dict:
    p = _abi.FlockParams()
    _abi.check(_abi.lib.flock_default_params(ctypes.c_float(side), ctypes.byref(p)))
    return _abi.params_to_dict(p)


def flock_obs_dim(params: dict) -> int:
    r = _abi.lib.flock_obs_dim(ctypes.byref(_abi.params_from_dict(params)))
    _abi.check(min(r, 0))
    return r


def flock_workspace_bytes(params: dict, n_agents: int, tuning: dict | None = None) -> int:
    out = ctypes.c_size_t(0)
    t = _abi.tuning_from_dict(tuning)
    _abi.check(_abi.lib.flock_workspace_bytes(ctypes.byref(_abi.params_from_dict(params)),
                                              ctypes.byref(t) if t is not None else None,
                                              int(n_agents), ctypes.byref(out)))
    return int(out.value)


def flock_derive(params: dict, tuning: dict | None = None) -> dict:
    d = _abi.FlockDerived()
    t = _abi.tuning_from_dict(tuning)
    _abi.check(_abi.lib.flock_derive(ctypes.byref(_abi.params_from_dict(params)),
                                     ctypes.byref(t) if t is not None else None, ctypes.byref(d)))
    return _abi.derived_to_dict(d)


class _Env:
    """Opaque handle (holds the workspace tensor alive)."""

    def __init__(self, handle, n, obs_dim, workspace):
        self.handle = handle
        self.n = n
        self.obs_dim = obs_dim
        self.workspace = workspace


def env_create(params: dict, n_agents: int, workspace, stream=None, tuning: dict | None = None):
    torch = _torch()
    if not isinstance(workspace, torch.Tensor) or workspace.dtype != torch.uint8:
        raise FlockError("workspace must be a uint8 CUDA tensor")
    h = ctypes.c_void_p()
    t = _abi.tuning_from_dict(tuning)
    _abi.check(_abi.lib.env_create(ctypes.byref(_abi.params_from_dict(params)),
                                   ctypes.byref(t) if t is not None else None, int(n_agents),
                                   _ptr(workspace, torch.uint8, name="workspace"),
                                   ctypes.c_size_t(workspace.numel()), _stream(stream),
                                   ctypes.byref(h)))
    return _Env(h, int(n_agents), flock_obs_dim(params), workspace)


def _outs(env, obs, reward, coll):
    torch = _torch()
    return (_ptr(obs, torch.float32, (env.n, env.obs_dim), "obs"),
            _ptr(reward, torch.float32, (env.n,), "reward"),
            _ptr(coll, torch.int32, (env.n,), "coll"))


def env_reset(env, state0, obs, reward, coll):
    torch = _torch()
    _abi.check(_abi.lib.env_reset(env.handle, _ptr(state0, torch.float32, (env.n, 4), "state0"),
                                  *_outs(env, obs, reward, coll)))


def env_step(env, actions, obs, reward, coll):
    torch = _torch()
    _abi.check(_abi.lib.env_step(env.handle, _ptr(actions, torch.int32, (env.n,), "actions"),
                                 *_outs(env, obs, reward, coll)))


def env_rollout(env, actions, obs, reward, coll, actions2=None):
    """T steps in one graph launch: actions (T, n) int32, or actions2 (T, n, 2)
    float32 continuous actions (then actions is None); obs (T, n, obs_dim),
    reward (T, n) float32 and coll (T, n) int32 receive every step."""
    torch = _torch()
    src = actions if actions is not None else actions2
    if src is None:
        raise FlockError("give actions or actions2")
    T = int(src.shape[0])
    a1 = _ptr(actions, torch.int32, (T, env.n), "actions") if actions is not None else None
    a2 = _ptr(actions2, torch.float32, (T, env.n, 2), "actions2") if actions2 is not None else None
    _abi.check(_abi.lib.env_rollout(
        env.handle, T, a1, a2, _ptr(obs, torch.float32, (T, env.n, env.obs_dim), "obs"),
        _ptr(reward, torch.float32, (T, env.n), "reward"),
        _ptr(coll, torch.int32, (T, env.n), "coll")))


def flock_gae(reward, value, gamma: float, lam: float, adv, ret, stream=None):
    """Generalised advantage estimation over a rollout on the GPU: reward
    (T, n), value (T + 1, n), adv and ret (T, n), float32 CUDA tensors."""
    torch = _torch()
    T, n = int(reward.shape[0]), int(reward.shape[1])
    _abi.check(_abi.lib.flock_gae(
        T, n, _ptr(reward, torch.float32, (T, n), "reward"),
        _ptr(value, torch.float32, (T + 1, n), "value"), ctypes.c_float(gamma),
        ctypes.c_float(lam), _ptr(adv, torch.float32, (T, n), "adv"),
        _ptr(ret, torch.float32, (T, n), "ret"), _stream(stream)))


def flock_seed_states(state, side: float, seed: int, speed: float = 0.5, stream=None):
    """Initial states drawn on the device from a seed (see flock.h): state is
    an (n, 4) float32 CUDA tensor, filled in place with x, y ~ U[0, side),
    theta ~ U[0, 2 pi) and the given speed, from SplitMix64 outputs of seed."""
    torch = _torch()
    n = int(state.shape[0])
    _abi.check(_abi.lib.flock_seed_states(
        _ptr(state, torch.float32, (n, 4), "state"), n, ctypes.c_float(side),
        ctypes.c_float(speed), ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), _stream(stream)))


def env_set_types(env, types):
    """Tag: agent types, (n,) uint8 CUDA tensor (0 runner, 1 chaser)."""
    torch = _torch()
    _abi.check(_abi.lib.env_set_types(env.handle, _ptr(types, torch.uint8, (env.n,), "types")))


def env_step_continuous(env, actions2, obs, reward, coll):
    """Step with continuous actions: actions2 is (n, 2) float32 (acceleration,
    rotation), clamped to [-speed_step, speed_step] x [-turn_step, turn_step]."""
    torch = _torch()
    _abi.check(_abi.lib.env_step_continuous(
        env.handle, _ptr(actions2, torch.float32, (env.n, 2), "actions2"),
        *_outs(env, obs, reward, coll)))


def env_step_policy(env, weights_bf16, actions, reward, coll, logits=None, obs=None):
    """Step whose next actions come from the fused BF16 policy MLP; actions
    (int32, n) are read, then overwritten with the greedy actions.
    weights_bf16: 5,961 bf16 values (torch.bfloat16, or int16/uint16 bits)."""
    torch = _torch()
    w = weights_bf16
    if not (isinstance(w, torch.Tensor) and w.is_cuda and w.numel() == 5961 and
            w.element_size() == 2 and w.is_contiguous()):
        raise FlockError("weights must be 5961 contiguous 16-bit values on the device")
    _abi.check(_abi.lib.env_step_policy(
        env.handle, ctypes.c_void_p(w.data_ptr()), _ptr(actions, torch.int32, (env.n,), "actions"),
        _ptr(reward, torch.float32, (env.n,), "reward"), _ptr(coll, torch.int32, (env.n,), "coll"),
        _ptr(logits, torch.float32, (env.n, 9), "logits") if logits is not None else None,
        _ptr(obs, torch.float32, (env.n, env.obs_dim), "obs") if obs is not None else None))


def _host_ptrs(env, actions, obs, reward, coll):
    """Host pointers of the four buffers of a host-memory step, checked."""
    import numpy as np
    torch = _torch()
    n, d = env.n, env.obs_dim
    np_types = {torch.int32: np.int32, torch.float32: np.float32}

    def hp(a, dtype, shape, name):
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != dtype or not a.is_contiguous() or tuple(a.shape) != shape:
                raise FlockError("%s: bad host tensor" % name)
            return ctypes.c_void_p(a.data_ptr())
        if (not isinstance(a, np.ndarray) or not a.flags.c_contiguous or a.shape != shape
                or a.dtype != np_types[dtype]):
            raise FlockError("%s: bad host array" % name)
        return ctypes.c_void_p(a.ctypes.data)

    return (hp(actions, torch.int32, (n,), "actions"), hp(obs, torch.float32, (n, d), "obs"),
            hp(reward, torch.float32, (n,), "reward"), hp(coll, torch.int32, (n,), "coll"))


def env_step_host(env, actions, obs, reward, coll):
    """Host-memory step: numpy arrays or pinned CPU tensors; waits for completion."""
    _abi.check(_abi.lib.env_step_host(env.handle, *_host_ptrs(env, actions, obs, reward, coll)))


def env_step_host_bind(env, actions, obs, reward, coll):
    """Checks the four host buffers of env_step_host once and returns a
    callable that runs env_step_host on them: the same C call, without
    re-checking the buffers on every step.  For loops that step many times
    through the same pinned buffers (refilling the actions and reading the
    outputs in place).  The buffers stay referenced by the callable; it
    raises once the environment is closed."""
    ptrs = _host_ptrs(env, actions, obs, reward, coll)
    keep = (actions, obs, reward, coll)
    lib_step, check = _abi.lib.env_step_host, _abi.check

    def step():
        h = env.handle
        if not h:
            raise FlockError("environment closed")
        check(lib_step(h, *ptrs))

    step.buffers = keep
    return step


def env_get_state(env, state):
    torch = _torch()
    _abi.check(_abi.lib.env_get_state(env.handle, _ptr(state, torch.float32, (env.n, 4), "state")))


def env_set_state(env, state):
    torch = _torch()
    _abi.check(_abi.lib.env_set_state(env.handle, _ptr(state, torch.float32, (env.n, 4), "state")))


def env_get_error(env) -> int:
    bits = ctypes.c_uint32(0)
    _abi.check(_abi.lib.env_get_error(env.handle, ctypes.byref(bits)))
    return int(bits.value)


def env_get_derived(env) -> dict:
    d = _abi.FlockDerived()
    _abi.check(_abi.lib.env_get_derived(env.handle, ctypes.byref(d)))
    return _abi.derived_to_dict(d)


def env_get_tuning(env) -> dict:
    t = _abi.FlockTuning()
    _abi.check(_abi.lib.env_get_tuning(env.handle, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in _abi.FlockTuning._fields_}


def env_set_timing(env, enable: bool):
    _abi.check(_abi.lib.env_set_timing(env.handle, 1 if enable else 0))


def env_get_phase_times(env) -> list:
    """Per-kernel milliseconds of the last step: apply+bin, scan, scatter, neighbours."""
    ms = (ctypes.c_float * 4)()
    _abi.check(_abi.lib.env_get_phase_times(env.handle, ms))
    return list(ms)


def env_destroy(env):
    if env is not None and env.handle:
        _abi.lib.env_destroy(env.handle)
        env.handle = None


class FlockEnv:
    """Convenience owner of one environment: allocates the workspace and the
    output tensors with torch and calls the C ABI."""

    def __init__(self, params: dict, n_agents: int, device="cuda", stream=None,
                 tuning: dict | None = None):
        torch = _torch()
        self.params = dict(params)
        self.n = int(n_agents)
        self.device = torch.device(device)
        self.obs_dim = flock_obs_dim(params)
        nbytes = flock_workspace_bytes(params, self.n, tuning)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        self.stream = stream
        self.env = env_create(params, self.n, self.workspace, stream, tuning)
        self.obs = torch.empty((self.n, self.obs_dim), dtype=torch.float32, device=self.device)
        self.reward = torch.empty(self.n, dtype=torch.float32, device=self.device)
        self.coll = torch.empty(self.n, dtype=torch.int32, device=self.device)

    def reset(self, state0):
        env_reset(self.env, state0, self.obs, self.reward, self.coll)
        return self.obs, self.reward, self.coll

    def step(self, actions):
        env_step(self.env, actions, self.obs, self.reward, self.coll)
        return self.obs, self.reward, self.coll

    def set_types(self, types):
        env_set_types(self.env, types)

    def step_continuous(self, actions2):
        env_step_continuous(self.env, actions2, self.obs, self.reward, self.coll)
        return self.obs, self.reward, self.coll

    def rollout(self, actions=None, actions2=None):
        """T steps in one launch; returns new (T, n, obs_dim), (T, n) and (T, n)
        tensors holding every step's outputs."""
        torch = _torch()
        src = actions if actions is not None else actions2
        T = int(src.shape[0])
        obs = torch.empty((T, self.n, self.obs_dim), dtype=torch.float32, device=self.device)
        rew = torch.empty((T, self.n), dtype=torch.float32, device=self.device)
        coll = torch.empty((T, self.n), dtype=torch.int32, device=self.device)
        env_rollout(self.env, actions, obs, rew, coll, actions2=actions2)
        return obs, rew, coll

    def state(self):
        torch = _torch()
        s = torch.empty((self.n, 4), dtype=torch.float32, device=self.device)
        env_get_state(self.env, s)
        return s

    def set_state(self, s):
        env_set_state(self.env, s)

    def error(self) -> int:
        return env_get_error(self.env)

    def derived(self) -> dict:
        return env_get_derived(self.env)

    def tuning(self) -> dict:
        return env_get_tuning(self.env)

    def close(self):
        env_destroy(self.env)
        self.env = None

    def __del__(self):
        try:
            if getattr(self, "env", None) is not None:
                self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Batched step (many instances, one persistent kernel per step)
# ---------------------------------------------------------------------------
def flock_instance_cells(params: dict, tuning: dict | None = None) -> int:
    out = ctypes.c_int(0)
    t = _abi.tuning_from_dict(tuning)
    _abi.check(_abi.lib.flock_instance_cells(ctypes.byref(_abi.params_from_dict(params)),
                                             ctypes.byref(t) if t is not None else None,
                                             ctypes.byref(out)))
    return int(out.value)


def flock_batch_workspace_bytes(max_instances: int, max_agents: int, max_cells: int,
                                tuning: dict | None = None) -> int:
    out = ctypes.c_size_t(0)
    t = _abi.tuning_from_dict(tuning)
    _abi.check(_abi.lib.flock_batch_workspace_bytes(int(max_instances), int(max_agents),
                                                    int(max_cells),
                                                    ctypes.byref(t) if t is not None else None,
                                                    ctypes.byref(out)))
    return int(out.value)


class _Batch:
    def __init__(self, handle, workspace):
        self.handle = handle
        self.workspace = workspace


def env_batch_create(max_instances, max_agents, max_cells, workspace, stream=None, tuning=None):
    torch = _torch()
    h = ctypes.c_void_p()
    t = _abi.tuning_from_dict(tuning)
    _abi.check(_abi.lib.env_batch_create(int(max_instances), int(max_agents), int(max_cells),
                                         ctypes.byref(t) if t is not None else None,
                                         _ptr(workspace, torch.uint8, name="workspace"),
                                         ctypes.c_size_t(workspace.numel()), _stream(stream),
                                         ctypes.byref(h)))
    return _Batch(h, workspace)


def env_batch_set(batch, params_list, n_agents, states, reset=None):
    """Active set: parallel lists of parameter dicts, agent counts, state
    tensors (n x 4 float32 on the device) and reset flags."""
    torch = _torch()
    k = len(params_list)
    P = (_abi.FlockParams * max(k, 1))(*[_abi.params_from_dict(p) for p in params_list])
    N = (ctypes.c_int * max(k, 1))(*[int(n) for n in n_agents])
    S = (ctypes.c_void_p * max(k, 1))(*[
        _ptr(st, torch.float32, (int(n), 4), "state").value if int(n) > 0 else None
        for st, n in zip(states, n_agents)])
    R = (ctypes.c_int * max(k, 1))(*[int(bool(r)) for r in (reset or [0] * k)])
    _abi.check(_abi.lib.env_batch_set(batch.handle, k, P, N, S, R))
    batch.states = list(states)  # keep the tensors alive while active


def env_batch_set_rows(batch, params_c, n_agents, arena, rows, reset=None):
    """Active set whose states are row ranges of one arena ((R, 4) float32 on
    the device): instance k's state is arena[rows[k] : rows[k] + n_agents[k]].
    params_c: FlockParams structs (from params_from_dict, built once per
    instance).  For callers that change the set often, such as the serving
    loop: one pass over the instances in plain Python and ctypes arrays, no
    per-instance tensor checks, dict conversions or numpy round trips."""
    torch = _torch()
    if not isinstance(arena, torch.Tensor) or arena.dim() != 2 or arena.shape[1] != 4:
        raise FlockError("arena must be an (R, 4) tensor")
    k = len(params_c)
    if len(n_agents) != k or len(rows) != k:
        raise FlockError("params, agent counts and rows differ in length")
    cap = int(arena.shape[0])
    nn = [int(x) for x in n_agents]
    rr = [int(x) for x in rows]
    fp = _abi.FlockParams
    for q, n_, r_ in zip(params_c, nn, rr):
        if n_ < 0 or r_ < 0 or r_ + n_ > cap:
            raise FlockError("row range outside the arena")
        if not isinstance(q, fp):
            raise FlockError("params_c must be FlockParams structs")
    base = _ptr(arena, torch.float32, name="arena").value
    m = max(k, 1)
    P = (fp * m)(*params_c)
    N = (ctypes.c_int * m)(*nn)
    S = (ctypes.c_void_p * m)(*[base + 16 * r_ for r_ in rr])
    R = (ctypes.c_int * m)(*([1 if x else 0 for x in reset] if reset is not None else []))
    _abi.check(_abi.lib.env_batch_set(batch.handle, k, P, N, S, R))
    batch.states = [arena]  # keep the arena alive while active


def env_batch_step(batch, actions, obs, reward, coll):
    torch = _torch()
    _abi.check(_abi.lib.env_batch_step(batch.handle, _ptr(actions, torch.int32, name="actions"),
                                       _ptr(obs, torch.float32, name="obs"),
                                       _ptr(reward, torch.float32, name="reward"),
                                       _ptr(coll, torch.int32, name="coll")))


def env_batch_get_error(batch) -> int:
    bits = ctypes.c_uint32(0)
    _abi.check(_abi.lib.env_batch_get_error(batch.handle, ctypes.byref(bits)))
    return int(bits.value)


def env_batch_set_spin_limit(batch, limit: int):
    _abi.check(_abi.lib.env_batch_set_spin_limit(batch.handle, ctypes.c_uint(limit)))


def env_batch_get_launch(batch):
    g = ctypes.c_int(0)
    b = ctypes.c_int(0)
    _abi.check(_abi.lib.env_batch_get_launch(batch.handle, ctypes.byref(g), ctypes.byref(b)))
    return int(g.value), int(b.value)


def env_batch_set_timing(batch, enable: bool):
    _abi.check(_abi.lib.env_batch_set_timing(batch.handle, 1 if enable else 0))


def env_batch_get_time(batch) -> float:
    ms = ctypes.c_float(0)
    _abi.check(_abi.lib.env_batch_get_time(batch.handle, ctypes.byref(ms)))
    return float(ms.value)


def env_batch_destroy(batch):
    if batch is not None and batch.handle:
        _abi.lib.env_batch_destroy(batch.handle)
        batch.handle = None


class FlockBatch:
    """Convenience owner of a batch: allocates the workspace and the
    flattened output tensors with torch and calls the C ABI.  With
    out_buffers=2 it keeps two sets of outputs, so that a step may write one
    set while the caller still reads the other (step(..., buf=k))."""

    def __init__(self, max_instances: int, max_agents: int, max_cells: int, obs_dim: int,
                 device="cuda", stream=None, tuning: dict | None = None, out_buffers: int = 1):
        torch = _torch()
        self.device = torch.device(device)
        self.obs_dim = int(obs_dim)
        nbytes = flock_batch_workspace_bytes(max_instances, max_agents, max_cells, tuning)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.batch = env_batch_create(max_instances, max_agents, max_cells, self.workspace,
                                      stream, tuning)
        m = max(max_agents, 1)
        self.outs = [(torch.empty((m, self.obs_dim), dtype=torch.float32, device=self.device),
                      torch.empty(m, dtype=torch.float32, device=self.device),
                      torch.empty(m, dtype=torch.int32, device=self.device))
                     for _ in range(max(1, int(out_buffers)))]
        self.obs, self.reward, self.coll = self.outs[0]
        self.n_total = 0
        self.offsets = []

    def set(self, params_list, n_agents, states, reset=None):
        env_batch_set(self.batch, params_list, n_agents, states, reset)
        self._offsets(n_agents)

    def set_rows(self, params_c, n_agents, arena, rows, reset=None):
        """The active set as row ranges of one arena (env_batch_set_rows)."""
        env_batch_set_rows(self.batch, params_c, n_agents, arena, rows, reset)
        self._offsets(n_agents)

    def _offsets(self, n_agents):
        self.offsets = []
        off = 0
        for n in n_agents:
            self.offsets.append(off)
            off += int(n)
        self.n_total = off

    def step(self, actions, buf: int = 0):
        obs, reward, coll = self.outs[buf]
        env_batch_step(self.batch, actions, obs, reward, coll)
        n = self.n_total
        return obs[:n], reward[:n], coll[:n]

    def error(self) -> int:
        return env_batch_get_error(self.batch)

    def close(self):
        env_batch_destroy(self.batch)
        self.batch = None

    def __del__(self):
        try:
            if getattr(self, "batch", None) is not None:
                self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Allocation-free step
# ---------------------------------------------------------------------------
def flock_step_static(params: dict, state, actions, obs, reward, coll, stream=None,
                      wait: bool = True):
    """One step whose scratch lives in the library's fixed device array, for
    callers that cannot allocate device memory (see flock.h).  state (n x 4)
    is updated in place; actions None observes without moving.  With wait,
    returns the step's FLOCK_ERR_* bits after the stream has finished."""
    torch = _torch()
    n = int(state.shape[0])
    d = flock_obs_dim(params)
    bits = ctypes.c_uint32(0)
    _abi.check(_abi.lib.flock_step_static(
        ctypes.byref(_abi.params_from_dict(params)), n,
        _ptr(state, torch.float32, (n, 4), "state"),
        _ptr(actions, torch.int32, (n,), "actions") if actions is not None else None,
        _ptr(obs, torch.float32, (n, d), "obs"), _ptr(reward, torch.float32, (n,), "reward"),
        _ptr(coll, torch.int32, (n,), "coll"), _stream(stream),
        ctypes.byref(bits) if wait else None))
    return int(bits.value) if wait else None


# ---------------------------------------------------------------------------
# Slabs (one square decomposed over several devices; see slab.py)
# ---------------------------------------------------------------------------
class FlockSlab:
    """A slab environment: the cell list of rows [row0, row0 + nrows) of a
    square's grid (modulo its cells per side), for at most n_max own and
    ghost agents.  apply() moves own agents; observe() observes the own
    agents over own and ghost agents (env_slab_apply / env_slab_observe)."""

    def __init__(self, params: dict, n_max: int, row0: int, nrows: int, device="cuda",
                 stream=None, tuning: dict | None = None):
        torch = _torch()
        self.params = dict(params)
        self.n_max = int(n_max)
        self.device = torch.device(device)
        self.obs_dim = flock_obs_dim(params)
        t = _abi.tuning_from_dict(tuning)
        pc = _abi.params_from_dict(params)
        nbytes = ctypes.c_size_t(0)
        _abi.check(_abi.lib.flock_slab_workspace_bytes(
            ctypes.byref(pc), ctypes.byref(t) if t is not None else None, self.n_max, int(row0),
            int(nrows), ctypes.byref(nbytes)))
        self.workspace = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8,
                                     device=self.device)
        h = ctypes.c_void_p()
        _abi.check(_abi.lib.env_slab_create(
            ctypes.byref(pc), ctypes.byref(t) if t is not None else None, self.n_max, int(row0),
            int(nrows), _ptr(self.workspace, torch.uint8, name="workspace"),
            ctypes.c_size_t(self.workspace.numel()), _stream(stream), ctypes.byref(h)))
        self.env = _Env(h, self.n_max, self.obs_dim, self.workspace)

    def apply(self, state, actions):
        """Actions (n int32) of the n agents of state (n x 4 float32), in place."""
        torch = _torch()
        n = int(state.shape[0])
        _abi.check(_abi.lib.env_slab_apply(
            self.env.handle, n, _ptr(state, torch.float32, (n, 4), "state"),
            _ptr(actions, torch.int32, (n,), "actions")))

    def observe(self, state, n_own: int, obs, reward, coll):
        """Observation, reward and collisions of the first n_own agents of
        state (own agents, then ghosts) over all of them."""
        torch = _torch()
        n = int(state.shape[0])
        _abi.check(_abi.lib.env_slab_observe(
            self.env.handle, int(n_own), n - int(n_own), _ptr(state, torch.float32, (n, 4), "state"),
            _ptr(obs, torch.float32, (int(n_own), self.obs_dim), "obs"),
            _ptr(reward, torch.float32, (int(n_own),), "reward"),
            _ptr(coll, torch.int32, (int(n_own),), "coll")))

    def error(self) -> int:
        return env_get_error(self.env)

    def close(self):
        if self.env is not None:
            env_destroy(self.env)
            self.env = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
