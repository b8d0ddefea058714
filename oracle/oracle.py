"""Loader for the flock oracle -- TEST INFRASTRUCTURE, NOT THE PRODUCT PATH.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It builds and loads
``oracle/libflock_oracle.so`` (plain C, ``flock_oracle.c``) with ctypes and
exposes it with numpy arrays.  Nothing here imports the CUDA product package.

The oracle states one update of the flock environment (arXiv 2207.03945,
Section 4.1 with Eq. 1, Fig. 3 and Fig. 4) as the brute-force O(N^2)
definition in FP32; see ``flock_oracle.c`` for the formulas and readings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flock_oracle.c")
LIB_PATH = os.path.join(_HERE, "libflock_oracle.so")

FLAG_ACTION = 1
FLAG_STATE = 2
FLAG_OVERFLOW = 8

MAXV = 128

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile flock_oracle.c into libflock_oracle.so (gcc, FP contraction off)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(_SRC)):
        return LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fno-unsafe-math-optimizations", "-fPIC", "-shared"]
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        # no OpenMP runtime: the oracle stays single-threaded
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("side", ctypes.c_float), ("view_radius", ctypes.c_float),
                ("fov", ctypes.c_float), ("agent_radius", ctypes.c_float),
                ("collision_penalty", ctypes.c_float), ("speed_min", ctypes.c_float),
                ("speed_max", ctypes.c_float), ("speed_step", ctypes.c_float),
                ("turn_step", ctypes.c_float), ("num_segments", ctypes.c_int)]


class _Derived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("L", "HL", "RV", "RV2", "RC2", "INV_SPAN", "TWO_PI", "CF", "SF",
                 "SMIN", "SMAX")] + [
        ("DT", ctypes.c_float * 3), ("DS", ctypes.c_float * 3),
        ("T", ctypes.c_float * (MAXV + 1)),
        ("v", ctypes.c_int), ("full", ctypes.c_int), ("K", ctypes.c_int),
        ("PK", ctypes.c_int64), ("NMAX", ctypes.c_int64)]


def _bind(path):
    lib = ctypes.CDLL(path)
    fp = ctypes.POINTER(ctypes.c_float)
    ip = ctypes.POINTER(ctypes.c_int32)
    up = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_derive.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Derived)]
    lib.oracle_derived_size.restype = ctypes.c_int
    lib.oracle_step.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, fp, ip, fp, fp,
                                ip, up, ctypes.c_int]
    lib.oracle_observe_rows.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, fp,
                                        ctypes.c_int, ip, fp, fp, ip, ctypes.c_int]
    lib.oracle_apply.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, fp, ip, up]
    lib.oracle_step_tag.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, fp,
                                    ctypes.POINTER(ctypes.c_uint8), fp, fp, fp, ip, up,
                                    ctypes.c_int]
    lib.oracle_gae.argtypes = [ctypes.c_int, ctypes.c_int, fp, fp, ctypes.c_float, ctypes.c_float,
                               fp, fp]
    lib.oracle_step_cont.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, fp, fp, ctypes.c_int,
                                     fp, fp, ip, up, ctypes.c_int]
    lib.oracle_sincos.argtypes = [ctypes.c_float, fp, fp]
    lib.oracle_diamond.argtypes = [ctypes.c_float, ctypes.c_float]
    lib.oracle_diamond.restype = ctypes.c_float
    if lib.oracle_derived_size() != ctypes.sizeof(_Derived):
        raise RuntimeError("oracle derived-constant layout mismatch")
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(LIB_PATH)
    return _lib


def use_library(path):
    """Point this module at another build of the oracle (e.g. a deliberately
    mutated copy built by a test); returns the previous handle."""
    global _lib
    with _lock:
        prev = _lib
        _lib = _bind(path) if isinstance(path, str) else path
    return prev


def build_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source to ``out_path`` (tests use
    this to plant mistakes and check that the pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", out_path, src, "-lm"], check=True, capture_output=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _params(p: dict) -> _Params:
    return _Params(*(float(p[k]) for k in ("side", "view_radius", "fov", "agent_radius",
                                             "collision_penalty", "speed_min", "speed_max",
                                             "speed_step", "turn_step")),
                   int(p["num_segments"]))


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def obs_dim(params: dict, layout: int = 0) -> int:
    """Observation length: layout 0 = (distance, count) per sector, speed,
    heading; layout 1 = distance per sector, speed (the paper's)."""
    v = int(params["num_segments"])
    return v + 1 if layout == 1 else 2 * v + 2


def derive(params: dict) -> dict:
    """The oracle's derived constants (its own computation) as a dict."""
    lib = _load()
    d = _Derived()
    rc = lib.oracle_derive(ctypes.byref(_params(params)), ctypes.byref(d))
    if rc != 0:
        raise ValueError("oracle rejected parameters (rc=%d)" % rc)
    out = {n: getattr(d, n) for n in ("L", "HL", "RV", "RV2", "RC2", "INV_SPAN", "TWO_PI",
                                       "CF", "SF", "SMIN", "SMAX", "v", "full", "K", "PK",
                                       "NMAX")}
    out["DT"] = list(d.DT)
    out["DS"] = list(d.DS)
    out["T"] = [d.T[m] for m in range(1, d.v + 1)]
    return out


def params_ok(params: dict) -> bool:
    lib = _load()
    d = _Derived()
    return lib.oracle_derive(ctypes.byref(_params(params)), ctypes.byref(d)) == 0


def step(params: dict, state: np.ndarray, actions: np.ndarray | None = None, threads: int = 1):
    """One update.  Returns (new_state, obs, reward, coll, flags).

    state: (N, 4) float32 (x, y, theta, s); actions: (N,) int32 in [0, 9) or
    None for a reset (observe the given state without moving)."""
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float32).copy()
    n = st.shape[0]
    D = obs_dim(params)
    obs = np.zeros((n, D), np.float32)
    rew = np.zeros(n, np.float32)
    coll = np.zeros(n, np.int32)
    flags = ctypes.c_uint32(0)
    act = None
    if actions is not None:
        act = np.ascontiguousarray(actions, dtype=np.int32)
        assert act.shape == (n,)
    rc = lib.oracle_step(ctypes.byref(_params(params)), n, _f(st),
                         _i(act) if act is not None else None, _f(obs), _f(rew), _i(coll),
                         ctypes.byref(flags), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected parameters (rc=%d)" % rc)
    return st, obs, rew, coll, int(flags.value)


def step_cont(params: dict, state: np.ndarray, actions: np.ndarray | None = None,
              layout: int = 1, threads: int = 0):
    """One update with continuous actions (N, 2) float32 (acceleration,
    rotation), or None for a reset.  Returns (new_state, obs, reward, coll,
    flags); obs has obs_dim(params, layout) columns."""
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float32).copy()
    n = st.shape[0]
    obs = np.zeros((n, obs_dim(params, layout)), np.float32)
    rew = np.zeros(n, np.float32)
    coll = np.zeros(n, np.int32)
    flags = ctypes.c_uint32(0)
    act = None
    if actions is not None:
        act = np.ascontiguousarray(actions, dtype=np.float32)
        assert act.shape == (n, 2)
    rc = lib.oracle_step_cont(ctypes.byref(_params(params)), n, _f(st),
                              _f(act) if act is not None else None, int(layout), _f(obs),
                              _f(rew), _i(coll), ctypes.byref(flags), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the call (rc=%d)" % rc)
    return st, obs, rew, coll, int(flags.value)


def step_tag(params: dict, state: np.ndarray, types: np.ndarray, actions: np.ndarray | None = None,
             threads: int = 0):
    """One tag update (Section 4.2): types (N,) uint8 (0 runner, 1 chaser),
    actions (N, 2) float32 (speed, rotation) or None for a reset.  Returns
    (new_state, obs (N, 2v), reward, coll, flags)."""
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float32).copy()
    n = st.shape[0]
    ty = np.ascontiguousarray(types, dtype=np.uint8)
    assert ty.shape == (n,)
    v = int(params["num_segments"])
    obs = np.zeros((n, 2 * v), np.float32)
    rew = np.zeros(n, np.float32)
    coll = np.zeros(n, np.int32)
    flags = ctypes.c_uint32(0)
    act = None
    if actions is not None:
        act = np.ascontiguousarray(actions, dtype=np.float32)
        assert act.shape == (n, 2)
    rc = lib.oracle_step_tag(ctypes.byref(_params(params)), n, _f(st),
                             ty.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                             _f(act) if act is not None else None, _f(obs), _f(rew), _i(coll),
                             ctypes.byref(flags), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the call (rc=%d)" % rc)
    return st, obs, rew, coll, int(flags.value)


def gae(reward: np.ndarray, value: np.ndarray, gamma: float, lam: float):
    """Advantages and value targets of a rollout (FP32, the oracle's order):
    reward (T, n), value (T + 1, n).  Returns (adv, ret), each (T, n)."""
    lib = _load()
    r = np.ascontiguousarray(reward, dtype=np.float32)
    v = np.ascontiguousarray(value, dtype=np.float32)
    T, n = r.shape
    assert v.shape == (T + 1, n)
    adv = np.zeros((T, n), np.float32)
    ret = np.zeros((T, n), np.float32)
    rc = lib.oracle_gae(T, n, _f(r), _f(v), ctypes.c_float(gamma), ctypes.c_float(lam), _f(adv),
                        _f(ret))
    if rc != 0:
        raise ValueError("oracle rejected the call (rc=%d)" % rc)
    return adv, ret


def apply(params: dict, state: np.ndarray, actions: np.ndarray):
    """Apply actions only; returns (new_state, flags)."""
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float32).copy()
    act = np.ascontiguousarray(actions, dtype=np.int32)
    flags = ctypes.c_uint32(0)
    rc = lib.oracle_apply(ctypes.byref(_params(params)), st.shape[0], _f(st), _i(act),
                          ctypes.byref(flags))
    if rc != 0:
        raise ValueError("oracle rejected parameters (rc=%d)" % rc)
    return st, int(flags.value)


def observe_rows(params: dict, state: np.ndarray, rows: np.ndarray, threads: int = 0):
    """Observation of the agents in ``rows`` only, over all N agents of the
    (already moved) ``state``.  Returns (obs_rows, reward_rows, coll_rows)."""
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float32)
    idx = np.ascontiguousarray(rows, dtype=np.int32)
    m = idx.shape[0]
    D = obs_dim(params)
    obs = np.zeros((m, D), np.float32)
    rew = np.zeros(m, np.float32)
    coll = np.zeros(m, np.int32)
    rc = lib.oracle_observe_rows(ctypes.byref(_params(params)), st.shape[0], _f(st), m, _i(idx),
                                 _f(obs), _f(rew), _i(coll), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected parameters (rc=%d)" % rc)
    return obs, rew, coll


def sincos(theta: float):
    """The oracle's deterministic FP32 (cos, sin)."""
    lib = _load()
    c = ctypes.c_float(0.0)
    s = ctypes.c_float(0.0)
    lib.oracle_sincos(ctypes.c_float(theta), ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def diamond(x: float, y: float) -> float:
    return _load().oracle_diamond(ctypes.c_float(x), ctypes.c_float(y))


def max_threads() -> int:
    return os.cpu_count() or 1
