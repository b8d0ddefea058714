"""ctypes declarations of include/flock.h and the loader of libflock.so.

Loading fails loudly when the library is missing: there is no fallback."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflock.so")

FLOCK_OK = 0
FLOCK_EINVAL = -1
FLOCK_ENOSPACE = -2
FLOCK_ECUDA = -3
FLOCK_ERR_ACTION = 1
FLOCK_ERR_STATE = 2
FLOCK_ERR_TIMEOUT = 4
FLOCK_ERR_OVERFLOW = 8
FLOCK_ERR_BOUNDS = 16
MAX_SEGMENTS = 128
STATIC_MAX_AGENTS = 65536
STATIC_MAX_CELLS = 32768

_NAMES = {FLOCK_EINVAL: "FLOCK_EINVAL", FLOCK_ENOSPACE: "FLOCK_ENOSPACE",
          FLOCK_ECUDA: "FLOCK_ECUDA"}


class FlockError(RuntimeError):
    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


class FlockParams(ctypes.Structure):
    _fields_ = [("side", ctypes.c_float), ("view_radius", ctypes.c_float),
                ("fov", ctypes.c_float), ("agent_radius", ctypes.c_float),
                ("collision_penalty", ctypes.c_float), ("speed_min", ctypes.c_float),
                ("speed_max", ctypes.c_float), ("speed_step", ctypes.c_float),
                ("turn_step", ctypes.c_float), ("num_segments", ctypes.c_int),
                ("obs_layout", ctypes.c_int), ("kind", ctypes.c_int)]


class FlockTuning(ctypes.Structure):
    _fields_ = [("stencil", ctypes.c_int), ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int),
                ("block", ctypes.c_int), ("mode", ctypes.c_int), ("lanes", ctypes.c_int)]


class FlockDerived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("side", "half_side", "view_radius", "rv2", "rc2", "inv_span", "two_pi",
                 "cos_half_fov", "sin_half_fov", "speed_min", "speed_max")] + [
        ("turn", ctypes.c_float * 3), ("accel", ctypes.c_float * 3),
        ("edge", ctypes.c_float * (MAX_SEGMENTS + 1)),
        ("v", ctypes.c_int), ("full_circle", ctypes.c_int), ("k_exp", ctypes.c_int),
        ("penalty_fixed", ctypes.c_int64), ("nmax", ctypes.c_int64),
        ("cells_per_side", ctypes.c_int), ("stencil", ctypes.c_int),
        ("inv_cell_width", ctypes.c_float)]


PARAM_KEYS = [k for k, _ in FlockParams._fields_]


def params_from_dict(p: dict) -> FlockParams:
    floats = [k for k, t in FlockParams._fields_ if t is ctypes.c_float]
    return FlockParams(*(float(p[k]) for k in floats), int(p["num_segments"]),
                       int(p.get("obs_layout", 0)), int(p.get("kind", 0)))


def params_to_dict(p: FlockParams) -> dict:
    return {k: getattr(p, k) for k in PARAM_KEYS}


def tuning_from_dict(t):
    if t is None:
        return None
    return FlockTuning(int(t.get("stencil", 0)), int(t.get("tile_w", 0)),
                       int(t.get("tile_h", 0)), int(t.get("block", 0)), int(t.get("mode", 0)),
                       int(t.get("lanes", 0)))


def derived_to_dict(d: FlockDerived) -> dict:
    out = {}
    for k, _ in FlockDerived._fields_:
        v = getattr(d, k)
        out[k] = list(v) if not isinstance(v, (int, float)) else v
    out["edge"] = out["edge"][1:d.v + 1]
    return out


def _load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("%s is not built; run __graft_entry__.build() "
                          "-- there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    P = ctypes.POINTER(FlockParams)
    T = ctypes.POINTER(FlockTuning)
    sigs = {
        "flock_default_params": [ctypes.c_float, P],
        "flock_obs_dim": [P],
        "flock_workspace_bytes": [P, T, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "flock_derive": [P, T, ctypes.POINTER(FlockDerived)],
        "env_create": [P, T, ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "env_reset": [vp, vp, vp, vp, vp],
        "env_step": [vp, vp, vp, vp, vp],
        "env_step_continuous": [vp, vp, vp, vp, vp],
        "env_rollout": [vp, ctypes.c_int, vp, vp, vp, vp, vp],
        "flock_seed_states": [vp, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_uint64, vp],
        "flock_gae": [ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_float, ctypes.c_float, vp, vp,
                      vp],
        "env_step_host": [vp, vp, vp, vp, vp],
        "env_step_policy": [vp, vp, vp, vp, vp, vp, vp],
        "env_get_state": [vp, vp],
        "env_set_state": [vp, vp],
        "env_set_types": [vp, vp],
        "env_get_error": [vp, ctypes.POINTER(ctypes.c_uint32)],
        "env_get_derived": [vp, ctypes.POINTER(FlockDerived)],
        "env_get_tuning": [vp, T],
        "env_set_timing": [vp, ctypes.c_int],
        "env_get_phase_times": [vp, ctypes.POINTER(ctypes.c_float)],
        "flock_instance_cells": [P, T, ctypes.POINTER(ctypes.c_int)],
        "flock_batch_workspace_bytes": [ctypes.c_int, ctypes.c_int, ctypes.c_int, T,
                                        ctypes.POINTER(ctypes.c_size_t)],
        "env_batch_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, T, vp, ctypes.c_size_t,
                             vp, ctypes.POINTER(vp)],
        "env_batch_set": [vp, ctypes.c_int, P, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)],
        "env_batch_step": [vp, vp, vp, vp, vp],
        "env_batch_get_error": [vp, ctypes.POINTER(ctypes.c_uint32)],
        "env_batch_set_spin_limit": [vp, ctypes.c_uint],
        "env_batch_get_launch": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "env_batch_set_timing": [vp, ctypes.c_int],
        "env_batch_get_time": [vp, ctypes.POINTER(ctypes.c_float)],
        "flock_step_static": [P, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                              ctypes.POINTER(ctypes.c_uint32)],
        "flock_slab_workspace_bytes": [P, T, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_size_t)],
        "env_slab_create": [P, T, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t,
                            vp, ctypes.POINTER(vp)],
        "env_slab_apply": [vp, ctypes.c_int, vp, vp],
        "env_slab_observe": [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.env_destroy.argtypes = [vp]
    lib.env_destroy.restype = None
    lib.env_batch_destroy.argtypes = [vp]
    lib.env_batch_destroy.restype = None
    lib.flock_last_cuda_error.argtypes = []
    lib.flock_last_cuda_error.restype = ctypes.c_char_p
    return lib


lib = _load()
DEBUG_LIB_PATH = os.path.join(HERE, "libflock_debug.so")


def use_library(path):
    """Makes the binding call the library at `path` (for example the
    FLOCK_DEBUG build, libflock_debug.so, whose index checks latch
    FLOCK_ERR_BOUNDS); returns the previous library handle, which
    restore_library puts back.  Handles created by one library must be used
    and destroyed with that library."""
    global lib
    prev = lib
    lib = _load(path)
    return prev


def restore_library(handle):
    global lib
    lib = handle


def check(rc):
    if rc == FLOCK_OK:
        return
    msg = _NAMES.get(rc, "error %d" % rc)
    if rc == FLOCK_ECUDA:
        msg += ": " + lib.flock_last_cuda_error().decode(errors="replace")
    raise FlockError(msg, rc)
