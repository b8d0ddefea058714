"""C-ABI checks that need no GPU: the library loads, exports every function
include/flock.h declares, validates parameters, and derives the same
constants as the oracle (each side computes its own)."""
import ctypes
import os
import re

import numpy as np
import pytest

import flock_inputs as fi
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_2207_03945_gb300 as F
    return F


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_exports_every_declared_symbol():
    F = _lib()
    lib = ctypes.CDLL(F.lib_path)
    names = declared_functions()
    assert "env_step" in names and "env_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_match_inputs_module():
    F = _lib()
    assert F.flock_default_params(100.0) == fi.default_params(100.0)


def test_obs_dim_and_workspace():
    F = _lib()
    p = fi.default_params(fi.side_for(50000))
    assert F.flock_obs_dim(p) == 18
    b = F.flock_workspace_bytes(p, 50000)
    assert 50000 * 36 < b < 50000 * 200
    assert F.flock_workspace_bytes(p, 0) > 0


def test_invalid_params_rejected():
    F = _lib()
    for bad in ({"view_radius": 0.0}, {"agent_radius": 3.0}, {"num_segments": 0},
                {"num_segments": 129}, {"fov": 7.0}, {"side": 9.0}, {"speed_max": -1.0},
                {"side": float("nan")}):
        with pytest.raises(F.FlockError):
            F.flock_derive(dict(fi.default_params(100.0), **bad))
    with pytest.raises(F.FlockError):
        F.flock_workspace_bytes(fi.default_params(100.0), -1)
    with pytest.raises(F.FlockError):
        F.flock_derive(fi.default_params(100.0), {"stencil": 3})
    # a square just over 2 d_v wide still has a cell list (one or two cells per side)
    assert F.flock_derive(fi.default_params(10.5))["cells_per_side"] == 2
    assert F.flock_derive(fi.default_params(10.5), {"stencil": 2})["cells_per_side"] == 4
    with pytest.raises(F.FlockError):
        F.flock_workspace_bytes(fi.default_params(100.0), 10, {"block": 48})


@pytest.mark.parametrize("over", [{}, {"fov": fi.FULL_FOV}, {"num_segments": 5},
                                  {"num_segments": 128, "fov": 3.0}, {"agent_radius": 0.0},
                                  {"collision_penalty": 0.375}, {"view_radius": 7.3}])
def test_derived_constants_equal_oracle(over):
    F = _lib()
    p = fi.default_params(fi.side_for(5000), **over)
    a = F.flock_derive(p)
    b = oracle.derive(p)
    pairs = [("side", "L"), ("half_side", "HL"), ("view_radius", "RV"), ("rv2", "RV2"),
             ("rc2", "RC2"), ("inv_span", "INV_SPAN"), ("two_pi", "TWO_PI"),
             ("cos_half_fov", "CF"), ("sin_half_fov", "SF"), ("speed_min", "SMIN"),
             ("speed_max", "SMAX"), ("turn", "DT"), ("accel", "DS"), ("edge", "T"),
             ("v", "v"), ("full_circle", "full"), ("k_exp", "K"), ("penalty_fixed", "PK"),
             ("nmax", "NMAX")]
    for ka, kb in pairs:
        assert a[ka] == b[kb], (ka, a[ka], b[kb])


def test_cell_geometry():
    F = _lib()
    for n, nc in ((1000, 19), (5000, 44), (50000, 141), (100000, 199)):
        d = F.flock_derive(fi.default_params(fi.side_for(n)))
        assert d["cells_per_side"] == nc
        # cells are at least the view radius wide
        assert d["side"] / d["cells_per_side"] >= 5.0
    d2 = F.flock_derive(fi.default_params(fi.side_for(50000)), {"stencil": 2})
    assert d2["cells_per_side"] == 282 and d2["stencil"] == 2


def test_obs_layouts():
    F = _lib()
    p = fi.default_params(100.0, num_segments=128)
    assert F.flock_obs_dim(p) == 258
    p["obs_layout"] = 1
    assert F.flock_obs_dim(p) == 129
    assert F.flock_obs_dim(fi.paper_params(16000)) == 129
    p["obs_layout"] = 2
    with pytest.raises(F.FlockError):
        F.flock_obs_dim(p)


def test_set_rows_argument_checks():
    """The row-range form of the batch set rejects, before any call into the
    library, ranges outside the arena, mismatched lengths, dicts in place of
    parameter structs and a host arena."""
    F = _lib()
    torch = pytest.importorskip("torch")
    from paper_2207_03945_gb300 import _abi
    p = _abi.params_from_dict(fi.default_params(100.0))
    arena = torch.zeros((100, 4))
    with pytest.raises(F.FlockError):  # rows 90..109 of 100
        F.env_batch_set_rows(None, [p], [20], arena, [90])
    with pytest.raises(F.FlockError):
        F.env_batch_set_rows(None, [p, p], [20], arena, [0])
    with pytest.raises(F.FlockError):
        F.env_batch_set_rows(None, [fi.default_params(100.0)], [20], arena, [0])
    with pytest.raises(F.FlockError):
        F.env_batch_set_rows(None, [p], [20], torch.zeros((100, 3)), [0])
    with pytest.raises(F.FlockError):  # a host tensor is not device memory
        F.env_batch_set_rows(None, [p], [20], arena, [0])


def test_binding_refuses_host_memory_and_bad_shapes():
    """No CPU fallback: every device entry point of the binding rejects host
    tensors (and wrong dtypes or shapes) with FlockError before it reaches
    the library; the host-buffer step rejects arrays of the wrong shape."""
    import types
    F = _lib()
    torch = pytest.importorskip("torch")
    env = types.SimpleNamespace(handle=None, n=10, obs_dim=18)
    a = torch.zeros(10, dtype=torch.int32)
    o = torch.zeros((10, 18))
    r = torch.zeros(10)
    c = torch.zeros(10, dtype=torch.int32)
    calls = [
        lambda: F.env_step(env, a, o, r, c),
        lambda: F.env_step_continuous(env, torch.zeros((10, 2)), o, r, c),
        lambda: F.env_rollout(env, torch.zeros((4, 10), dtype=torch.int32),
                              torch.zeros((4, 10, 18)), torch.zeros((4, 10)),
                              torch.zeros((4, 10), dtype=torch.int32)),
        lambda: F.env_rollout(env, None, o, r, c),
        lambda: F.flock_gae(torch.zeros((4, 10)), torch.zeros((5, 10)), 0.99, 0.95,
                            torch.zeros((4, 10)), torch.zeros((4, 10))),
        lambda: F.env_set_types(env, torch.zeros(10, dtype=torch.uint8)),
        lambda: F.env_get_state(env, torch.zeros((10, 4))),
        lambda: F.env_step_host(env, np.zeros(9, np.int32), np.zeros((10, 18), np.float32),
                                np.zeros(10, np.float32), np.zeros(10, np.int32)),
        lambda: F.env_step_host(env, np.zeros(10, np.int32), np.zeros((10, 17), np.float32),
                                np.zeros(10, np.float32), np.zeros(10, np.int32)),
        lambda: F.env_step_host(env, torch.zeros(10, dtype=torch.int64), o, r, c),
    ]
    for k, call in enumerate(calls):
        with pytest.raises(F.FlockError):
            call()


def test_bound_host_step_makes_the_same_call(monkeypatch):
    """env_step_host_bind checks the buffers once and then issues exactly the
    env_step_host call (same handle, same four host pointers) per step; it
    refuses to run once the environment is closed."""
    import types
    F = _lib()
    torch = pytest.importorskip("torch")
    from paper_2207_03945_gb300 import _abi
    calls = []
    fake = types.SimpleNamespace(env_step_host=lambda *a: calls.append(a) or 0)
    monkeypatch.setattr(_abi, "lib", fake)
    env = types.SimpleNamespace(handle=12345, n=10, obs_dim=18)
    bufs = (np.zeros(10, np.int32), np.zeros((10, 18), np.float32), np.zeros(10, np.float32),
            torch.zeros(10, dtype=torch.int32))
    F.env_step_host(env, *bufs)
    step = F.env_step_host_bind(env, *bufs)
    step()
    step()
    assert len(calls) == 3
    ref = [calls[0][0]] + [p.value for p in calls[0][1:]]
    for c in calls[1:]:
        assert [c[0]] + [p.value for p in c[1:]] == ref
    assert ref[1] == bufs[0].ctypes.data and ref[4] == bufs[3].data_ptr()
    env.handle = None
    with pytest.raises(F.FlockError):
        step()
    with pytest.raises(F.FlockError):  # float64 observations are refused
        F.env_step_host_bind(env, bufs[0], np.zeros((10, 18)), bufs[2], bufs[3])
