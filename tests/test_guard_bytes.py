"""Guard bytes around every buffer the library writes: the workspace, the
outputs and (for a batch) the instance states live inside larger device
allocations whose margins hold a fixed byte pattern.  After resets and steps
of single environments (discrete and continuous actions, a ragged agent
count, the policy step, the host-buffer step writing page-locked host
buffers) and of batches in all three launch forms, every margin is unchanged: no
write lands outside the buffers handed over through the C ABI.  (An
out-of-bounds check that needs no sanitizer; nothing here can fault.)"""
import numpy as np
import pytest

import flock_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402
from paper_2207_03945_gb300 import _abi  # noqa: E402

DEV = torch.device("cuda:0")
PAD = 4096    # margin on each side, bytes (keeps the 256-byte alignment)
PATTERN = 0xA5


class Guarded:
    """nbytes of device memory (host=True: page-locked host memory) with PAD
    guard bytes on each side."""

    def __init__(self, nbytes, host=False):
        self.nbytes = int(nbytes)
        if host:
            self.buf = torch.full((self.nbytes + 2 * PAD,), PATTERN, dtype=torch.uint8).pin_memory()
        else:
            self.buf = torch.full((self.nbytes + 2 * PAD,), PATTERN, dtype=torch.uint8, device=DEV)
        self.inner = self.buf[PAD:PAD + self.nbytes]

    def as_(self, dtype, shape):
        return self.inner.view(dtype).view(*shape)

    def intact(self):
        g = torch.cat([self.buf[:PAD], self.buf[PAD + self.nbytes:]])
        return bool((g == PATTERN).all().item())


@pytest.mark.parametrize("case", ["discrete", "continuous"])
def test_single_environment_writes_stay_inside_its_buffers(case):
    if case == "discrete":
        n = 4999
        p = fi.default_params(fi.side_for(n))
    else:
        n = 2000
        p = fi.paper_params(n)
    d = F.flock_obs_dim(p)
    ws = Guarded(F.flock_workspace_bytes(p, n))
    go, gr, gc = Guarded(n * d * 4), Guarded(n * 4), Guarded(n * 4)
    obs, rew = go.as_(torch.float32, (n, d)), gr.as_(torch.float32, (n,))
    coll = gc.as_(torch.int32, (n,))
    env = F.env_create(p, n, ws.inner)
    F.env_reset(env, torch.from_numpy(fi.initial_state(n, p["side"], 31)).to(DEV), obs, rew, coll)
    if case == "discrete":
        acts = torch.from_numpy(fi.random_actions(n, 3, 31)).to(DEV)
        for t in range(3):
            F.env_step(env, acts[t], obs, rew, coll)
    else:
        acts = torch.from_numpy(fi.random_cont_actions(n, 3, 31, p["speed_step"],
                                                        p["turn_step"])).to(DEV)
        for t in range(3):
            F.env_step_continuous(env, acts[t].contiguous(), obs, rew, coll)
    torch.cuda.synchronize()
    assert F.env_get_error(env) == 0
    F.env_destroy(env)
    for g in (ws, go, gr, gc):
        assert g.intact()


@pytest.mark.parametrize("mode", [2, 3, 4])
def test_batch_writes_stay_inside_its_buffers(mode):
    sizes = [1500, 99, 4001]
    tuning = {"stencil": 1, "mode": mode}
    params = [fi.default_params(max(fi.side_for(n), 12.0)) for n in sizes]
    cells = sum(F.flock_instance_cells(p, tuning) for p in params)
    total = sum(sizes)
    ws = Guarded(F.flock_batch_workspace_bytes(len(sizes), total, cells, tuning))
    b = F.env_batch_create(len(sizes), total, cells, ws.inner, tuning=tuning)
    ga = Guarded(total * 16)
    arena = ga.as_(torch.float32, (total, 4))
    rows = list(np.cumsum([0] + sizes[:-1]))
    for (p, n), r in zip(zip(params, sizes), rows):
        arena[r:r + n] = torch.from_numpy(fi.initial_state(n, p["side"], 40 + r)).to(DEV)
    go, gr, gc = Guarded(total * 18 * 4), Guarded(total * 4), Guarded(total * 4)
    obs, rew = go.as_(torch.float32, (total, 18)), gr.as_(torch.float32, (total,))
    coll = gc.as_(torch.int32, (total,))
    F.env_batch_set_rows(b, [_abi.params_from_dict(p) for p in params], sizes, arena, rows,
                         reset=[1, 1, 1])
    acts = torch.from_numpy(fi.random_actions(total, 3, 41)).to(DEV)
    for t in range(3):
        F.env_batch_step(b, acts[t], obs, rew, coll)
        if t == 0:  # clear the reset flags after the observing step
            F.env_batch_set_rows(b, [_abi.params_from_dict(p) for p in params], sizes, arena,
                                 rows, reset=[0, 0, 0])
    torch.cuda.synchronize()
    assert F.env_batch_get_error(b) == 0
    F.env_batch_destroy(b)
    for g in (ws, ga, go, gr, gc):
        assert g.intact()


@pytest.mark.parametrize("lanes", [1, 2, 4, 32])
def test_policy_step_writes_stay_inside_its_buffers(lanes):
    n = 4999
    p = fi.default_params(fi.side_for(n))
    ws = Guarded(F.flock_workspace_bytes(p, n, {"lanes": lanes}))
    ga, gr, gc, gl, go = (Guarded(n * 4), Guarded(n * 4), Guarded(n * 4), Guarded(n * 36),
                          Guarded(n * 72))
    act = ga.as_(torch.int32, (n,))
    act.copy_(torch.from_numpy(fi.random_actions(n, 1, 35)[0]))
    rew, coll = gr.as_(torch.float32, (n,)), gc.as_(torch.int32, (n,))
    logits, obs = gl.as_(torch.float32, (n, 9)), go.as_(torch.float32, (n, 18))
    w = fi.policy_weights(7)
    blob = torch.from_numpy(w["blob"].view(np.int16)).to(DEV)
    env = F.env_create(p, n, ws.inner, tuning={"lanes": lanes})
    F.env_reset(env, torch.from_numpy(fi.initial_state(n, p["side"], 35)).to(DEV), obs, rew, coll)
    for _ in range(3):
        F.env_step_policy(env, blob, act, rew, coll, logits, obs)
    torch.cuda.synchronize()
    assert F.env_get_error(env) == 0
    F.env_destroy(env)
    for g in (ws, ga, gr, gc, gl, go):
        assert g.intact()


@pytest.mark.parametrize("n,tuning", [(4999, None), (4999, {"lanes": 32}), (120001, {"lanes": 1})])
def test_host_step_writes_stay_inside_its_host_buffers(n, tuning):
    """Page-locked host buffers with margins: the agent-order scan (or, with
    32 lanes, the copy kernel) writes only the rows it is given."""
    p = fi.default_params(fi.side_for(n))
    ws = Guarded(F.flock_workspace_bytes(p, n, tuning))
    go, gr, gc = Guarded(n * 72, True), Guarded(n * 4, True), Guarded(n * 4, True)
    ga = Guarded(n * 4, True)
    obs, rew = go.as_(torch.float32, (n, 18)), gr.as_(torch.float32, (n,))
    coll, act = gc.as_(torch.int32, (n,)), ga.as_(torch.int32, (n,))
    env = F.env_create(p, n, ws.inner, tuning=tuning)
    dobs = torch.empty((n, 18), dtype=torch.float32, device=DEV)
    drew = torch.empty(n, dtype=torch.float32, device=DEV)
    dcoll = torch.empty(n, dtype=torch.int32, device=DEV)
    F.env_reset(env, torch.from_numpy(fi.initial_state(n, p["side"], 37)).to(DEV), dobs, drew,
                dcoll)
    acts = fi.random_actions(n, 2, 37)
    for t in range(2):
        act.copy_(torch.from_numpy(acts[t]))
        F.env_step_host(env, act, obs, rew, coll)
    assert F.env_get_error(env) == 0
    F.env_destroy(env)
    for g in (ws, go, gr, gc, ga):
        assert g.intact()
