"""GPU tests of the batched step (one persistent kernel for many instances).

Each instance of a mixed batch must equal the oracle run on that instance
alone (bit-exact: state, observation, collisions, reward), and equal the
single-environment path; the active set may change between steps; the
grid-barrier wait bound turns a stalled barrier into FLOCK_ERR_TIMEOUT.
Mode 2 runs every phase in one persistent launch; mode 3 bins in the
persistent launch and scans neighbours in a second one; mode 4 bins with
three kernels (apply and count, scan, scatter) over all instances, then
scans neighbours in a fourth launch."""
import numpy as np
import pytest

import flock_inputs as fi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2207_03945_gb300 as F  # noqa: E402

DEV = torch.device("cuda:0")


def make_instances(sizes, seed, **over):
    out = []
    for k, n in enumerate(sizes):
        side = max(fi.side_for(n), 12.0)
        p = fi.default_params(side, **over)
        st = fi.initial_state(n, side, seed + k)
        out.append((p, n, st))
    return out


def batch_for(insts, tuning=None):
    mc = sum(F.flock_instance_cells(p, tuning) for p, _, _ in insts)
    na = sum(n for _, n, _ in insts)
    return F.FlockBatch(max(len(insts), 1), na, max(mc, 1), 2 * insts[0][0]["num_segments"] + 2,
                        device=DEV, tuning=tuning)


MODES = pytest.mark.parametrize("mode", [2, 3, 4])
BARRIER_MODES = pytest.mark.parametrize("mode", [2, 3])  # the forms with grid barriers


@MODES
def test_mixed_batch_matches_oracle_per_instance(mode):
    sizes = [100, 1, 0, 2500, 731, 5000, 64, 33, 12000]
    insts = make_instances(sizes, 100)
    b = batch_for(insts, {"mode": mode})
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1] * len(sizes))
    steps = 4
    rng = np.random.Generator(np.random.PCG64(5))
    acts = [rng.integers(0, 9, size=sum(sizes), dtype=np.int32) for _ in range(steps + 1)]
    ref_st = [st.copy() for _, _, st in insts]
    for t in range(steps + 1):
        obs, rew, coll = b.step(torch.from_numpy(acts[t]).to(DEV))
        torch.cuda.synchronize()
        o_all, r_all, c_all = obs.cpu().numpy(), rew.cpu().numpy(), coll.cpu().numpy()
        for k, (p, n, _) in enumerate(insts):
            off = b.offsets[k]
            a = None if t == 0 else acts[t][off:off + n]
            st2, o, r, c, _ = oracle.step(p, ref_st[k], a, threads=0)
            ref_st[k] = st2
            assert np.array_equal(o_all[off:off + n], o), (t, k)
            assert np.array_equal(r_all[off:off + n], r), (t, k)
            assert np.array_equal(c_all[off:off + n], c), (t, k)
            assert np.array_equal(states[k].cpu().numpy(), st2), (t, k)
    assert b.error() == 0
    b.close()


def test_batch_equals_single_environment():
    sizes = [4000, 300, 9000]
    insts = make_instances(sizes, 200, fov=fi.FULL_FOV)
    b = batch_for(insts)
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1, 1, 1])
    acts = fi.random_actions(sum(sizes), 3, 7)
    outs = []
    b.step(torch.from_numpy(acts[0]).to(DEV))
    for t in range(1, 3):
        obs, rew, coll = b.step(torch.from_numpy(acts[t]).to(DEV))
        outs.append((obs.cpu().numpy().copy(), rew.cpu().numpy().copy()))
    for k, (p, n, st) in enumerate(insts):
        off = b.offsets[k]
        env = F.FlockEnv(p, n, device=DEV)
        env.reset(torch.from_numpy(st).to(DEV))
        for t in range(1, 3):
            o, r, _ = env.step(torch.from_numpy(np.ascontiguousarray(acts[t][off:off + n])).to(DEV))
            assert np.array_equal(o.cpu().numpy(), outs[t - 1][0][off:off + n])
            assert np.array_equal(r.cpu().numpy(), outs[t - 1][1][off:off + n])
        env.close()
    b.close()


def test_set_rows_equals_set():
    """The active set given as row ranges of one arena (the serving loop's
    form, instances in an order and at rows unlike their flattened order)
    steps exactly like the same set given as one tensor per instance."""
    sizes = [3000, 150, 7000]
    insts = make_instances(sizes, 210)
    rows = [9000, 0, 1000]  # arena rows of each instance
    arena = torch.zeros((16000, 4), dtype=torch.float32, device=DEV)
    for (p, n, st), r in zip(insts, rows):
        arena[r:r + n] = torch.from_numpy(st).to(DEV)
    b1, b2 = batch_for(insts), batch_for(insts)
    b1.set([p for p, _, _ in insts], sizes, [torch.from_numpy(st).to(DEV) for _, _, st in insts],
           reset=[1, 1, 1])
    from paper_2207_03945_gb300 import _abi
    b2.set_rows([_abi.params_from_dict(p) for p, _, _ in insts], sizes, arena, rows,
                reset=[1, 1, 1])
    assert b1.offsets == b2.offsets and b1.n_total == b2.n_total
    acts = fi.random_actions(sum(sizes), 3, 21)
    for t in range(3):
        a = torch.from_numpy(acts[t]).to(DEV)
        o1, r1, c1 = (x.cpu().numpy().copy() for x in b1.step(a))
        o2, r2, c2 = (x.cpu().numpy().copy() for x in b2.step(a))
        assert np.array_equal(o1, o2) and np.array_equal(r1, r2) and np.array_equal(c1, c2), t
    assert b1.error() == 0 and b2.error() == 0
    b1.close()
    b2.close()


@MODES
def test_active_set_changes_between_steps(mode):
    """Sessions leave and join between steps; the graph is reused (mode 3:
    updated in place for the new chunk count)."""
    sizes = [500, 800, 1200]
    insts = make_instances(sizes, 300)
    extra = make_instances([700], 400)[0]
    b = F.FlockBatch(4, 4000, 20000, 18, device=DEV, tuning={"mode": mode})
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1, 1, 1])
    b.step(torch.zeros(sum(sizes), dtype=torch.int32, device=DEV))
    ref = [oracle.step(p, st, None)[0] for p, _, st in insts]
    # instance 1 leaves, a new one joins (observed first), the others continue
    xs = torch.from_numpy(extra[2]).to(DEV)
    keep = [insts[0], insts[2], extra]
    kst = [states[0], states[2], xs]
    b.set([p for p, _, _ in keep], [n for _, n, _ in keep], kst, reset=[0, 0, 1])
    a = fi.random_actions(sum(n for _, n, _ in keep), 1, 9)[0]
    obs, rew, coll = b.step(torch.from_numpy(a).to(DEV))
    torch.cuda.synchronize()
    exp = [oracle.step(insts[0][0], ref[0], a[:500]),
           oracle.step(insts[2][0], ref[2], a[500:1700]),
           oracle.step(extra[0], extra[2], None)]
    o = obs.cpu().numpy()
    assert np.array_equal(o[:500], exp[0][1])
    assert np.array_equal(o[500:1700], exp[1][1])
    assert np.array_equal(o[1700:2400], exp[2][1])
    assert np.array_equal(xs.cpu().numpy(), extra[2])  # observed, not moved
    assert b.error() == 0
    b.close()


def test_batch_stencil_5x5_and_generic_segments():
    sizes = [1500, 2500]
    for tuning, over in (({"stencil": 2}, {}), ({"stencil": 1}, {"num_segments": 5})):
        insts = make_instances(sizes, 500, **over)
        b = batch_for(insts, tuning)
        states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
        b.set([p for p, _, _ in insts], sizes, states)
        a = fi.random_actions(sum(sizes), 1, 3)[0]
        obs, rew, coll = b.step(torch.from_numpy(a).to(DEV))
        torch.cuda.synchronize()
        for k, (p, n, st) in enumerate(insts):
            off = b.offsets[k]
            _, o, r, c, _ = oracle.step(p, st, a[off:off + n])
            assert np.array_equal(obs[off:off + n].cpu().numpy(), o)
            assert np.array_equal(rew[off:off + n].cpu().numpy(), r)
        b.close()


def test_mixed_segment_counts_rejected():
    b = F.FlockBatch(2, 100, 1000, 18, device=DEV)
    p1 = fi.default_params(40.0)
    p2 = fi.default_params(40.0, num_segments=6)
    s = torch.zeros((10, 4), device=DEV)
    with pytest.raises(F.FlockError):
        b.set([p1, p2], [10, 10], [s, s])
    with pytest.raises(F.FlockError):  # more agents than the batch holds
        b.set([p1], [101], [torch.zeros((101, 4), device=DEV)])
    b.close()


@BARRIER_MODES
def test_barrier_wait_bound_reports_timeout_and_recovers(mode):
    """With the wait bound at zero every barrier gives up at once: the step
    returns with FLOCK_ERR_TIMEOUT latched and no hang (mode 3: the
    neighbour launch sees the bit and leaves the step unobserved); after
    restoring the bound the next steps are correct again."""
    sizes = [3000, 2000]
    insts = make_instances(sizes, 600)
    b = batch_for(insts, {"mode": mode})
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1, 1])
    F.env_batch_set_spin_limit(b.batch, 0)
    b.step(torch.zeros(sum(sizes), dtype=torch.int32, device=DEV))
    err = b.error()
    if F.env_batch_get_launch(b.batch)[0] > 1:
        assert err & F.FLOCK_ERR_TIMEOUT
    # recover: restore the bound, re-load the states, step again
    F.env_batch_set_spin_limit(b.batch, 1 << 22)
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1, 1])
    a = fi.random_actions(sum(sizes), 2, 1)
    b.step(torch.from_numpy(a[0]).to(DEV))
    obs, rew, coll = b.step(torch.from_numpy(a[1]).to(DEV))
    torch.cuda.synchronize()
    for k, (p, n, st) in enumerate(insts):
        off = b.offsets[k]
        _, o, r, c, _ = oracle.step(p, st, a[1][off:off + n])
        assert np.array_equal(obs[off:off + n].cpu().numpy(), o)
    assert b.error() == 0
    b.close()


@MODES
def test_benchmark_mix_sampled_rows(mode):
    """The 256-instance mix of the benchmark (agent counts log-uniform in
    [100, 20000]): every state bit-exact after two steps, and the outputs of
    sampled rows of every instance bit-exact against the oracle."""
    sizes = fi.batch_sizes(256, 100, 20000, 0)
    insts = make_instances(sizes, 1000)
    b = batch_for(insts, {"mode": mode})
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1] * len(sizes))
    b.step(torch.zeros(sum(sizes), dtype=torch.int32, device=DEV))
    a = fi.random_actions(sum(sizes), 1, 11)[0]
    obs, rew, coll = b.step(torch.from_numpy(a).to(DEV))
    torch.cuda.synchronize()
    o_all, r_all, c_all = obs.cpu().numpy(), rew.cpu().numpy(), coll.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(2))
    for k, (p, n, st) in enumerate(insts):
        off = b.offsets[k]
        st2, _ = oracle.apply(p, st, a[off:off + n])
        assert np.array_equal(states[k].cpu().numpy(), st2), k
        rows = rng.choice(n, size=min(n, 16), replace=False).astype(np.int32)
        o, r, c = oracle.observe_rows(p, st2, rows)
        assert np.array_equal(o_all[off + rows], o), k
        assert np.array_equal(r_all[off + rows], r), k
        assert np.array_equal(c_all[off + rows], c), k
    assert b.error() == 0
    b.close()


@pytest.mark.parametrize("tuning", [{"mode": 3, "block": 64}, {"mode": 3, "block": 256},
                                    {"mode": 4, "block": 64}, {"mode": 4, "block": 256},
                                    {"mode": 4, "stencil": 2, "block": 128},
                                    {"mode": 4, "lanes": 1}, {"mode": 4, "lanes": 2},
                                    {"mode": 3, "lanes": 4, "stencil": 2}],
                         ids=lambda d: "-".join("%s%s" % kv for kv in d.items()))
def test_neighbour_launch_block_sizes(tuning):
    """Every block size of the separate neighbour launch (the autotuner's
    choices) gives the oracle's bits, on a mix with empty and one-agent
    instances."""
    sizes = [900, 0, 1, 4100, 37, 2600]
    insts = make_instances(sizes, 700)
    b = batch_for(insts, tuning)
    states = [torch.from_numpy(st).to(DEV) for _, _, st in insts]
    b.set([p for p, _, _ in insts], sizes, states, reset=[1] * len(sizes))
    assert F.env_batch_get_launch(b.batch)[0] > 0
    b.step(torch.zeros(sum(sizes), dtype=torch.int32, device=DEV))
    a = fi.random_actions(sum(sizes), 2, 7)
    ref = [st.copy() for _, _, st in insts]
    for t in range(2):
        obs, rew, coll = b.step(torch.from_numpy(a[t]).to(DEV))
        torch.cuda.synchronize()
        for k, (p, n, _) in enumerate(insts):
            off = b.offsets[k]
            ref[k], o, r, c, _ = oracle.step(p, ref[k], a[t][off:off + n])
            assert np.array_equal(obs[off:off + n].cpu().numpy(), o), (t, k)
            assert np.array_equal(rew[off:off + n].cpu().numpy(), r), (t, k)
            assert np.array_equal(coll[off:off + n].cpu().numpy(), c), (t, k)
            assert np.array_equal(states[k].cpu().numpy(), ref[k]), (t, k)
    assert b.error() == 0
    b.close()
