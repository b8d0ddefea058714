"""The decomposition of one square over several ranks (slab.py) on the CPU:
each band's compute is the oracle on the band's own and ghost agents, so
these tests check the decomposition itself -- the bands, which agents
migrate, which become ghosts, the exchange and the stitching -- against the
oracle's step of the undivided square, bit for bit (states, observations,
rewards, collisions).  Bands emulated in one process (LocalExchange), and
two real ranks exchanging over gloo (DistExchange).  The CUDA band compute
is tested on the GPU (test_gpu_slab.py)."""
import os
import socket
import sys

import numpy as np
import pytest

import flock_inputs as fi
import oracle

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2207_03945_gb300 import slab  # noqa: E402


class OracleBand:
    """Band compute by the oracle (test infrastructure): apply moves the own
    agents; observe gives the own agents' outputs over own and ghosts."""
    action_dtype = torch.int32

    def __init__(self, params):
        self.params = params

    def apply(self, state, actions):
        st, flags = oracle.apply(self.params, state.numpy(), actions.numpy())
        assert flags == 0
        state.copy_(torch.from_numpy(st))

    def observe(self, own, ghosts):
        st = torch.cat([own, ghosts]).numpy()
        rows = np.arange(own.shape[0], dtype=np.int32)
        o, r, c = oracle.observe_rows(self.params, st, rows)
        return torch.from_numpy(o), torch.from_numpy(r), torch.from_numpy(c)


def stitch(parts, n, d):
    obs = np.full((n, d), np.nan, np.float32)
    rew = np.full(n, np.nan, np.float32)
    coll = np.full(n, -1, np.int32)
    seen = np.zeros(n, np.int64)
    for ids, o, r, c in parts:
        ids = ids.numpy()
        obs[ids], rew[ids], coll[ids] = o.numpy(), r.numpy(), c.numpy()
        seen[ids] += 1
    assert np.all(seen == 1), "every agent observed by exactly one band"
    return obs, rew, coll


def states_of(bands_, n):
    st = np.full((n, 4), np.nan, np.float32)
    for b in bands_:
        st[b.ids.numpy()] = b.st.numpy()
    return st


def run_emulated(n, world, steps, seed, side=None):
    side = side or fi.side_for(n)
    p = fi.default_params(side)
    nc, halo, invw = slab.geometry(p)
    st0 = fi.initial_state(n, side, seed)
    acts = fi.random_actions(n, steps, seed)
    bands_ = [slab.SlabBand(nc, halo, invw, b, world, OracleBand(p)) for b in range(world)]
    for b in bands_:
        b.load(np.arange(n), st0)
    ex = slab.LocalExchange()
    d = oracle.obs_dim(p)
    # initial observation, then steps
    got = [stitch(slab.step_local(bands_, ex), n, d)]
    ref_st, o, r, c, _ = oracle.step(p, st0, None, threads=0)
    ref = [(o, r, c)]
    sts = [states_of(bands_, n)]
    ref_sts = [ref_st]
    for t in range(steps):
        got.append(stitch(slab.step_local(bands_, ex, torch.from_numpy(acts[t])), n, d))
        sts.append(states_of(bands_, n))
        ref_st, o, r, c, _ = oracle.step(p, ref_st, acts[t], threads=0)
        ref.append((o, r, c))
        ref_sts.append(ref_st)
    return got, ref, sts, ref_sts


@pytest.mark.parametrize("world", [2, 3, 4])
def test_emulated_bands_equal_the_undivided_square(world):
    got, ref, sts, ref_sts = run_emulated(3000, world, 4, 17)
    for t, (g, r) in enumerate(zip(got, ref)):
        for k in range(3):
            assert np.array_equal(g[k], r[k]), (world, t, k)
        assert np.array_equal(sts[t], ref_sts[t]), (world, t)


def test_agents_cross_band_edges_every_step():
    """Speeds at the maximum and a small square: agents migrate between
    bands and ghosts change every step."""
    n = 800
    side = fi.side_for(n)
    p = fi.default_params(side)
    nc, halo, invw = slab.geometry(p)
    st0 = fi.initial_state(n, side, 5)
    st0[:, 3] = np.float32(1.0)  # full speed
    bands_ = [slab.SlabBand(nc, halo, invw, b, 2, OracleBand(p)) for b in range(2)]
    for b in bands_:
        b.load(np.arange(n), st0)
    ex = slab.LocalExchange()
    slab.step_local(bands_, ex)
    acts = fi.random_actions(n, 6, 5)
    owners = [set(b.ids.tolist()) for b in bands_]
    ref_st = st0
    moved = 0
    for t in range(6):
        parts = slab.step_local(bands_, ex, torch.from_numpy(acts[t]))
        ref_st, o, r, c, _ = oracle.step(p, ref_st, acts[t], threads=0)
        obs, rew, coll = stitch(parts, n, oracle.obs_dim(p))
        assert np.array_equal(obs, o) and np.array_equal(rew, r) and np.array_equal(coll, c)
        now = [set(b.ids.tolist()) for b in bands_]
        moved += len(now[0] - owners[0]) + len(now[1] - owners[1])
        owners = now
        assert sum(b.ghost_ids.numel() for b in bands_) > 0
    assert moved > 0


def test_band_geometry_and_rows():
    assert slab.bands(10, 2, 1) == [(0, 5), (5, 10)]
    assert slab.bands(10, 3, 1) == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        slab.bands(4, 4, 2)  # bands thinner than the halo
    rows = np.arange(10)
    assert slab.in_rows(rows, -1, 6, 10).tolist() == [True] * 6 + [False] * 3 + [True]
    p = fi.default_params(fi.side_for(5000))
    nc, halo, invw = slab.geometry(p)
    y = fi.initial_state(5000, p["side"], 1)[:, 1]
    r1 = slab.cell_rows(y, invw, nc)
    r2 = slab.cell_rows(torch.from_numpy(y), invw, nc).numpy()
    assert np.array_equal(r1, r2) and r1.min() >= 0 and r1.max() < nc


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, steps, seed, q):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "oracle"), os.path.join(ROOT, "tests")]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import flock_inputs as fi_
    from paper_2207_03945_gb300 import slab as slab_
    from test_slab import OracleBand as OB
    p = fi_.default_params(fi_.side_for(n))
    nc, halo, invw = slab_.geometry(p)
    band = slab_.SlabBand(nc, halo, invw, rank, world, OB(p))
    band.load(np.arange(n), fi_.initial_state(n, p["side"], seed))
    ex = slab_.DistExchange(device="cpu")
    acts = fi_.random_actions(n, steps, seed)
    out = [tuple(x.numpy() for x in slab_.step_dist(band, ex))]
    for t in range(steps):
        out.append(tuple(x.numpy() for x in
                         slab_.step_dist(band, ex, torch.from_numpy(acts[t]))))
    q.put((rank, out, band.ids.numpy(), band.st.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_over_gloo_equal_the_undivided_square():
    import torch.multiprocessing as mp
    n, steps, seed, world = 2500, 3, 23, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, steps, seed, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = fi.default_params(fi.side_for(n))
    d = oracle.obs_dim(p)
    st, o, r, c, _ = oracle.step(p, fi.initial_state(n, p["side"], seed), None, threads=0)
    acts = fi.random_actions(n, steps, seed)
    for t in range(steps + 1):
        if t:
            st, o, r, c, _ = oracle.step(p, st, acts[t - 1], threads=0)
        parts = [tuple(torch.from_numpy(np.asarray(x)) for x in res[b][1][t])
                 for b in range(world)]
        obs, rew, coll = stitch(parts, n, d)
        assert np.array_equal(obs, o) and np.array_equal(rew, r) and np.array_equal(coll, c), t
    final = np.full((n, 4), np.nan, np.float32)
    for b in range(world):
        final[res[b][2]] = res[b][3]
    assert np.array_equal(final, st)
