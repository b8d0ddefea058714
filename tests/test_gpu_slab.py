"""The slab environment on the GPU: one square decomposed into bands, each
band's compute by the library's slab calls (env_slab_apply,
env_slab_observe through slab.CudaBand), the bands emulated one after the
other on one device with the in-memory exchange (no kernel waits for
another band).  The stitched result must be the oracle's step of the
undivided square, bit for bit, for several band counts, both stencils and
lane counts (the ghosts' rows in the output loop are skipped by every lane
layout)."""
import numpy as np
import pytest

import flock_inputs as fi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_03945_gb300 import slab  # noqa: E402

DEV = torch.device("cuda:0")


def stitch(parts, n, d):
    obs = np.full((n, d), np.nan, np.float32)
    rew = np.full(n, np.nan, np.float32)
    coll = np.full(n, -1, np.int32)
    seen = np.zeros(n, np.int64)
    for ids, o, r, c in parts:
        ids = ids.cpu().numpy()
        obs[ids], rew[ids], coll[ids] = o.cpu().numpy(), r.cpu().numpy(), c.cpu().numpy()
        seen[ids] += 1
    assert np.all(seen == 1)
    return obs, rew, coll


@pytest.mark.parametrize("world,tuning", [
    (2, None), (3, None), (4, {"lanes": 1}), (2, {"lanes": 32}),
    (3, {"stencil": 2, "lanes": 2})], ids=lambda v: str(v))
def test_cuda_bands_equal_the_undivided_square(world, tuning):
    n, steps, seed = 6000, 3, 41
    p = fi.default_params(fi.side_for(n))
    stencil = (tuning or {}).get("stencil", 1)
    nc, halo, invw = slab.geometry(p, stencil)
    st0 = fi.initial_state(n, p["side"], seed)
    acts = fi.random_actions(n, steps, seed)
    lo_hi = slab.bands(nc, world, halo)
    backends = [slab.CudaBand(p, nc, halo, lo, hi, device=DEV, n_max=2 * n // world,
                              tuning=tuning) for lo, hi in lo_hi]
    bands_ = [slab.SlabBand(nc, halo, invw, b, world, backends[b], device=DEV)
              for b in range(world)]
    for b in bands_:
        b.load(np.arange(n), st0)
    ex = slab.LocalExchange()
    d = oracle.obs_dim(p)
    st, o, r, c, _ = oracle.step(p, st0, None, threads=0)
    got = stitch(slab.step_local(bands_, ex), n, d)
    for k, ref in enumerate((o, r, c)):
        assert np.array_equal(got[k], ref), ("reset", k)
    for t in range(steps):
        parts = slab.step_local(bands_, ex, torch.from_numpy(acts[t]).to(DEV))
        st, o, r, c, _ = oracle.step(p, st, acts[t], threads=0)
        got = stitch(parts, n, d)
        for k, ref in enumerate((o, r, c)):
            assert np.array_equal(got[k], ref), (t, k)
        final = np.full((n, 4), np.nan, np.float32)
        for b in bands_:
            final[b.ids.cpu().numpy()] = b.st.cpu().numpy()
        assert np.array_equal(final, st), t
    for be in backends:
        assert be.error() == 0
        be.close()


def test_slab_rejects_bad_geometry():
    p = fi.default_params(fi.side_for(2000))
    nc, halo, _ = slab.geometry(p)
    from paper_2207_03945_gb300 import FlockError, FlockSlab
    with pytest.raises(FlockError):
        FlockSlab(p, 100, 0, 2, device=DEV)          # fewer rows than the stencil
    with pytest.raises(FlockError):
        FlockSlab(p, 100, nc, 5, device=DEV)         # first row outside the grid
    with pytest.raises(FlockError):
        FlockSlab(p, 100, 0, 5, device=DEV, tuning={"mode": 1})  # tiles: whole squares only
