"""The autotuner: every candidate launch shape gives the same bits (the
tuner checks this before keeping the fastest), and its choice is cached."""
import pytest

import flock_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_03945_gb300 import autotune as at  # noqa: E402


def test_single_instance_candidates_identical_and_cached(tmp_path):
    n = 20000
    side = fi.side_for(n)
    p = fi.default_params(side)
    st = fi.initial_state(n, side, 3)
    cache = str(tmp_path / "tune.json")
    tuning, report = at.autotune(p, st, steps=3, warmup=2, cache=cache)
    assert len(report) >= 8
    assert all(same for _, _, same in report), report
    assert tuning["mode"] in (1, 2) and tuning["stencil"] in (1, 2)
    again, _ = at.autotune(p, st, steps=3, warmup=2, cache=cache)
    assert again == tuning


def test_batch_stencil_choice():
    sizes = [3000, 800, 12000]
    params = [fi.default_params(fi.side_for(n)) for n in sizes]
    states = [fi.initial_state(n, fi.side_for(n), k) for k, n in enumerate(sizes)]
    tuning, report = at.autotune_batch(params, sizes, states, steps=2, warmup=2)
    assert len(report) == len(at.BATCH_CANDIDATES) and all(same for _, _, same in report)
    assert tuning["stencil"] in (1, 2) and tuning["mode"] in (2, 3, 4)
    # the separate neighbour launch's block size is part of the search
    assert {c.get("block") for c, _, _ in report} >= {64, 128, 256}
