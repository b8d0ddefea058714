"""Initial states drawn from a seed (flock_seed_states).

CPU: the oracle's restatement (oracle/seeds.py, SplitMix64 from its published
definition) is pinned by its outputs run backwards through the finaliser
(each step inverted on its own) to the counter they came from, and by what a
uniform draw must satisfy: every value in its range, the moments of U[0, 1),
flat histograms, flat histograms of pairs (the three columns of an agent and
consecutive agents: a generator without its finaliser, a bare Weyl sequence,
fails these), and determinism by seed.
GPU: the kernel equals the oracle bit for bit, and bad arguments are refused
before any launch."""
import numpy as np
import pytest

import seeds

N = 200_000


def _unit(st, side):
    two_pi = float(seeds.TWO_PI_F32)
    return np.stack([st[:, 0] / side, st[:, 1] / side, st[:, 2] / two_pi], axis=1).astype(np.float64)


@pytest.mark.parametrize("side", [1.0, 3.0, 223.6068, 10000.0])
def test_ranges_and_speed(side):
    st = seeds.seed_states(N, side, 12345, speed=0.75)
    L = np.float32(side)
    assert st.dtype == np.float32 and st.shape == (N, 4)
    assert (st[:, 0] >= 0).all() and (st[:, 0] < L).all()
    assert (st[:, 1] >= 0).all() and (st[:, 1] < L).all()
    assert (st[:, 2] >= 0).all() and (st[:, 2] < seeds.TWO_PI_F32).all()
    assert (st[:, 3] == np.float32(0.75)).all()


def test_moments_of_a_uniform_draw():
    u = _unit(seeds.seed_states(N, 100.0, 7), 100.0)
    # standard error of the mean 0.29 / sqrt(N) = 6.5e-4: 6 sigma
    assert np.abs(u.mean(axis=0) - 0.5).max() < 4e-3
    assert np.abs(u.var(axis=0) - 1.0 / 12.0).max() < 2e-3


def test_histograms_are_flat():
    u = _unit(seeds.seed_states(N, 100.0, 11), 100.0)
    bins = 64
    e = N / bins
    for c in range(3):
        h = np.bincount(np.minimum((u[:, c] * bins).astype(int), bins - 1), minlength=bins)
        chi2 = ((h - e) ** 2 / e).sum()
        assert chi2 < bins + 6 * np.sqrt(2 * bins), (c, chi2)  # 63 degrees of freedom


@pytest.mark.parametrize("pair", ["x-y", "y-theta", "x-next-x"])
def test_pairs_are_flat(pair):
    """Two-dimensional histograms: a generator whose outputs follow each other
    by a fixed step (no finaliser) puts its pairs on a few lines."""
    u = _unit(seeds.seed_states(N, 100.0, 13), 100.0)
    a, b = {"x-y": (u[:, 0], u[:, 1]), "y-theta": (u[:, 1], u[:, 2]),
            "x-next-x": (u[:-1, 0], u[1:, 0])}[pair]
    g = 16
    cells = np.minimum((a * g).astype(int), g - 1) * g + np.minimum((b * g).astype(int), g - 1)
    h = np.bincount(cells, minlength=g * g)
    e = len(a) / (g * g)
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < g * g + 6 * np.sqrt(2 * g * g), chi2
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.015


def test_bare_weyl_sequence_fails_the_pair_test():
    """The pair test has teeth: the same draw without the finaliser (the
    seed plus multiples of the golden-ratio step) is far from flat."""
    k = np.arange(2 * N, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(13) + (k + np.uint64(1)) * seeds.GAMMA
    u = seeds.unit24(z).astype(np.float64)
    a, b = u[0::2], u[1::2]
    g = 16
    cells = np.minimum((a * g).astype(int), g - 1) * g + np.minimum((b * g).astype(int), g - 1)
    h = np.bincount(cells, minlength=g * g)
    e = len(a) / (g * g)
    assert ((h - e) ** 2 / e).sum() > 10 * g * g


def _unxorshift(y: int, s: int) -> int:
    """Inverse of z -> z ^ (z >> s) on 64-bit words: the top s bits are
    unchanged, each further block of s bits follows from the ones above it."""
    x = y
    for _ in range(64 // s + 1):
        x = y ^ (x >> s)
    return x


def _unfinalise(z: int) -> int:
    """The finaliser of each output run backwards, step by step: the xor-shifts
    by 31, 27 and 30 undone as above, the multiplications by the two odd
    constants undone by their inverses modulo 2^64."""
    M = 1 << 64
    z = _unxorshift(z, 31)
    z = (z * pow(0x94D049BB133111EB, -1, M)) % M
    z = _unxorshift(z, 27)
    z = (z * pow(0xBF58476D1CE4E5B9, -1, M)) % M
    return _unxorshift(z, 30)


def test_outputs_invert_to_the_weyl_sequence():
    """Each output run backwards through the finaliser gives back the counter
    seed + (k + 1) * 0x9E3779B97F4A7C15: a dropped or altered step of the
    forward mix (a shift, a multiplication, the counter) fails this."""
    rng = np.random.Generator(np.random.PCG64(5))
    for seed in [0, 1, 2 ** 63 + 5, 2 ** 64 - 1] + [int(x) for x in rng.integers(0, 2 ** 63, 4)]:
        k = np.arange(50, dtype=np.uint64) * np.uint64(97)
        out = seeds.splitmix64(seed, k)
        for kk, z in zip(k.tolist(), out.tolist()):
            assert _unfinalise(int(z)) == (seed + (kk + 1) * 0x9E3779B97F4A7C15) % (1 << 64)


def test_seed_determines_the_draw():
    a = seeds.seed_states(1000, 50.0, 99)
    assert np.array_equal(a, seeds.seed_states(1000, 50.0, 99))
    b = seeds.seed_states(1000, 50.0, 100)
    assert (a[:, :3] != b[:, :3]).mean() > 0.99
    # agent i's row does not depend on n
    assert np.array_equal(seeds.seed_states(10, 50.0, 99), a[:10])
    assert seeds.seed_states(0, 50.0, 99).shape == (0, 4)


@pytest.mark.gpu
@pytest.mark.parametrize("n", [1, 255, 256, 257, 100_001])
@pytest.mark.parametrize("side,seed", [(1.0, 0), (223.6068, 1), (707.1068, 2 ** 63 + 5),
                                       (10000.0, 2 ** 64 - 1)])
def test_gpu_equals_oracle(n, side, seed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2207_03945_gb300 as F
    st = torch.full((n, 4), -1.0, dtype=torch.float32, device="cuda")
    F.flock_seed_states(st, side, seed, speed=0.5)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), seeds.seed_states(n, side, seed, 0.5))


@pytest.mark.gpu
def test_gpu_refuses_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2207_03945_gb300 as F
    st = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    for side in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(F.FlockError):
            F.flock_seed_states(st, side, 1)
    with pytest.raises(F.FlockError):
        F.flock_seed_states(st, 10.0, 1, speed=float("nan"))
    buf = torch.zeros(41, dtype=torch.float32, device="cuda")
    with pytest.raises(F.FlockError):  # 4 bytes off a 16-byte boundary
        F.flock_seed_states(buf[1:].view(10, 4), 10.0, 1)
    assert (buf == 0).all()
    F.flock_seed_states(st[:0], 10.0, 1)  # no agents: nothing to do
