"""Initial states from a seed -- TEST INFRASTRUCTURE, NOT THE PRODUCT PATH.

Only ``tests/`` may import this module (nothing in the product imports it).
It restates, in numpy, what ``flock_seed_states`` (include/flock.h) draws:
the paper leaves initial conditions open, and the library's reading is
uniform positions on the square, uniform headings and one speed.  The random
numbers are SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written here from that published
definition: output k of seed S is the finaliser applied to
S + (k + 1) * 0x9E3779B97F4A7C15 (all arithmetic modulo 2^64).

Pins (``tests/test_seed_states.py``): every output, run backwards through the
finaliser step by step (the xor-shifts and the multiplications by odd
constants each inverted on its own), gives back its counter; and the draws
have the properties of a uniform draw (ranges, moments, flat histograms of
single columns and of pairs, which a bare counter without the finaliser
fails).  The constants themselves are those of the published definition as
written here; no published output of the generator was at hand offline to
compare against.  The CUDA path must equal this module bit for bit.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
TWO_PI_F32 = np.float32(2.0 * np.pi)


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """Outputs k (uint64 array, counted from 0) of SplitMix64 seeded with seed."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k.astype(np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))


def unit24(z: np.ndarray) -> np.ndarray:
    """The top 24 bits of each output as a float32 in [0, 1) (exact)."""
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def seed_states(n: int, side: float, seed: int, speed: float = 0.5) -> np.ndarray:
    """(n, 4) float32 rows (x, y, theta, s): agent i takes outputs 4i, 4i + 1 and
    4i + 2; x = min(u * side, side-) with one FP32 rounding, y likewise, theta =
    min(u * (float)2pi, (float)2pi-), s = speed."""
    L = np.float32(side)
    k = np.arange(n, dtype=np.uint64) * np.uint64(4)
    ux, uy, ut = (unit24(splitmix64(seed, k + np.uint64(j))) for j in range(3))
    below_l = np.nextafter(L, np.float32(0))
    below_2pi = np.nextafter(TWO_PI_F32, np.float32(0))
    x = np.minimum(ux * L, below_l)
    y = np.minimum(uy * L, below_l)
    th = np.minimum(ut * TWO_PI_F32, below_2pi)
    s = np.full(n, np.float32(speed), np.float32)
    return np.ascontiguousarray(np.stack([x, y, th, s], axis=1).astype(np.float32))
