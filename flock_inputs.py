"""Seeded synthetic inputs for the flock environment.

This module is shared by the tests, the benchmark and the smoke check; it
feeds the CUDA library and the CPU oracle the same bytes.  It holds none of
the environment's arithmetic: only parameter presets, uniform and Gaussian
draws (numpy PCG64), and the shapes of the workloads of arXiv 2207.03945
(Section 4.1 flock, Section 5 benchmark protocol) as this project
instantiates them:

* agents uniform on the periodic square at density 0.1 per unit area (1,000
  agents on a 100 x 100 square; the side grows as sqrt(N / 1000));
* headings uniform in [0, 2pi), speed 0.5;
* actions uniform over 3 turns x 3 speed changes;
* batched instances with agent counts log-uniform in [100, 20,000];
* policy weights Gaussian(0, 0.1), rounded to bfloat16;
* serving sessions with Poisson arrivals, log-uniform agent counts and
  uniform episode lengths.
"""
from __future__ import annotations

import math

import numpy as np

DENSITY = 0.1
TWO_PI_F32 = np.float32(2.0 * math.pi)


def side_for(n_agents: int, density: float = DENSITY) -> float:
    """Side of the square that holds n_agents at the given density, as float32."""
    return float(np.float32(math.sqrt(n_agents / density)))


def default_params(side: float, **overrides) -> dict:
    """Flock parameters: view radius 5, agent radius 0.5 (collide below 1.0),
    penalty 1, speed in [0, 1] with steps of 0.25, turns of pi/8, 8 sectors,
    field of view 250 degrees.  Keyword overrides replace any field."""
    p = {
        "side": float(np.float32(side)),
        "view_radius": 5.0,
        "fov": float(np.float32(250.0 * math.pi / 180.0)),
        "agent_radius": 0.5,
        "collision_penalty": 1.0,
        "speed_min": 0.0,
        "speed_max": 1.0,
        "speed_step": 0.25,
        "turn_step": float(np.float32(math.pi / 8.0)),
        "num_segments": 8,
        "obs_layout": 0,
        "kind": 0,
    }
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return p


FULL_FOV = float(TWO_PI_F32)


def _below(x: np.ndarray, hi: np.float32) -> np.ndarray:
    """Replace values that rounding pushed to hi or above by the float below hi."""
    lim = np.nextafter(np.float32(hi), np.float32(0))
    return np.where(x >= hi, lim, x).astype(np.float32)


def initial_state(n: int, side: float, seed: int, speed: float = 0.5) -> np.ndarray:
    """(n, 4) float32 rows (x, y, theta, s): x, y ~ U[0, side), theta ~ U[0, 2pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = np.float32(side)
    x = _below((rng.random(n) * float(L)).astype(np.float32), L)
    y = _below((rng.random(n) * float(L)).astype(np.float32), L)
    th = _below((rng.random(n) * 2.0 * math.pi).astype(np.float32), TWO_PI_F32)
    s = np.full(n, speed, np.float32)
    return np.ascontiguousarray(np.stack([x, y, th, s], axis=1).astype(np.float32))


def random_actions(n: int, steps: int, seed: int) -> np.ndarray:
    """(steps, n) int32 actions uniform over {0, ..., 8}."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.integers(0, 9, size=(steps, n), dtype=np.int32)


def paper_params(n_agents: int, **overrides) -> dict:
    """The paper's own flock variant (Section 4.1 and Section 5): 128 sectors,
    a view distance of a tenth of the side, field of view 250 degrees, the
    view-only observation (obs_layout 1: 128 distances and the speed), on the
    square of density 0.1 (side sqrt(n / 0.1)); agent radius, speeds and the
    action ranges as in default_params.  The paper does not give the density;
    0.1 keeps the collision rate of the other workloads."""
    side = side_for(n_agents)
    p = default_params(side, view_radius=float(np.float32(side / 10.0)), num_segments=128,
                       obs_layout=1)
    p.update(overrides)
    return p


def tag_params(n_agents: int, **overrides) -> dict:
    """The tag environment as the paper runs it (Section 4.2, Section 5): two
    colour channels of 64 sectors (a 128-value view), view a tenth of the
    side, field of view 250 degrees, density 0.1; speeds in [0, 1], turns up
    to pi/8 per step."""
    side = side_for(n_agents)
    p = default_params(side, view_radius=float(np.float32(side / 10.0)), num_segments=64,
                       kind=1)
    p.update(overrides)
    return p


def random_cont_actions(n: int, steps: int, seed: int, a_max: float, t_max: float,
                        over: float = 1.25) -> np.ndarray:
    """(steps, n, 2) float32 continuous actions (acceleration, rotation),
    uniform in [-over * a_max, over * a_max] x [-over * t_max, over * t_max];
    with over > 1 some fall outside the ranges (they are clamped)."""
    rng = np.random.Generator(np.random.PCG64(seed + 15485863))
    u = rng.random((steps, n, 2)) * 2.0 - 1.0
    scale = np.array([a_max, t_max], np.float64) * over
    return (u * scale).astype(np.float32)


def tag_types(n: int, seed: int, chaser_fraction: float = 0.1) -> np.ndarray:
    """(n,) uint8 agent types for the tag environment: 1 (chaser) for a
    random chaser_fraction of the agents (Section 5: a tenth are chasers),
    0 (runner) for the rest."""
    rng = np.random.Generator(np.random.PCG64(seed + 32452843))
    t = np.zeros(n, np.uint8)
    t[rng.permutation(n)[:int(round(chaser_fraction * n))]] = 1
    return t


def tag_actions(n: int, steps: int, seed: int, s_max: float, t_max: float,
                over: float = 1.25) -> np.ndarray:
    """(steps, n, 2) float32 tag actions (speed, rotation), uniform in
    [-0.25 s_max, over * s_max] x [-over * t_max, over * t_max] (some clamp)."""
    rng = np.random.Generator(np.random.PCG64(seed + 49979687))
    u = rng.random((steps, n, 2))
    spd = -0.25 * s_max + u[..., 0] * (over + 0.25) * s_max
    rot = (u[..., 1] * 2.0 - 1.0) * over * t_max
    return np.stack([spd, rot], axis=-1).astype(np.float32)


def batch_sizes(n_inst: int = 256, lo: int = 100, hi: int = 20000, seed: int = 0) -> list:
    """Agent counts round(exp(U[ln lo, ln hi])) for a batch of instances."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    u = rng.random(n_inst)
    return [int(round(math.exp(math.log(lo) + t * (math.log(hi) - math.log(lo))))) for t in u]


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = b + 0x7FFF + ((b >> 16) & 1)
    return (b >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


POLICY_SHAPES = (("W1", (64, 18)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
                 ("W3", (9, 64)), ("b3", (9,)))


def policy_weights(seed: int = 0, std: float = 0.1) -> dict:
    """Gaussian(0, std) weights and biases for 18 -> 64 -> 64 -> 9, rounded to
    bfloat16.  Returns float32 arrays (exact bf16 values) plus ``blob``: all
    5,961 bf16 bit patterns concatenated in the order W1, b1, W2, b2, W3, b3
    (row-major, each W as [out][in])."""
    rng = np.random.Generator(np.random.PCG64(seed + 31337))
    out = {}
    parts = []
    for name, shape in POLICY_SHAPES:
        w = (rng.standard_normal(shape) * std).astype(np.float32)
        bits = to_bf16_bits(w)
        out[name] = bf16_bits_to_f32(bits).reshape(shape)
        parts.append(bits.reshape(-1))
    out["blob"] = np.concatenate(parts)
    return out


def session_stream(rate: float, duration: float, seed: int, n_lo: int = 500,
                   n_hi: int = 50000, len_lo: int = 100, len_hi: int = 2000) -> list:
    """Poisson arrivals over ``duration`` seconds: list of (t_arrival, n_agents,
    episode_steps, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed + 65537))
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        u = float(rng.random())
        n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
        steps = int(rng.integers(len_lo, len_hi + 1))
        out.append((t, n, steps, int(rng.integers(0, 2**31 - 1))))
    return out
