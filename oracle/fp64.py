"""Double-precision restatements -- TEST INFRASTRUCTURE, NOT THE PRODUCT PATH.

Two independent references used by the tests:

* ``reevaluate``: the flock observation, collisions and reward (arXiv
  2207.03945, Section 4.1, Eq. 1, Fig. 3, Fig. 4) in float64 with true
  angles (``atan2``), true distances (``hypot``) and exact minimum-image
  wrapping.  It shares no formula with the FP32 oracle's pseudo-angle,
  rotation or wrap code, so it pins those: every decision (in range,
  collision, sector) must agree except for pairs within a small tolerance of
  a boundary, which it reports as ambiguous.

* ``mlp_forward``: the shared policy network of Section 5 (two hidden
  layers of 64 with tanh) in float64, 18 -> 64 -> 64 -> 9 as the fused
  policy uses it, on given weights and observations.

Numpy only; nothing here imports the CUDA product package.
"""
from __future__ import annotations

import math

import numpy as np


def reevaluate(params: dict, state: np.ndarray, rows=None, tol_r: float = 1e-5,
               tol_a: float = 2e-5):
    """Observation of the (already moved) ``state`` in float64.

    Returns a dict with, per evaluated row: ``cnt`` (m, v) int sector counts,
    ``mind`` (m, v) nearest distance per sector (view radius when empty),
    ``coll`` (m,) int, ``reward`` (m,) float64, ``absf`` (m,) float64 sum of
    |f_ij| (the scale of the reward's rounding error), and ``ambiguous`` (m,)
    bool: the row has a pair within ``tol_r`` (relative) of the view or
    collision distance, or within ``tol_a`` radians of a sector edge."""
    st = np.asarray(state, dtype=np.float64)
    n = st.shape[0]
    L = float(np.float32(params["side"]))
    rv = float(np.float32(params["view_radius"]))
    dr2 = 2.0 * float(np.float32(params["agent_radius"]))
    P = float(np.float32(params["collision_penalty"]))
    v = int(params["num_segments"])
    fov32 = np.float32(params["fov"])
    full = fov32 == np.float32(2.0 * math.pi)
    fov = 2.0 * math.pi if full else float(fov32)
    width = fov / v
    rows = np.arange(n) if rows is None else np.asarray(rows)
    m = len(rows)
    cnt = np.zeros((m, v), np.int64)
    mind = np.full((m, v), rv)
    coll = np.zeros(m, np.int64)
    reward = np.zeros(m)
    absf = np.zeros(m)
    amb = np.zeros(m, bool)
    x, y, th = st[:, 0], st[:, 1], st[:, 2]
    for r, i in enumerate(rows):
        dx = x - x[i]
        dy = y - y[i]
        dx = dx - L * np.round(dx / L)
        dy = dy - L * np.round(dy / L)
        d = np.hypot(dx, dy)
        d[i] = np.inf
        inr = d < rv
        near_edge = np.abs(d - rv) < tol_r * rv
        if dr2 > 0:
            near_edge |= np.abs(d - dr2) < tol_r * max(dr2, 1e-30)
        if np.any(near_edge):
            amb[r] = True
        di = d[inr]
        col = di < dr2
        f = np.where(col, -P, (rv - di) / (rv - dr2))
        coll[r] = int(col.sum())
        reward[r] = float(f.sum())
        absf[r] = float(np.abs(f).sum())
        # direction of each in-range neighbour, measured counter-clockwise
        # from the start edge of the field of view (heading - fov/2)
        phi = np.arctan2(dy[inr], dx[inr])
        start = th[i] - 0.5 * fov
        alpha = np.mod(phi - start, 2.0 * math.pi)
        coincident = (dx[inr] == 0) & (dy[inr] == 0)
        seen = (~coincident) & (alpha < fov)
        k = np.floor(alpha / width).astype(np.int64)
        edge = alpha / width
        dist_edge = np.abs(edge - np.round(edge)) * width
        if np.any(dist_edge[~coincident] < tol_a) or np.any(
                np.abs(alpha[~coincident] - 2.0 * math.pi) < tol_a):
            amb[r] = True
        for kk, dd in zip(k[seen], di[seen]):
            kk = min(int(kk), v - 1)
            cnt[r, kk] += 1
            if dd < mind[r, kk]:
                mind[r, kk] = dd
    return {"cnt": cnt, "mind": mind, "coll": coll, "reward": reward, "absf": absf,
            "ambiguous": amb, "rows": rows}


def apply_fp64(params: dict, state: np.ndarray, actions: np.ndarray) -> np.ndarray:
    """Section 4.1's action update in float64 with the library cosine/sine:
    clamp the speed, turn, wrap the heading into [0, 2pi), move, wrap."""
    st = np.asarray(state, dtype=np.float64).copy()
    L = float(np.float32(params["side"]))
    a = np.asarray(actions).astype(np.int64)
    a = np.where((a < 0) | (a >= 9), 4, a)
    turn = (a // 3 - 1) * float(np.float32(params["turn_step"]))
    acc = (a % 3 - 1) * float(np.float32(params["speed_step"]))
    s = np.clip(st[:, 3] + acc, float(np.float32(params["speed_min"])),
                float(np.float32(params["speed_max"])))
    th = np.mod(st[:, 2] + turn, 2.0 * math.pi)
    x = np.mod(st[:, 0] + s * np.cos(th), L)
    y = np.mod(st[:, 1] + s * np.sin(th), L)
    return np.stack([x, y, th, s], axis=1)


def mlp_forward(weights: dict, obs: np.ndarray) -> np.ndarray:
    """Policy logits in float64: tanh(W1 x + b1) -> tanh(W2 h + b2) -> W3 h + b3.

    weights: W1 (64, 18), b1 (64,), W2 (64, 64), b2 (64,), W3 (9, 64), b3 (9,)
    (any float dtype; taken at their exact values).  obs: (N, 18)."""
    x = np.asarray(obs, dtype=np.float64)
    W1 = np.asarray(weights["W1"], np.float64)
    W2 = np.asarray(weights["W2"], np.float64)
    W3 = np.asarray(weights["W3"], np.float64)
    b1 = np.asarray(weights["b1"], np.float64)
    b2 = np.asarray(weights["b2"], np.float64)
    b3 = np.asarray(weights["b3"], np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3


def greedy(logits: np.ndarray) -> np.ndarray:
    """Greedy action: the lowest index among the largest logits."""
    return np.argmax(logits, axis=1).astype(np.int32)
