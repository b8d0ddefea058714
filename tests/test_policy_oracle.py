"""Pins of the float64 policy oracle (oracle/fp64.py mlp_forward), CPU only.

* closed form: with W1 = W2 = 0 the hidden layers are tanh(b1) and tanh(b2),
  so the logits are W3 tanh(b2) + b3 whatever the input;
* tanh is odd: with zero biases the network is odd, f(-x) = -f(x);
* small weights: tanh(z) = z + O(z^3), so the network tends to the linear map
  W3 W2 W1 x; a transposed or dropped layer breaks this limit;
* greedy actions take the lowest index among equal logits."""
import math

import numpy as np

import flock_inputs as fi
import fp64


def _w(seed, scale):
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = dict(fi.POLICY_SHAPES)
    return {k: rng.standard_normal(s) * scale for k, s in shapes.items()}


def test_closed_form_with_zero_inner_weights():
    w = _w(1, 0.3)
    w["W1"][:] = 0.0
    w["W2"][:] = 0.0
    x = np.random.Generator(np.random.PCG64(2)).standard_normal((5, 18)) * 4
    want = w["W3"] @ np.tanh(w["b2"]) + w["b3"]
    got = fp64.mlp_forward(w, x)
    assert np.allclose(got, np.broadcast_to(want, got.shape), rtol=0, atol=1e-14)
    # and a single hand-computed value: one active unit
    w = {k: np.zeros(s) for k, s in fi.POLICY_SHAPES}
    w["b2"][3] = math.atanh(0.5)
    w["W3"][7, 3] = 2.0
    w["b3"][7] = 0.25
    assert abs(fp64.mlp_forward(w, np.zeros((1, 18)))[0, 7] - 1.25) < 1e-15


def test_odd_symmetry_without_biases():
    w = _w(3, 0.2)
    for b in ("b1", "b2", "b3"):
        w[b][:] = 0.0
    x = np.random.Generator(np.random.PCG64(4)).standard_normal((50, 18)) * 3
    assert np.allclose(fp64.mlp_forward(w, -x), -fp64.mlp_forward(w, x), atol=1e-14)


def test_small_weight_linear_limit():
    w = _w(5, 1.0)
    for b in ("b1", "b2", "b3"):
        w[b][:] = 0.0
    x = np.random.Generator(np.random.PCG64(6)).standard_normal((20, 18))
    eps = 1e-3
    ws = {k: v * (eps if k.startswith("W") else 1.0) for k, v in w.items()}
    lin = (w["W3"] @ w["W2"] @ w["W1"] @ x.T).T * eps ** 3
    got = fp64.mlp_forward(ws, x)
    # relative deviation is O(eps^2)
    assert np.abs(got - lin).max() <= 1e-4 * np.abs(lin).max()
    # a transposed middle layer is far from the limit
    wt = dict(ws)
    wt["W2"] = ws["W2"].T.copy()
    assert np.abs(fp64.mlp_forward(wt, x) - lin).max() > 0.1 * np.abs(lin).max()


def test_greedy_ties_take_lowest_index():
    lg = np.array([[0.0, 1.0, 1.0, -1.0], [2.0, 2.0, 2.0, 2.0]])
    assert list(fp64.greedy(lg)) == [1, 0]


def test_weight_blob_layout():
    w = fi.policy_weights(0)
    blob = fi.bf16_bits_to_f32(w["blob"])
    assert w["blob"].shape == (5961,)
    off = 0
    for name, shape in fi.POLICY_SHAPES:
        size = int(np.prod(shape))
        assert np.array_equal(blob[off:off + size].reshape(shape), w[name])
        off += size
    # bf16 rounding: every value has a zero low half
    assert np.all((w["W2"].view(np.uint32) & 0xFFFF) == 0)
    assert abs(float(np.std(w["W2"])) - 0.1) < 0.01
