"""Pins of the FP64 warm-start network reference (oracle/mlp.py)."""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2407_14675_gb300 import workloads as W


def test_gelu_values_and_derivative():
    # GELU(z) = z Phi(z): Phi(1) = 0.841344746068543, Phi(0) = 1/2
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.841344746068543, abs=1e-15)
    assert mlp.gelu(np.array([-1.0]))[0] == pytest.approx(-(1 - 0.841344746068543), abs=1e-15)
    assert mlp.gelu(np.array([8.0]))[0] == pytest.approx(8.0, abs=1e-12)
    z = np.linspace(-4, 4, 81)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(z)).max() < 1e-8
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5


@pytest.mark.parametrize("sizes", [(4, 5, 6, 7, 3), (4, 256, 256, 256, 3)])
def test_backward_matches_central_differences(sizes):
    rng = np.random.default_rng(3)
    params = W.mlp_init_params(seed=5, sizes=sizes)
    X = rng.uniform(-1, 1, size=(6, 4))
    T = rng.uniform(-1, 1, size=(6, 3))
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, Y, T)
    h = 1e-6
    for li, layer in enumerate(params):
        for pi, P in enumerate(layer):
            flat = P.reshape(-1)
            idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
            for k in idx:
                old = flat[k]
                flat[k] = old + h
                lp = mlp.loss(mlp.forward(params, X)[0], T)
                flat[k] = old - h
                lm = mlp.loss(mlp.forward(params, X)[0], T)
                flat[k] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][pi].reshape(-1)[k]
                assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (li, pi, k)


def test_output_layer_is_linear_and_shapes():
    params = W.mlp_init_params(seed=1)
    X = np.zeros((3, 4))
    Y, cache = mlp.forward(params, X)
    assert Y.shape == (3, 3)
    assert [c[1].shape[1] for c in cache] == [256, 256, 256, 3]
    # the output is affine in the last hidden layer
    a3 = cache[3][0]
    assert np.allclose(Y, a3 @ params[3][0].T + params[3][1], atol=1e-14)


def test_adam_first_step_is_lr_times_sign():
    params = [[np.array([[1.0, -2.0]]), np.array([0.5])]]
    grads = [[np.array([[3.0, -0.25]]), np.array([-7.0])]]
    state = {}
    mlp.adam_step(params, grads, state, lr=1e-3)
    assert params[0][0] == pytest.approx(np.array([[1.0 - 1e-3, -2.0 + 1e-3]]), abs=1e-9)
    assert params[0][1] == pytest.approx(np.array([0.5 + 1e-3]), abs=1e-9)


def test_normalisation_maps_box_to_unit_cube():
    lo, hi = (0.95, -0.1, 0.85, 0.9), (1.15, 0.1, 1.1, 1.0)
    X = np.array([lo, hi, [(a + b) / 2 for a, b in zip(lo, hi)]])
    N = mlp.normalise_states(X, lo, hi)
    assert np.allclose(N, [[-1] * 4, [1] * 4, [0] * 4], atol=1e-12)


def test_bf16_rounding_pins():
    # values with at most 8 significant bits are exact; round to nearest even
    # at the midpoint between two BF16 neighbours; relative error <= 2^-8
    # (half a unit of the 8th significant bit; the FP32 step adds 2^-24)
    exact = np.array([0.0, 1.0, -1.5, 0.75, 2.0 ** -20, 3.0 * 2 ** 10, 255.0, -1.0 / 128])
    assert (mlp.bf16(exact) == exact).all()
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0                    # tie to even (1.0)
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6    # tie to even (up)
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(0).normal(size=10000) * 10.0 ** np.random.default_rng(1).uniform(-6, 6, 10000)
    r = mlp.bf16(x)
    assert (np.abs(r - x) <= (2.0 ** -8 + 2.0 ** -24) * np.abs(x)).all()
    assert (mlp.bf16(r) == r).all()


def test_bf16_reference_is_the_fp64_network_with_rounded_operands():
    # without the roundings (all values already representable) the BF16
    # reference is the FP64 network; with them it moves by O(2^-8) of scale
    rng = np.random.default_rng(4)
    params = W.mlp_init_params(seed=6)
    X = rng.uniform(-1, 1, size=(64, 4))
    T = rng.uniform(-1, 1, size=(64, 3))
    Y, cache = mlp.forward(params, X)
    Yb, cache_b = mlp.forward_bf16(params, X)
    scale = np.abs(Y).max()
    assert 0 < np.abs(Yb - Y).max() <= 2e-2 * scale
    g = mlp.backward(params, cache, Y, T)
    gb = mlp.backward_bf16(params, cache_b, Yb, T)
    for li in range(4):
        for pi in range(2):
            rel = np.linalg.norm(gb[li][pi] - g[li][pi]) / np.linalg.norm(g[li][pi])
            assert rel < 5e-2, (li, pi, rel)
    # a network whose operands are exactly representable: identical results
    params_r = [[mlp.bf16(Wt), mlp.bf16(bv)] for Wt, bv in params]
    Xr = mlp.bf16(X)
    Y1, c1 = mlp.forward(params_r, Xr)
    Y2, c2 = mlp.forward_bf16(params_r, Xr)
    # hidden activations still round, so compare the first layer's pre-activation
    assert np.array_equal(c1[0][1], c2[0][1])


def test_bf16_reference_rounds_exactly_the_documented_operands():
    # which operands the BF16-faithful reference rounds: the hidden activations
    # (inputs of layers 2-4), the weights of layers 2 and 3, and the hidden
    # pre-activation gradients; not the inputs, W1, W4 or the biases
    rng = np.random.default_rng(11)
    params = W.mlp_init_params(seed=12)
    X = rng.uniform(-1, 1, size=(16, 4))
    T = rng.uniform(-1, 1, size=(16, 3))
    Y, cache = mlp.forward_bf16(params, X)
    for li in (1, 2, 3):
        a_in = cache[li][0]
        assert np.array_equal(mlp.bf16(a_in), a_in), li
    assert not np.array_equal(mlp.bf16(cache[0][0]), cache[0][0])       # inputs stay FP32

    def with_rounded(layers):
        return [[mlp.bf16(Wt) if li in layers else Wt, bv] for li, (Wt, bv) in enumerate(params)]

    # pre-rounding W2 and W3 changes nothing, forward or backward
    Y23, c23 = mlp.forward_bf16(with_rounded((1, 2)), X)
    assert np.array_equal(Y23, Y)
    g = mlp.backward_bf16(params, cache, Y, T)
    g23 = mlp.backward_bf16(with_rounded((1, 2)), c23, Y23, T)
    for li in range(4):
        for pi in range(2):
            assert np.array_equal(g23[li][pi], g[li][pi]), (li, pi)
    # pre-rounding W1 or W4 does change the output: they are used as they are
    for li in (0, 3):
        assert not np.array_equal(mlp.forward_bf16(with_rounded((li,)), X)[0], Y), li
    # one sample: the hidden layers' bias gradients are the rounded
    # pre-activation gradients themselves
    Y1, c1 = mlp.forward_bf16(params, X[:1])
    g1 = mlp.backward_bf16(params, c1, Y1, T[:1])
    for li in (0, 1, 2):
        db = g1[li][1]
        assert np.array_equal(mlp.bf16(db), db), li
    assert not np.array_equal(mlp.bf16(g1[3][1]), g1[3][1])              # the output layer's is not rounded
