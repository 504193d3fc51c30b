"""FP64 reference of the warm-start network (test infrastructure).

Not part of the paper: the network is the learned warm start of the value
function and the thrust angle.  Architecture 4 -> 256 -> 256 -> 256 -> 3,
GELU (exact erf form) after the three hidden layers, linear output
(V / M, cos alpha, sin alpha).  Loss: mean squared error over the batch and
the three outputs.  Plain numpy in float64, one layer at a time; the
backward pass is pinned by central finite differences in the tests.

Only the test suite uses this module.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SIZES = (4, 256, 256, 256, 3)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(params, X):
    """Returns the output and the per-layer pre-activations / inputs."""
    a = np.asarray(X, np.float64)
    cache = []
    for li, (W, b) in enumerate(params):
        z = a @ W.T + b
        cache.append((a, z))
        a = gelu(z) if li < len(params) - 1 else z
    return a, cache


def loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def backward(params, cache, Y, T):
    """Gradients of the mean squared error with respect to every W and b."""
    n = Y.size
    d = 2.0 * (Y - T) / n                       # dL/dy
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        a_in, z = cache[li]
        if li < len(params) - 1:
            d = d * gelu_grad(z)                # through the activation
        W, b = params[li]
        grads[li] = [d.T @ a_in, d.sum(axis=0)]
        d = d @ W
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (in place); state = dict(t, m, v)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    if "m" not in state:
        state["m"] = [[np.zeros_like(p) for p in layer] for layer in params]
        state["v"] = [[np.zeros_like(p) for p in layer] for layer in params]
    for li, layer in enumerate(params):
        for pi in range(2):
            g = grads[li][pi]
            m = state["m"][li][pi] = b1 * state["m"][li][pi] + (1 - b1) * g
            v = state["v"][li][pi] = b2 * state["v"][li][pi] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            layer[pi] -= lr * mh / (np.sqrt(vh) + eps)


def normalise_states(X, lo, hi):
    """Map box coordinates to [-1, 1]^4."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return 2.0 * (np.asarray(X, np.float64) - lo) / (hi - lo) - 1.0
