"""FP64 reference of the warm-start network (test infrastructure).

Not part of the paper: the network is the learned warm start of the value
function and the thrust angle.  Architecture 4 -> 256 -> 256 -> 256 -> 3,
GELU (exact erf form) after the three hidden layers, linear output
(V / M, cos alpha, sin alpha).  Loss: mean squared error over the batch and
the three outputs.  Plain numpy in float64, one layer at a time; the
backward pass is pinned by central finite differences in the tests.

forward_bf16 / backward_bf16 are the same network with BF16 rounding (round
to nearest even) applied where a tensor-core implementation with BF16
operands and FP32 accumulation rounds: the hidden activations, the weights
of the two 256 x 256 layers and the back-propagated pre-activation
gradients.  Everything else stays FP64, so the GPU path differs from them only
by FP32 accumulation and by isolated one-unit rounding flips, which lets a
test check its outputs element by element.

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


def bf16(a):
    """Round to BF16 (8 significant bits, round to nearest even) through FP32,
    returned as float64.  Finite inputs of FP32 range only."""
    x = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, X):
    """Forward pass with BF16 hidden activations and BF16 weights of layers 2
    and 3 (inputs, layer 1 and the output layer in full precision).  Returns
    the output and the per-layer (input, pre-activation) pairs."""
    a = np.asarray(X, np.float32).astype(np.float64)
    cache = []
    last = len(params) - 1
    for li, (W, b) in enumerate(params):
        W = np.asarray(W, np.float32).astype(np.float64)
        b = np.asarray(b, np.float32).astype(np.float64)
        if 0 < li < last:
            W = bf16(W)
        z = a @ W.T + b
        cache.append((a, z))
        a = bf16(gelu(z)) if li < last else z
    return a, cache


def backward_bf16(params, cache, Y, T):
    """Gradients of the mean squared error for forward_bf16: the gradients of
    the pre-activations of the hidden layers are rounded to BF16 before they
    are propagated and reduced, and layers 2 and 3 back-propagate through
    their BF16 weights."""
    n = Y.size
    d = 2.0 * (Y - T) / n
    grads = [None] * len(params)
    last = len(params) - 1
    for li in range(last, -1, -1):
        a_in, z = cache[li]
        if li < last:
            d = bf16(d * gelu_grad(z))
        W = np.asarray(params[li][0], np.float32).astype(np.float64)
        if 0 < li < last:
            W = bf16(W)
        grads[li] = [d.T @ a_in, d.sum(axis=0)]
        d = d @ W
    return grads


def normalise_states(X, lo, hi):
    """Map box coordinates to [-1, 1]^4."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return 2.0 * (np.asarray(X, np.float64) - lo) / (hi - lo) - 1.0
