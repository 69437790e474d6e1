"""TEST INFRASTRUCTURE ONLY: the plain FP64 multilayer perceptron the value-network kernels are
checked against.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
module; the product path never does, and this module never imports the product path.

The network (a leaf-value model for depth-limited solving; the paper has no learned part) is
y = W_L(...ReLU(W_1 x + b_1)...) + b_L with W_l of shape [out, in], trained on the mean squared error
L = (1 / (B n_out)) sum (y - t)^2 by Adam (Kingma and Ba, 2015, Algorithm 1, with bias correction).
Everything is FP64 numpy, layer by layer, with no fusion.  ``bf16=True`` reproduces the points where the
GPU path rounds to BF16 (round to nearest even): the weights and the input, each hidden layer's output
after ReLU, the output gradient dL/dy, and each hidden layer's masked gradient; the products themselves
stay exact (FP64), the GPU accumulating in FP32.

Parameters are a list of (W, b) pairs; ``flatten`` / ``unflatten`` use the library's host layout (layer
by layer, W row-major, then b).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """x rounded to the nearest BF16 value (ties to even), as FP64.  BF16 keeps FP32's sign and
    exponent and the top 7 of its 23 fraction bits; the value is first rounded to FP32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def init_params(dims, rng: np.random.Generator, scale: float = 1.0):
    """He-style initialisation: W ~ N(0, scale^2 2 / in), b ~ N(0, 0.01^2)."""
    return [(rng.normal(0.0, scale * np.sqrt(2.0 / dims[l]), size=(dims[l + 1], dims[l])),
             rng.normal(0.0, 0.01, size=dims[l + 1])) for l in range(len(dims) - 1)]


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat, dims):
    out, k = [], 0
    for l in range(len(dims) - 1):
        n_w = dims[l + 1] * dims[l]
        W = np.asarray(flat[k:k + n_w], dtype=np.float64).reshape(dims[l + 1], dims[l])
        k += n_w
        b = np.asarray(flat[k:k + dims[l + 1]], dtype=np.float64)
        k += dims[l + 1]
        out.append((W, b))
    return out


def _rounder(bf16: bool):
    return bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))


def dense(a, W, b, bf16: bool = False):
    """One layer's pre-activation Z = a W^T + b, a [B][in] used as given, W [out][in] (rounded to BF16
    in BF16 mode), b [out]."""
    return np.asarray(a, dtype=np.float64) @ _rounder(bf16)(W).T + np.asarray(b, dtype=np.float64)


def hidden(z, bf16: bool = False):
    """A hidden layer's output ReLU(Z), rounded to BF16 in BF16 mode."""
    return _rounder(bf16)(np.maximum(z, 0.0))


def output_gradient(y, t):
    """dL/dy of the mean squared error L = (1 / (B n)) sum (y - t)^2, before any rounding."""
    y = np.asarray(y, dtype=np.float64)
    B, n = y.shape
    return 2.0 * (y - np.asarray(t, dtype=np.float64)) / (B * n)


def layer_gradients(dz, a):
    """dL/dW = dZ^T a and dL/db = the column sums of dZ, for one layer with input a."""
    dz = np.asarray(dz, dtype=np.float64)
    return dz.T @ np.asarray(a, dtype=np.float64), dz.sum(axis=0)


def masked_product(dz, W, a, bf16: bool = False):
    """(dZ W) where the layer below's ReLU output a is positive, else 0 (W rounded to BF16 in BF16
    mode): dL/dZ of the layer below before any rounding of the result."""
    return (np.asarray(dz, dtype=np.float64) @ _rounder(bf16)(W)) * (np.asarray(a) > 0)


def input_gradient(dz, W, a, bf16: bool = False):
    """dL/dZ of the layer below, rounded to BF16 in BF16 mode."""
    return _rounder(bf16)(masked_product(dz, W, a, bf16))


def forward(params, x, bf16: bool = False):
    """Returns (y, activations): activations[0] is the input (as used), activations[l] the output of
    hidden layer l - 1 after ReLU."""
    a = _rounder(bf16)(x)
    acts = [a]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = dense(a, W, b, bf16)
        if l + 1 < L:
            a = hidden(z, bf16)
            acts.append(a)
        else:
            return z, acts
    raise AssertionError("unreachable")


def loss_and_grads(params, x, t, bf16: bool = False):
    """Mean squared error and its gradient with respect to every W and b (backpropagation)."""
    y, acts = forward(params, x, bf16)
    B, n = y.shape
    d = y - np.asarray(t, dtype=np.float64)
    loss = float(np.sum(d * d) / (B * n))
    dz = _rounder(bf16)(output_gradient(y, t))
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = layer_gradients(dz, acts[l])
        if l > 0:
            dz = input_gradient(dz, W, acts[l], bf16)
    return loss, grads


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step; state = {"t": steps so far, "m": [...], "v": [...]} (created when empty).
    Returns the new parameters."""
    if not state:
        state.update(t=0, m=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
                     v=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    state["t"] += 1
    t = state["t"]
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m = beta1 * state["m"][l][j] + (1.0 - beta1) * g
            v = beta2 * state["v"][l][j] + (1.0 - beta2) * g * g
            mh = m / (1.0 - beta1 ** t)
            vh = v / (1.0 - beta2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
            ms, vs = list(state["m"][l]), list(state["v"][l])
            ms[j], vs[j] = m, v
            state["m"][l], state["v"][l] = tuple(ms), tuple(vs)
        out.append((new[0], new[1]))
    return out
