"""FP64 reference of the learned surrogate's MLP (forward, backward, Adam).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain NumPy in double
precision, with an option to round stored activations to bfloat16 at the
same points the GPU path stores them, so the GPU can be compared on identical
inputs.

Network: x [B][n_in] -> (Linear -> GELU) x depth -> Linear -> y [B][n_out];
GELU(x) = x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2)) (Hendrycks & Gimpel 2016);
loss = mean over batch and outputs of (y - t)^2; Adam (Kingma & Ba 2015).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (via float32, round to nearest even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(params, x, bf16_acts=False):
    """params: list of (W [in][out], b [out]).  Returns (y, cache)."""
    a = np.asarray(x, np.float64)
    cache = []
    for li, (W, b) in enumerate(params):
        z = a @ W + b
        cache.append((a, z))
        if li < len(params) - 1:
            a = gelu(z)
            if bf16_acts:
                a = bf16(a)
        else:
            a = z
    return a, cache


def loss_and_grad_out(y, t):
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, cache, dy, bf16_acts=False):
    """Gradients [(dW, db)] of the loss whose output gradient is dy.  With
    bf16_acts the stored gradients are rounded where the GPU stores them: the
    output gradient, and each layer's (G W^T) * GELU'(z) after the product."""
    grads = [None] * len(params)
    g = bf16(dy) if bf16_acts else dy
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        a, z = cache[li]
        grads[li] = (a.T @ g, g.sum(0))
        if li > 0:
            _, zp = cache[li - 1]
            g = (g @ W.T) * gelu_grad(zp)
            if bf16_acts:
                g = bf16(g)
    return grads


def adam(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state = dict(t, m, v)."""
    state["t"] += 1
    t = state["t"]
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        for j, (p, gp) in enumerate(((W, gW), (b, gb))):
            m = state["m"][i][j] = b1 * state["m"][i][j] + (1 - b1) * gp
            v = state["v"][i][j] = b2 * state["v"][i][j] + (1 - b2) * gp * gp
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            p -= lr * mh / (np.sqrt(vh) + eps)


def adam_state(params):
    return {"t": 0, "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}


def init_params(n_in, width, depth, n_out, seed=0):
    """He-normal weights, zero biases (the initial values are an input, not the method)."""
    rng = np.random.default_rng(seed)
    sizes = [n_in] + [width] * depth + [n_out]
    return [(rng.standard_normal((sizes[i], sizes[i + 1])) * np.sqrt(2.0 / sizes[i]), np.zeros(sizes[i + 1]))
            for i in range(len(sizes) - 1)]
