"""FP64 reference of the warm-start multilayer perceptron (TEST
INFRASTRUCTURE; the paper has no learned component: the network only
proposes the initial guess of the theta-step solve, which PCG then drives to
the same tolerance).

Network: x (n_in) -> silu(W1 x + b1) -> silu(W2 h + b2) -> silu(W3 h + b3)
-> W4 h + b4 (n_out), with silu(z) = z / (1 + exp(-z)).  Weights W_l are
(n_out_l, n_in_l).  Loss over a batch (rows of X, Y):
    L = 1/(2 B) sum_b ||f(x_b) - y_b||^2.
Backward pass by the chain rule, layer by layer.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X):
    """params: list of (W, b); X: (B, n_in).  Returns output and the cache."""
    h = X
    cache = []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = silu(z) if li < len(params) - 1 else z
    return h, cache


def loss_and_grads(params, X, Y, with_deltas=False):
    """Loss and per-layer (dW, db); with_deltas also returns, per layer, the
    gradient with respect to its pre-activation and its input (g_l, h_in_l),
    the factors of dW_l = g_l^T h_in_l."""
    out, cache = forward(params, X)
    B = X.shape[0]
    diff = out - Y
    loss = 0.5 * np.sum(diff * diff) / B
    g = diff / B                                   # dL/d(out)
    grads = [None] * len(params)
    deltas = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        h_in, z = cache[li]
        if li < len(params) - 1:
            g = g * dsilu(z)                       # through the activation
        W, _ = params[li]
        grads[li] = (g.T @ h_in, g.sum(axis=0))    # dW, db
        deltas[li] = (g, h_in)
        g = g @ W                                  # to the previous layer
    if with_deltas:
        return loss, grads, deltas
    return loss, grads
