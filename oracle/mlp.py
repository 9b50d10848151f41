"""FP64 reference of the surrogate's MLP -- TEST INFRASTRUCTURE.

The surrogate maps a ray's entry state to the residual of its exit line
(learned part of the image generator; the paper itself has none).  The
network: 16 inputs (5 features, zero padded) -> 128 -> 128 -> 128 -> 128 -> 4,
ReLU after each hidden layer, mean-squared-error loss over the batch and the
4 outputs, Adam (Kingma & Ba 2015) on all weights and biases.

Parameters are one flat float vector, layer by layer, each layer W [out][in]
(row-major) followed by b [out] -- the same layout the CUDA library uses.
Only tests and the bench's baseline use this module.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(16, 128), (128, 128), (128, 128), (128, 128), (128, 4)]   # (in, out)


def n_params() -> int:
    return sum(i * o + o for i, o in LAYERS)


def unpack(p):
    out, off = [], 0
    for i, o in LAYERS:
        W = p[off:off + i * o].reshape(o, i)
        off += i * o
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def init(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6/in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in LAYERS:
        bound = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-bound, bound, size=(o, i)).ravel())
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32)
    r = ((b >> 16) & 1) + np.uint32(0x7FFF)
    return ((b + r) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)


def forward(p, X, bf16=False):
    """X [n][16] -> (Y [n][4], list of layer inputs H_0..H_4).  With bf16,
    every hidden activation is stored rounded to BF16 (as a BF16 network
    keeps it between layers)."""
    H = np.asarray(X, dtype=np.float64)
    hs = []
    layers = unpack(np.asarray(p, dtype=np.float64))
    for li, (W, b) in enumerate(layers):
        hs.append(H)
        Z = H @ W.T + b
        if li < len(layers) - 1:
            H = np.maximum(Z, 0.0)
            if bf16:
                H = bf16_round(H)
        else:
            H = Z
    return H, hs


def loss_and_grad(p, X, T, bf16=False):
    """MSE loss mean((Y - T)^2) over n x 4 and its gradient (flat).  With
    bf16, activations and every back-propagated dZ are rounded to BF16 before
    they enter a product, and ReLU masks come from the rounded activations."""
    Y, hs = forward(p, X, bf16)
    n = X.shape[0]
    loss = np.mean((Y - T) ** 2)
    dZ = 2.0 * (Y - T) / (n * Y.shape[1])
    if bf16:
        dZ = bf16_round(dZ)
    layers = unpack(np.asarray(p, dtype=np.float64))
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        H = hs[li]
        grads[li] = (dZ.T @ H, dZ.sum(axis=0))
        if li > 0:
            dH = dZ @ W
            dZ = dH * (H > 0.0)
            if bf16:
                dZ = bf16_round(dZ)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return loss, flat


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
