"""The band-predictor network in float64 -- TEST INFRASTRUCTURE (oracle).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use this module.  The product's CUDA kernels compute the same network in
float32 with bf16 weights; the two share no code.

The network is not part of the paper.  It maps the 32 pair features to
y = log2(1 + w), w the predicted band half-width:

    h1 = relu(W1 x + b1)        W1: 64 x 32
    h2 = relu(W2 h1 + b2)       W2: 64 x 64
    y  = w3 . h2 + b3           w3: 64

Flat parameter vector (this order, row-major): W1, b1, W2, b2, w3, b3;
NPARAMS = 6337.  Loss over a batch of B samples with targets t:
    L = (1 / (2B)) * sum_b (y_b - t_b)^2
Gradients are the plain chain rule of that expression (relu'(0) = 0).
Adam (Kingma & Ba, 2015, Algorithm 1) with bias correction; step counts
from 1.  bf16 is round-to-nearest-even of float32 to its top 16 bits.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 32, 64
SIZES = (("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
         ("b3", (1,)))
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    """Views of the named tensors inside a flat parameter vector."""
    out, k = {}, 0
    for name, shape in SIZES:
        size = int(np.prod(shape))
        out[name] = p[k:k + size].reshape(shape)
        k += size
    return out


def forward(p: np.ndarray, X: np.ndarray):
    """y[B] and the activations (float64)."""
    P = unpack(np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_grad(p: np.ndarray, X: np.ndarray, t: np.ndarray):
    """(L, dL/dp) at p for the batch (X, t), float64."""
    P = unpack(np.asarray(p, dtype=np.float64))
    y, (X, z1, h1, z2, h2) = forward(p, X)
    t = np.asarray(t, dtype=np.float64)
    B = len(t)
    r = y - t
    L = 0.5 * float(np.dot(r, r)) / B
    dy = r / B                                   # dL/dy_b
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    d2 = np.outer(dy, P["w3"]) * (z2 > 0)        # dL/dz2
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (z1 > 0)               # dL/dz1
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return L, flat


def adam_step(master, m, v, g, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update; returns new (master, m, v).  step >= 1."""
    master = np.asarray(master, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return master - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16_bits(x) -> np.ndarray:
    """bf16 bit patterns (uint16) of float32 values, round to nearest even (finite inputs)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    return ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)


def bf16_to_f32(bits) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)

