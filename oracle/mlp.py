"""The schedule MLP, oracle side: plain numpy, fp64.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Network: 6 inputs -> 64 tanh -> 64 tanh -> 1 linear, parameters packed in one
flat vector [W1 (64x6, row-major), b1 (64), W2 (64x64), b2 (64), W3 (64),
b3 (1)] = 4673 values. The GPU keeps fp32 master parameters and computes with
their bf16 roundings and fp32 accumulation; `bf16_round` emulates that
rounding so the oracle can evaluate the same network in fp64.
Loss over a batch: (1/B) sum_b (y_b - t_b)^2 / 2.
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr (m / (1-b1^k)) / (sqrt(v / (1-b2^k)) + eps).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 6, 64
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)  # 4673


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16_round(x):
    """Round fp32 values to bf16 (nearest, ties to even), returned as fp64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X):
    """Outputs y [B] and the hidden activations (for backward)."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ w["W1"].T + w["b1"])
    h2 = np.tanh(h1 @ w["W2"].T + w["b2"])
    y = h2 @ w["W3"] + w["b3"][0]
    return y, (X, h1, h2)


def loss(p, X, T):
    y, _ = forward(p, X)
    return float(0.5 * np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def grad(p, X, T):
    """Gradient of loss(p, X, T) with respect to p (flat), by the chain rule."""
    w = unpack(p)
    y, (X, h1, h2) = forward(p, X)
    B = X.shape[0]
    dy = (y - np.asarray(T, dtype=np.float64)) / B           # dL/dy
    g = {}
    g["W3"] = dy @ h2
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, w["W3"]) * (1.0 - h2 * h2)             # through tanh
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ w["W2"]) * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return pack(g)


def adam(p, g, m, v, k, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
