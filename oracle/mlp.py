"""The schedule MLP (16 -> 64 -> 64 -> 2, ReLU) in float64 — test infrastructure only.

Parameters are one flat vector in this order: W1 [16][64], b1 [64], W2 [64][64],
b2 [64], W3 [64][2], b3 [2] (row-major, y = x @ W + b). The loss is the weighted
mean squared error (1/N) sum_i sum_k w_k (y_ik - t_ik)^2; Adam is the published
update of Kingma & Ba (2015) with bias correction:
    m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
Parity status: backpropagation pinned by central finite differences and
hand-worked forward passes (tests/test_oracle_learned.py).
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (16, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 2)), ("b3", (2,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray):
    out, off = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = p[off:off + k].reshape(shp)
        off += k
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p: np.ndarray, X: np.ndarray, return_hidden: bool = False):
    w = unpack(np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ w["W1"] + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w["W3"] + w["b3"]
    return (y, h1, h2) if return_hidden else y


def loss(p, X, T, wk=(1.0, 1.0)) -> float:
    y = forward(p, X)
    return float(np.mean(np.sum(np.asarray(wk) * (y - T) ** 2, axis=1)))


def grad(p, X, T, wk=(1.0, 1.0)) -> np.ndarray:
    """Gradient of `loss` by backpropagation."""
    w = unpack(np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    y, h1, h2 = forward(p, X, return_hidden=True)
    N = X.shape[0]
    dy = 2.0 * np.asarray(wk) * (y - T) / N
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dh2 = (dy @ w["W3"].T) * (h2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ w["W2"].T) * (h1 > 0)
    g["W1"] = X.T @ dh1
    g["b1"] = dh1.sum(0)
    return pack(g)


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform initial weights, zero biases (a fixed seeded draw)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shp[0])
            d[name] = rng.uniform(-lim, lim, size=shp)
        else:
            d[name] = np.zeros(shp)
    return pack(d)
