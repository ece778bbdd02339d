"""FP64 forward/backward of the chemical-potential seed network (not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network: x (32) -> h1 = tanh(W1 x + b1) (64) -> h2 = tanh(W2 h1 + b2) (64) -> y = W3 h2 + b3.
Loss: L = (1/n) sum_s (y_s - t_s)^2.  Parameters packed as [W1 (64x32 row-major), b1, W2 (64x64
row-major), b2, W3 (64), b3].  The backward pass is the chain rule written out; it is pinned by
central finite differences of L in FP64.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 32, 64
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, off = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(theta, X):
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, h1, h2)


def loss(theta, X, T):
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def grad(theta, X, T):
    """Analytic gradient of the mean squared error."""
    p = unpack(theta)
    y, (X, h1, h2) = forward(theta, X)
    n = X.shape[0]
    dy = 2.0 * (y - np.asarray(T, dtype=np.float64)) / n          # (n,)
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["W3"]) * (1.0 - h2 ** 2)                  # (n, 64)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def finite_difference_grad(theta, X, T, idx, h=1e-6):
    """Central differences of the loss for the parameters listed in idx."""
    theta = np.asarray(theta, dtype=np.float64)
    out = []
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        out.append((loss(tp, X, T) - loss(tm, X, T)) / (2 * h))
    return np.array(out)
