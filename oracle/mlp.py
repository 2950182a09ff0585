"""FP64 oracle of the tuner network -- TEST INFRASTRUCTURE ONLY.

The tuner is not in the paper: it is the learned-knob subsystem built around the
method (it predicts the partition size of Eq. 1/2, the ELL width cap and the
threads per row).  The network is a 3-layer perceptron 16 -> 64 -> 64 -> 4 with
ReLU after the two hidden layers and a linear output, trained on the mean squared
error with Adam (Kingma & Ba, 2015).  Parameters are stored as
W1 (64x16), b1 (64), W2 (64x64), b2 (64), W3 (4x64), b3 (4): 5,508 numbers.

Everything here is plain numpy in float64, written from those definitions.
"""
from __future__ import annotations

import numpy as np

SIZES = (16, 64, 64, 4)
SHAPES = (("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (4, 64)), ("b3", (4,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Split the flat parameter vector (in SHAPES order, row-major) into named arrays."""
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def forward(theta: np.ndarray, X: np.ndarray):
    """X: (B, 16).  Returns (out (B, 4), cache)."""
    p = unpack(np.asarray(theta, np.float64))
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (X, z1, h1, z2, h2)


def loss(theta, X, T) -> float:
    """L = mean over the batch and the 4 outputs of (out - T)^2."""
    out, _ = forward(theta, X)
    return float(np.mean((out - np.asarray(T, np.float64)) ** 2))


def grad(theta, X, T):
    """(L, dL/dtheta) by back-propagation through the three layers."""
    p = unpack(np.asarray(theta, np.float64))
    out, (X, z1, h1, z2, h2) = forward(theta, X)
    T = np.asarray(T, np.float64)
    B = X.shape[0]
    L = float(np.mean((out - T) ** 2))
    d_out = 2.0 * (out - T) / (B * out.shape[1])          # dL/dout
    gW3 = d_out.T @ h2
    gb3 = d_out.sum(0)
    d_h2 = d_out @ p["W3"]
    d_z2 = d_h2 * (z2 > 0)
    gW2 = d_z2.T @ h1
    gb2 = d_z2.sum(0)
    d_h1 = d_z2 @ p["W2"]
    d_z1 = d_h1 * (z1 > 0)
    gW1 = d_z1.T @ X
    gb1 = d_z1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(theta, m, v, g, t: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step number t >= 1).  Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def init(seed: int) -> np.ndarray:
    """He-uniform initial weights (bound sqrt(6/fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            bound = np.sqrt(6.0 / shp[1])
            parts.append(rng.uniform(-bound, bound, shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts)
