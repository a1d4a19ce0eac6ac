"""FP64 reference of the learned-correction network — TEST INFRASTRUCTURE ONLY.

The network maps n_in features to one output through two hidden ReLU layers; the loss is
the mean squared error against targets. Parameters use the flat layout W1[H][D], b1[H],
W2[H][H], b2[H], W3[H], b3 (the same layout the CUDA library documents). The gradient is
derived by hand here and pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def unpack(theta: np.ndarray, n_in: int, hidden: int):
    D, H = n_in, hidden
    o = 0
    W1 = theta[o:o + H * D].reshape(H, D); o += H * D
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, W3, b3


def param_count(n_in: int, hidden: int) -> int:
    return hidden * n_in + hidden + hidden * hidden + hidden + hidden + 1


def forward(theta, x, n_in, hidden):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64), n_in, hidden)
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    return h2 @ W3 + b3


def loss(theta, x, t, n_in, hidden) -> float:
    y = forward(theta, x, n_in, hidden)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def gradient(theta, x, t, n_in, hidden):
    """Loss and its gradient with respect to the flat parameter vector."""
    theta = np.asarray(theta, np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    n = x.shape[0]
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    dy = 2.0 * (y - t) / n
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return float(np.mean((y - t) ** 2)), g


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)
