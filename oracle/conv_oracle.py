"""FP64 CPU oracle of the surrogate network's operations (3x3 periodic convolution, its two
gradients, MSE, Adam).

TEST INFRASTRUCTURE, NOT PRODUCT CODE (same import rule as ``oracle.vlb_oracle``).

Layouts follow the CUDA kernels: activations [H][W][C], weights [C_out][3][3][C_in]; tap
t = 3 (dy + 1) + (dx + 1) reads the input at (y + dy, x + dx), periodic in both directions.
The network is not part of the paper; these are the textbook definitions, written out.
"""
from __future__ import annotations

import numpy as np


def _shift(x, dy, dx):
    """s[y, x] = x[(y + dy) % H, (x + dx) % W]."""
    return np.roll(np.roll(x, -dy, axis=0), -dx, axis=1)


def conv3x3(x, w, b=None, relu=False, mask=None):
    """y[p, co] = act(sum_{t, ci} x[p + d_t, ci] w[co, t, ci] + b[co])."""
    H, W, _ = x.shape
    cout = w.shape[0]
    y = np.zeros((H, W, cout))
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        y += _shift(x, dy, dx) @ w[:, t // 3, t % 3, :].T
    if b is not None:
        y += b
    if relu:
        y = np.maximum(y, 0.0)
    if mask is not None:
        y = np.where(mask > 0, y, 0.0)
    return y


def conv3x3_grad_input(dy, w):
    """dx[p, ci] = sum_{t, co} dy[p - d_t, co] w[co, t, ci]."""
    H, W, _ = dy.shape
    cin = w.shape[3]
    dx = np.zeros((H, W, cin))
    for t in range(9):
        sy, sx = t // 3 - 1, t % 3 - 1
        dx += _shift(dy, -sy, -sx) @ w[:, t // 3, t % 3, :]
    return dx


def conv3x3_grad_weight(x, dy):
    """dw[co, t, ci] = sum_p dy[p, co] x[p + d_t, ci];  db[co] = sum_p dy[p, co]."""
    H, W, cin = x.shape
    cout = dy.shape[2]
    dw = np.zeros((cout, 3, 3, cin))
    D = dy.reshape(-1, cout)
    for t in range(9):
        sy, sx = t // 3 - 1, t % 3 - 1
        dw[:, t // 3, t % 3, :] = D.T @ _shift(x, sy, sx).reshape(-1, cin)
    return dw, D.sum(axis=0)


def mse(pred, target):
    """mean (pred - target)^2 and its gradient."""
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015); returns the new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    return p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps), m, v


def bf16_round(x):
    """Round FP32/FP64 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    u = ((u + r) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
