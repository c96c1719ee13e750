"""FP64 oracle of the learned cost model (16 -> 64 -> 64 -> 1 MLP, ReLU).

TEST INFRASTRUCTURE ONLY (tests and the smoke check).  Plain NumPy, written
independently of the CUDA kernels: the forward pass, the mean-squared-error
loss, its gradient by backpropagation, and one Adam step.  Parameters are
flat in the library's order: W1 [64 x 16], b1 [64], W2 [64 x 64], b2 [64],
W3 [1 x 64], b3 [1].  bf16() rounds to bfloat16 (round to nearest, ties to
even) so that the oracle sees the same weights as the BF16 kernels.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 16, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (1, N_H)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X):
    P = unpack(theta)
    h1 = np.maximum(X @ P["W1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
    y = (h2 @ P["W3"].T + P["b3"])[:, 0]
    return y, (h1, h2)


def loss_grad(theta, X, t):
    """Mean squared error and its gradient with respect to theta."""
    P = unpack(theta)
    n = X.shape[0]
    y, (h1, h2) = forward(theta, X)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n                                # dL/dy
    g = {"W3": dy[None, :] @ h2, "b3": np.array([dy.sum()])}
    dh2 = (dy[:, None] @ P["W3"]) * (h2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ P["W2"]) * (h1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns theta, m, v."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
