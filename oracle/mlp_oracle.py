"""FP64 CPU oracle for the alpha/m predictor MLP (6 -> 64 -> 64 -> 2, ReLU).

TEST INFRASTRUCTURE ONLY: plain numpy definitions that the library's CUDA training and
inference kernels are checked against. Not imported by the library.

Parameters are one flat vector of 4738 values laid out as W1[64][6], b1[64], W2[64][64],
b2[64], W3[2][64], b3[2] (row-major). Loss: mean over samples of 1/2 ||y - t||^2.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 6, 64, 2
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed):
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            d[name] = rng.uniform(-lim, lim, size=shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)


def forward(theta, X):
    """Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X."""
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = np.maximum(z2, 0.0)
    y = a2 @ p["W3"].T + p["b3"]
    return y, (X, z1, a1, z2, a2)


def loss(theta, X, T):
    y, _ = forward(theta, X)
    return 0.5 * np.sum((y - T) ** 2) / X.shape[0]


def grad(theta, X, T):
    """Gradient of loss by backpropagation (chain rule through the three layers)."""
    p = unpack(theta)
    y, (X, z1, a1, z2, a2) = forward(theta, X)
    B = X.shape[0]
    dy = (y - T) / B
    g = {"W3": dy.T @ a2, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return pack(g), 0.5 * np.sum((y - T) ** 2) / B


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, bias-corrected moments); t is the 1-based step count."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def to_bf16(a):
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X):
    """Forward with bfloat16 weights, inputs and activations (exact accumulation)."""
    p = {k: to_bf16(v) for k, v in unpack(np.asarray(theta, np.float32)).items()}
    x = to_bf16(np.asarray(X, np.float32))
    a1 = to_bf16(np.maximum(x @ p["W1"].T + p["b1"], 0.0))
    a2 = to_bf16(np.maximum(a1 @ p["W2"].T + p["b2"], 0.0))
    return a2 @ p["W3"].T + p["b3"]
