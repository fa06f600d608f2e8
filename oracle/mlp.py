"""CPU oracle of the RACE-parameter predictor — TEST INFRASTRUCTURE ONLY.

A 16 -> 64 -> 64 -> 3 perceptron (ReLU hidden layers, linear output) with the
loss L = 1/(2B) sum_b sum_k w_k (y_bk - t_bk)^2 and the Adam update
(Kingma & Ba, "Adam: A Method for Stochastic Optimization", 2015, Alg. 1),
written out in FP64 numpy.  Parameters use the library's packed layout:
W1[64][16] b1[64] W2[64][64] b2[64] W3[3][64] b3[3].
Pinned in tests/test_oracle_mlp.py by finite differences, a closed-form
network and the closed form of Adam's first step.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 16, 64, 3
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p, x):
    """Returns y (B x 3) and the cache (z1, h1, z2, h2)."""
    P = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"].T + P["b3"]
    return y, (z1, h1, z2, h2)


def loss(p, x, t, w):
    y, _ = forward(p, x)
    return 0.5 * np.sum(np.asarray(w) * (y - t) ** 2) / x.shape[0]


def backward(p, x, t, w):
    """Gradient of loss() with respect to the packed parameters (chain rule)."""
    P = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    y, (z1, h1, z2, h2) = forward(p, x)
    dy = np.asarray(w) * (y - t) / B
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = dy @ P["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return pack(g)


def adam_step(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step; returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
