"""FP64 reference of the initial-guess network -- TEST INFRASTRUCTURE ONLY.

A 6-64-64-1 perceptron with tanh hidden layers and a linear output,
y = W3 tanh(W2 tanh(W1 xn + b1) + b2) + b3, on normalised inputs
xn = (x - mean) / scale, trained with the mean squared error
L = mean_b (y_b - t_b)^2.  The forward pass and the hand-derived backward
pass below are what the CUDA training kernels must reproduce; they are pinned
by central finite differences in tests/test_oracle_mlp.py.

Parameter vector layout (float64 here, float32 on the GPU), the same as the
library's weight blob without the normalisation tail:
    W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3[1]   (4673 values)
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 6, 64
SIZES = [(N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_H,), (1,)]
N_PARAMS = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    out, k = [], 0
    for s in SIZES:
        c = int(np.prod(s))
        out.append(np.asarray(theta[k:k + c], dtype=np.float64).reshape(s))
        k += c
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 1 / np.sqrt(N_IN), (N_H, N_IN))
    W2 = rng.normal(0, 1 / np.sqrt(N_H), (N_H, N_H))
    W3 = rng.normal(0, 1 / np.sqrt(N_H), (N_H,))
    return pack([W1, np.zeros(N_H), W2, np.zeros(N_H), W3, np.zeros(1)])


def forward(theta, xn):
    """xn: [B, 6] normalised inputs. Returns (y [B], cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z1 = xn @ W1.T + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2.T + b2
    h2 = np.tanh(z2)
    y = h2 @ W3 + b3[0]
    return y, (xn, h1, h2)


def loss_and_grad(theta, xn, target):
    """Mean squared error and its gradient with respect to theta."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    y, (x, h1, h2) = forward(theta, xn)
    B = x.shape[0]
    r = y - target
    L = float(np.mean(r * r))
    dy = 2.0 * r / B                       # dL/dy
    gW3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    dz2 = (dy[:, None] * W3[None, :]) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3])
