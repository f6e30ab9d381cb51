"""Plain FP64 numpy reference of the surrogate network.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU legs use it; the CUDA path never imports it. The paper defines no learned
component, so this module follows the textbook definitions of a circular 3x3
convolution, its two adjoints and the tanh form of GELU; it is pinned in
tests/test_cnn_oracle.py against scipy's wrap-mode correlation, the adjoint
identity and finite differences.

Network: x0 = [Q (6 channels), n_x, n_y, n_z] on a periodic H x W lattice;
  a1 = GELU(conv1(x0));  a_k = a_{k-1} + GELU(conv_k(a_{k-1})), k = 2..5;
  dQ = scale * conv6(a5);  Q_next = Q + dQ,
with 3x3 convolutions with circular padding (the lattice is periodic) and the
tanh form of GELU. Activations are (H, W, C); weights (Cout, Cin, 3, 3).
"""
from __future__ import annotations

import math

import numpy as np

K_GELU = math.sqrt(2.0 / math.pi)


def conv3x3(x: np.ndarray, w: np.ndarray, b=None) -> np.ndarray:
    """y[i, j, n] = b[n] + sum_{ky, kx, c} w[n, c, ky, kx] x[i+ky-1, j+kx-1, c] (indices mod H, W)."""
    H, W, _ = x.shape
    y = np.zeros((H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            xs = np.roll(x, shift=(1 - ky, 1 - kx), axis=(0, 1))
            y += xs @ w[:, :, ky, kx].T
    if b is not None:
        y += b
    return y


def conv3x3_input_grad(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 with respect to x: dx[p, c] = sum g[p - off, n] w[n, c, off]."""
    H, W, _ = g.shape
    dx = np.zeros((H, W, w.shape[1]))
    for ky in range(3):
        for kx in range(3):
            dx += np.roll(g @ w[:, :, ky, kx], shift=(ky - 1, kx - 1), axis=(0, 1))
    return dx


def conv3x3_weight_grad(g: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dw[n, c, ky, kx] = sum_p g[p, n] x[p + (ky-1, kx-1), c]."""
    Cout, Cin = g.shape[2], x.shape[2]
    dw = np.zeros((Cout, Cin, 3, 3))
    for ky in range(3):
        for kx in range(3):
            xs = np.roll(x, shift=(1 - ky, 1 - kx), axis=(0, 1))
            dw[:, :, ky, kx] = np.einsum("hwn,hwc->nc", g, xs)
    return dw


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(K_GELU * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(K_GELU * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * K_GELU * (1.0 + 3.0 * 0.044715 * x * x)


def forward(x0, weights, biases, scale):
    """Returns (dQ, cache). weights/biases: lists of 6 arrays."""
    zs, acts = [], [x0]
    z = conv3x3(x0, weights[0], biases[0])
    zs.append(z)
    a = gelu(z)
    acts.append(a)
    for k in range(1, 5):
        z = conv3x3(a, weights[k], biases[k])
        zs.append(z)
        a = a + gelu(z)
        acts.append(a)
    out = conv3x3(a, weights[5], biases[5])
    return scale * out, (zs, acts)


def backward(dout, weights, cache, scale):
    """Gradients of sum(dout * dQ) with respect to weights and biases."""
    zs, acts = cache
    g = dout * scale
    dW = [None] * 6
    dB = [None] * 6
    dW[5] = conv3x3_weight_grad(g, acts[5])
    dB[5] = g.sum(axis=(0, 1))
    da = conv3x3_input_grad(g, weights[5])
    for k in range(4, 0, -1):
        dz = da * gelu_grad(zs[k])
        dW[k] = conv3x3_weight_grad(dz, acts[k])
        dB[k] = dz.sum(axis=(0, 1))
        da = da + conv3x3_input_grad(dz, weights[k])
    dz = da * gelu_grad(zs[0])
    dW[0] = conv3x3_weight_grad(dz, acts[0])
    dB[0] = dz.sum(axis=(0, 1))
    return dW, dB
