"""FP64 CPU reference of the warm-start network (test infrastructure).

A plain numpy forward and backward pass of the three-layer perceptron
  Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2, H2 = relu(Z2),
  Y = H2 W3^T + b3,
with the loss used to train it, averaged over the batch:
  l = (Y_0 - T_0)^2 + (1 - (a.b)^2 / (|a|^2 |b|^2)),  a = Y_1.., b = T_1..
(log step length in T_0; the target null vector in T_1.., defined up to sign,
hence the squared cosine).  Used to check the GPU kernels' gradients; its own
gradients are pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grad_out(Y, T):
    """Batch-mean loss and dL/dY."""
    B = Y.shape[0]
    d0 = Y[:, 0] - T[:, 0]
    a, b = Y[:, 1:], T[:, 1:]
    ab = np.sum(a * b, axis=1)
    aa = np.sum(a * a, axis=1)
    bb = np.sum(b * b, axis=1)
    cos2 = ab * ab / (aa * bb)
    loss = np.mean(d0 * d0 + (1.0 - cos2))
    dY = np.zeros_like(Y)
    dY[:, 0] = 2.0 * d0 / B
    # d(1 - cos2)/da = -(2 ab b / (aa bb) - 2 ab^2 a / (aa^2 bb))
    dY[:, 1:] = -(2.0 * ab[:, None] * b / (aa * bb)[:, None]
                  - 2.0 * (ab * ab)[:, None] * a / (aa * aa * bb)[:, None]) / B
    return loss, dY


def backward(params, cache, dY):
    W1, b1, W2, b2, W3, b3 = params
    X, Z1, H1, Z2, H2 = cache
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dH2 = dY @ W3
    dZ2 = dH2 * (Z2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def loss_grad(params, X, T):
    Y, cache = forward(params, X)
    loss, dY = loss_and_grad_out(Y, T)
    return loss, backward(params, cache, dY)
