"""FP64 CPU oracle of the learned-proposal network (test infrastructure only).

y = W2 relu(W1 x + b1) + b2 per sample; loss = (1 / (B d_out)) sum (y - t)^2.
The GPU runs its forward and backward passes with FP16 working copies of W1
and W2; `fp16_weights=True` rounds them the same way so both sides evaluate
the same function.  Gradients are the textbook backpropagation of that
function, pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def _w(W, fp16):
    return W.astype(np.float16).astype(np.float64) if fp16 else W.astype(np.float64)


def forward(X, W1, b1, W2, b2, fp16_weights=False):
    W1e, W2e = _w(W1, fp16_weights), _w(W2, fp16_weights)
    Z1 = X.astype(np.float64) @ W1e.T + b1
    A1 = np.maximum(Z1, 0.0)
    Y = A1 @ W2e.T + b2
    return Y, (Z1, A1, W1e, W2e)


def loss_and_grads(X, T, W1, b1, W2, b2, fp16_weights=False):
    Y, (Z1, A1, W1e, W2e) = forward(X, W1, b1, W2, b2, fp16_weights)
    B, D = Y.shape
    R = Y - T.astype(np.float64)
    loss = float(np.sum(R * R) / (B * D))
    dY = 2.0 * R / (B * D)
    gW2 = dY.T @ A1
    gb2 = dY.sum(axis=0)
    dZ1 = (dY @ W2e) * (Z1 > 0)
    gW1 = dZ1.T @ X.astype(np.float64)
    gb1 = dZ1.sum(axis=0)
    return loss, gW1, gb1, gW2, gb2
