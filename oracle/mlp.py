"""FP64 reference of the predictor network (test infrastructure only).

A plain numpy statement of the network the library trains: y = W3 r(W2 r(W1 x
+ b1) + b2) + b3 with r = ReLU, loss (1/2B) sum (y - t)^2, and its gradient by
the chain rule written out layer by layer.  Parameters use the library's
layout: W1[h1][in], b1, W2[h2][h1], b2, W3[out][h2], b3.
"""
from __future__ import annotations

import numpy as np


def unpack(params, sizes):
    i, h1, h2, o = sizes
    p = np.asarray(params, dtype=np.float64)
    k = 0
    out = []
    for shape in [(h1, i), (h1,), (h2, h1), (h2,), (o, h2), (o,)]:
        n = int(np.prod(shape))
        out.append(p[k:k + n].reshape(shape))
        k += n
    assert k == p.size
    return out


def forward(params, sizes, X):
    W1, b1, W2, b2, W3, b3 = unpack(params, sizes)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3.T + b3
    return y, (X, z1, a1, z2, a2)


def loss(params, sizes, X, T):
    y, _ = forward(params, sizes, X)
    B = y.shape[0]
    return 0.5 * np.sum((y - np.asarray(T, dtype=np.float64)) ** 2) / B


def gradients(params, sizes, X, T):
    W1, b1, W2, b2, W3, b3 = unpack(params, sizes)
    y, (X, z1, a1, z2, a2) = forward(params, sizes, X)
    B = y.shape[0]
    dy = (y - np.asarray(T, dtype=np.float64)) / B      # d loss / d y
    gW3 = dy.T @ a2
    gb3 = dy.sum(axis=0)
    da2 = dy @ W3
    dz2 = da2 * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ W2
    dz1 = da1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


class Adam:
    """Adam with bias correction (Kingma and Ba, 2015) and decoupled weight
    decay (Loshchilov and Hutter, 2019), FP64:
    m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, t <- t + 1,
    P <- P - lr (m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + wd P)."""

    def __init__(self, n, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.b1, self.b2, self.eps = b1, b2, eps

    def step(self, params, grad, lr, wd=0.0):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return params - lr * (mh / (np.sqrt(vh) + self.eps) + wd * params)
