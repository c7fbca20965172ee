"""Float64 reference of the row-size predictor (not in the paper: the learned
sizing of the output is an addition on top of the paper's method).

TEST INFRASTRUCTURE ONLY.

Network: x (F features) -> h1 = relu(W1 x + b1) (32) -> h2 = relu(W2 h1 + b2)
(32) -> y = w3 . h2 + b3.  Loss = mean over samples of (y - t)^2 / 2.
Parameters are one flat vector in the order W1 (32 x F, row-major), b1 (32),
W2 (32 x 32, row-major), b2 (32), w3 (32), b3 (1).

Row features (all log2(1 + .)): flops_i, |A(i,:)|, max_k |B(k,:)|, n,
flops_i / |A(i,:)|, min(flops_i, n); target log2(1 + nnz(C(i,:))).
"""
from __future__ import annotations

import numpy as np

H = 32
F = 6


def param_count(F: int = F) -> int:
    return H * F + H + H * H + H + H + 1


def unpack(p: np.ndarray, F: int = F):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p, X.shape[1])
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(p, X, t):
    """Mean squared-error loss / 2 and its gradient by backpropagation."""
    W1, b1, W2, b2, w3, b3 = unpack(p, X.shape[1])
    y, (X, z1, h1, z2, h2) = forward(p, X)
    N = X.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = 0.5 * np.mean(r * r)
    dy = r / N
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dh2 = np.outer(dy, w3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g


def row_features(A, B) -> np.ndarray:
    """Feature matrix (m x F, float64) of the rows of A.B, from the patterns."""
    rp = np.asarray(A.rowptr, dtype=np.int64)
    col = np.asarray(A.col, dtype=np.int64)
    lenB = np.diff(np.asarray(B.rowptr, dtype=np.int64))
    d = np.diff(rp)
    rows = np.repeat(np.arange(A.nrows), d)
    kl = lenB[col]
    flops = np.bincount(rows, weights=kl, minlength=A.nrows)
    mx = np.zeros(A.nrows)
    np.maximum.at(mx, rows, kl)
    n = float(B.ncols)
    mean = np.where(d > 0, flops / np.maximum(d, 1), 0.0)
    X = np.stack([flops, d, mx, np.full(A.nrows, n), mean, np.minimum(flops, n)], axis=1)
    return np.log2(1.0 + X)
