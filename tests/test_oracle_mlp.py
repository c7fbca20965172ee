"""Pins for the float64 predictor reference: analytic gradients against
central finite differences, and the feature map against its definition on a
hand-checkable product."""
import numpy as np

import oracle
from oracle import mlp
from paper_1510_00844_gb300 import inputs


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, mlp.F)) * 2
    t = rng.normal(size=40)
    p = rng.normal(size=mlp.param_count()) * 0.3
    loss, g = mlp.loss_and_grad(p, X, t)
    h = 1e-6
    idx = rng.choice(p.size, 60, replace=False)
    for q in idx:
        e = np.zeros_like(p)
        e[q] = h
        fd = (mlp.loss_and_grad(p + e, X, t)[0] - mlp.loss_and_grad(p - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q])), q


def test_forward_is_the_stated_network():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(5, mlp.F))
    p = rng.normal(size=mlp.param_count())
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    for s in range(5):
        h1 = [max(0.0, sum(W1[j, f] * X[s, f] for f in range(mlp.F)) + b1[j]) for j in range(32)]
        h2 = [max(0.0, sum(W2[j, k] * h1[k] for k in range(32)) + b2[j]) for j in range(32)]
        y = sum(w3[j] * h2[j] for j in range(32)) + b3
        assert abs(mlp.forward(p, X[s:s + 1])[0][0] - y) <= 1e-12 * max(1, abs(y))


def test_row_features_definition():
    # A row 0 = {0, 2}, row 1 = {}, row 2 = {1}; B rows of length 3, 1, 2; n = 7
    A = inputs.CSR(3, 3, np.array([0, 2, 2, 3]), np.array([0, 2, 1]), np.ones(3))
    B = inputs.CSR(3, 7, np.array([0, 3, 4, 6]), np.array([0, 1, 2, 5, 3, 6]), np.ones(6))
    X = mlp.row_features(A, B)
    fl, d, mx, n = 5.0, 2.0, 3.0, 7.0
    np.testing.assert_allclose(X[0], np.log2(1 + np.array([fl, d, mx, n, fl / d, min(fl, n)])))
    np.testing.assert_allclose(X[1], np.log2(1 + np.array([0, 0, 0, n, 0, 0])))
    assert oracle.row_flops(A, B).tolist() == [5, 0, 1]
