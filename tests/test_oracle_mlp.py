"""Pins for the oracle's rank-predictor network: finite differences and a
hand-computed tiny case."""
import numpy as np

import oracle


def _params(F, H1, H2, NB, rng):
    return rng.standard_normal(oracle.mlp_nparams(F, H1, H2, NB)) * 0.5


def test_gradient_matches_finite_differences():
    F, H1, H2, NB = 5, 7, 6, 4
    rng = np.random.default_rng(0)
    P = _params(F, H1, H2, NB, rng)
    X = rng.standard_normal((9, F))
    y = rng.integers(0, NB, 9)
    loss, g = oracle.mlp_loss_grad(P, X, y, F, H1, H2, NB)
    eps = 1e-6
    num = np.zeros_like(P)
    for i in range(len(P)):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += eps
        Pm[i] -= eps
        num[i] = (oracle.mlp_loss_grad(Pp, X, y, F, H1, H2, NB)[0]
                  - oracle.mlp_loss_grad(Pm, X, y, F, H1, H2, NB)[0]) / (2 * eps)
    np.testing.assert_allclose(g, num, atol=1e-7)


def test_forward_by_hand():
    # 1 feature, 1 hidden, 1 hidden, 2 classes
    F, H1, H2, NB = 1, 1, 1, 2
    P = np.array([2.0, -1.0,   3.0, 0.5,   1.0, -1.0,  0.0, 0.25])
    X = np.array([[1.5], [0.2]])
    lo = oracle.mlp_forward(P, X, F, H1, H2, NB)
    h1 = np.maximum(2 * X[:, 0] - 1, 0)
    h2 = np.maximum(3 * h1 + 0.5, 0)
    np.testing.assert_allclose(lo, np.stack([h2, -h2 + 0.25], 1), atol=1e-15)
    loss, _ = oracle.mlp_loss_grad(P, X, np.array([0, 1], np.int32), F, H1, H2, NB)
    p = np.exp(lo) / np.exp(lo).sum(1, keepdims=True)
    np.testing.assert_allclose(loss, -np.mean(np.log([p[0, 0], p[1, 1]])), atol=1e-14)
