"""Pins of the cost model's reference network (CPU only): its analytic gradient equals
central finite differences of its loss, and a network with zero weights reduces to a
constant whose gradient has a closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    d, n = 12, 7
    p = rng.normal(scale=0.3, size=mlp.n_params(d))
    x, t = rng.normal(size=(n, d)), rng.normal(size=n)
    L, g = mlp.grad(p, x, t)
    assert L == pytest.approx(mlp.loss(p, x, t), rel=1e-14)
    eps = 1e-6
    idx = rng.choice(len(p), size=80, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_zero_weights_give_a_constant_and_its_gradient():
    d, n = 12, 5
    p = np.zeros(mlp.n_params(d))
    p[-1] = 0.7  # b3
    t = np.arange(n, dtype=float)
    x = np.random.default_rng(1).normal(size=(n, d))
    np.testing.assert_array_equal(mlp.forward(p, x), 0.7)
    L, g = mlp.grad(p, x, t)
    assert L == pytest.approx(np.mean((0.7 - t) ** 2))
    assert g[-1] == pytest.approx(np.mean(2 * (0.7 - t)))
    assert np.all(g[:-1] == 0)  # ReLU units are all zero: no other parameter moves
