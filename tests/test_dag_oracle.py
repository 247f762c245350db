"""Pins of the random-DAG oracle and generator (CPU only): binomial weights, impulse
responses and border clamps of the stencil, 3x3 maximum by brute force, saturation of
the product, node 0 as the frame over full scale, and the generator's topological
order."""
import itertools

import numpy as np
import pytest

from oracle import dag as od
from synth import dags as sd


@pytest.mark.parametrize("r,exp", [(0, [1]), (1, [1, 2, 1]), (2, [1, 4, 6, 4, 1]), (3, [1, 6, 15, 20, 15, 6, 1])])
def test_binomial_weights(r, exp):
    w = od.binomial_weights(r)
    np.testing.assert_allclose(w, np.array(exp) / 4.0 ** r)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_stencil_impulse_constant_and_corner(r):
    x = np.zeros((15, 17))
    x[7, 8] = 1.0
    y = od.stage(4, x, None, r, 0, 0)
    w = od.binomial_weights(r)
    exp = np.zeros_like(x)
    exp[7 - r:7 + r + 1, 8 - r:8 + r + 1] = np.outer(w, w)
    np.testing.assert_allclose(y, exp, atol=1e-15)
    np.testing.assert_allclose(od.stage(4, np.full((6, 9), 0.3), None, r, 0, 0), 0.3, rtol=1e-14)
    c = np.zeros((9, 9))
    c[0, 0] = 1.0
    assert od.stage(4, c, None, r, 0, 0)[0, 0] == pytest.approx(w[:r + 1].sum() ** 2, abs=1e-15)


def test_max3_matches_brute_force():
    rng = np.random.default_rng(1)
    for H, W in ((1, 1), (2, 5), (6, 3), (7, 8)):
        x = rng.integers(-3, 4, size=(H, W)).astype(float)
        y = od.stage(5, x, None, 1, 0, 0)
        for i, j in itertools.product(range(H), range(W)):
            nb = [x[a, b] for a in range(max(i - 1, 0), min(i + 2, H)) for b in range(max(j - 1, 0), min(j + 2, W))]
            assert y[i, j] == max(nb)


def test_pointwise_stages():
    x = np.array([[-2.0, 0.5], [3.0, -7.0]])
    z = np.array([[4.0, 2.0], [10.0, 3.0]])
    np.testing.assert_array_equal(od.stage(1, x, None, 0, -1.5, 0.25), -1.5 * x + 0.25)
    np.testing.assert_array_equal(od.stage(2, x, None, 0, 0, 0), np.abs(x))
    np.testing.assert_array_equal(od.stage(3, x, z, 0, 0, 0), [[-8.0, 1.0], [16.0, -16.0]])


def test_node_zero_is_the_frame_in_units_of_full_scale():
    nodes = od.run_frame([(1, 0, -1, 0, 1.0, 0.0)], np.array([[0, 51, 255]], dtype=np.uint8))
    np.testing.assert_array_equal(nodes[0], [[0.0, 0.2, 1.0]])
    np.testing.assert_array_equal(nodes[1], nodes[0])


def test_random_dags_are_topological_and_sized():
    for seed in range(30):
        st = sd.random_dag(seed)
        assert 12 <= len(st) <= 24
        for i, s in enumerate(st, start=1):
            assert 0 <= s.in1 < i and (s.kind != "product" or 0 <= s.in2 < i)
            assert 0 <= s.radius <= 3
    assert sd.random_dag(5) == sd.random_dag(5) and sd.random_dag(5) != sd.random_dag(6)


def test_run_frame_composes_the_stages():
    st = sd.random_dag(3)
    rows = sd.to_array(st)
    f = np.random.default_rng(2).integers(0, 256, (11, 13), dtype=np.uint8)
    nodes = od.run_frame(rows, f)
    assert len(nodes) == len(st) + 1
    for i, (kind, i1, i2, r, a, b) in enumerate(rows, start=1):
        np.testing.assert_array_equal(nodes[i], od.stage(kind, nodes[i1], nodes[i2] if i2 >= 0 else None, r, a, b))
        assert np.all(np.isfinite(nodes[i]))
