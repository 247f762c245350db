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


def _fp32_run(rows, frame_u8):
    """The DAG evaluated in float32, written independently of the oracle's stage code:
    every product and sum rounded to float32 (no fused multiply-add), stencils as two
    passes of recursive sums over clamped neighbours, in the order the stage lists its
    taps."""
    f32 = np.float32
    H, W = frame_u8.shape
    ys = lambda d: np.clip(np.arange(H) + d, 0, H - 1)  # noqa: E731
    xs = lambda d: np.clip(np.arange(W) + d, 0, W - 1)  # noqa: E731
    nodes = [frame_u8.astype(f32) * f32(1.0 / 255.0)]
    for kind, i1, i2, r, a, b in rows:
        x = nodes[i1]
        if kind == 1:
            y = f32(a) * x + f32(b)
        elif kind == 2:
            y = np.abs(x)
        elif kind == 3:
            y = np.clip(x * nodes[i2], f32(-16), f32(16))
        elif kind == 4:
            w = [f32(v) for v in od.binomial_weights(r)]
            y = np.zeros_like(x)
            for iy, dy in enumerate(range(-r, r + 1)):
                row = np.zeros_like(x)
                for ix, dx in enumerate(range(-r, r + 1)):
                    row = w[ix] * x[np.ix_(ys(dy), xs(dx))] + row
                y = w[iy] * row + y
        else:
            y = x.copy()
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    y = np.maximum(y, x[np.ix_(ys(dy), xs(dx))])
        nodes.append(y.astype(f32))
    return nodes


@pytest.mark.parametrize("seed,deep", [(1, False), (2, False), (3, False), (5013, True), (5012, True)])
def test_fp32_error_bound_holds_for_a_float32_evaluation(seed, deep):
    """The per-pixel FP32 error bound (running error analysis of the stage definitions)
    covers every node of an independent float32 evaluation of random and deep DAGs, and
    is tight enough to be a useful tolerance (within 1e-5 of the output's magnitude)."""
    from synth import video as sv
    rows = sd.to_array(sd.deep_dag(seed) if deep else sd.random_dag(seed))
    fr, _ = sv.generate(sv.VideoSpec(T=1, H=40, W=56, seed=seed, n_blobs=4, n_patches=2), pitch=64)
    f = fr[0][:, :56]
    ref = od.run_frame(rows, f)
    got = _fp32_run(rows, f)
    bound = od.fp32_error_bounds(rows, f)
    for i, (g, r, e) in enumerate(zip(got, ref, bound)):
        err = np.abs(g.astype(np.float64) - r)
        assert np.all(err <= e), (i, float(np.max(err - e)))
    assert np.max(bound[-1]) <= 1e-5 * np.max(np.abs(ref[-1]))


def test_fp32_error_bound_by_hand():
    """Hand values: node 0 gets 2u|x|; an affine stage |a| e + u(2|a x| + |b| + |y|); a
    product |x1| e2 + |x2| e1 + e1 e2 plus u times |x1 x2| and that; abs passes e on."""
    u, g = od.U32, 1.0 + 2.0 ** -10
    f = np.array([[51]], dtype=np.uint8)  # x0 = 0.2
    rows = [(1, 0, -1, 0, -1.5, 0.25), (3, 1, 0, 0, 0.0, 0.0), (2, 2, -1, 0, 0.0, 0.0)]
    e = od.fp32_error_bounds(rows, f)
    e0 = 2 * u * 0.2 * g
    assert e[0][0, 0] == pytest.approx(e0, rel=1e-12)
    y1 = -1.5 * 0.2 + 0.25
    e1 = (1.5 * e0 + u * (2 * 1.5 * 0.2 + 0.25 + abs(y1))) * g
    assert e[1][0, 0] == pytest.approx(e1, rel=1e-12)
    ex = abs(y1) * e0 + 0.2 * e1 + e1 * e0
    assert e[2][0, 0] == pytest.approx((ex + u * (abs(y1) * 0.2 + ex)) * g, rel=1e-12)
    assert e[3][0, 0] == pytest.approx(e[2][0, 0] * g, rel=1e-12)


def test_fp32_error_bound_of_stencil_and_max_by_hand():
    """A radius-1 stencil of a constant frame: e0 + 2 * 3 * u * (x + e0) (the weights sum
    to 1); a 3x3 maximum takes the largest input bound of the window, here set by a bright
    pixel next to the centre."""
    u, g = od.U32, 1.0 + 2.0 ** -10
    f = np.full((5, 5), 51, dtype=np.uint8)
    e = od.fp32_error_bounds([(4, 0, -1, 1, 0.0, 0.0)], f)
    e0 = 2 * u * 0.2 * g
    np.testing.assert_allclose(e[1], (e0 + 6 * u * (0.2 + e0)) * g, rtol=1e-12)
    f2 = np.full((5, 5), 51, dtype=np.uint8)
    f2[2, 3] = 255
    e2 = od.fp32_error_bounds([(5, 0, -1, 1, 0.0, 0.0)], f2)
    big, small = 2 * u * 1.0 * g, 2 * u * 0.2 * g
    assert e2[1][2, 2] == pytest.approx(big * g, rel=1e-12)  # the bright pixel is in its window
    assert e2[1][2, 0] == pytest.approx(small * g, rel=1e-12)  # it is not
    assert e2[1][0, 4] == pytest.approx(small * g, rel=1e-12)
