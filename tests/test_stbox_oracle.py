"""Pins of the spatio-temporal group's reference (CPU only): the temporal binomial's impulse
response, start clamp and delay of a ramp in time; the integer chain against the FP64
chain on real values built from the pinned stage functions of the paper's own chain; a
ramp whose gradient magnitude is exactly the threshold; a brute-force evaluation with exact rationals; the clipped box reads by enumeration; and
Eq. 6 as the maximiser of Eq. 3 for this group's reaches."""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

from oracle import partition as opart
from oracle import stbox as ost


def _gray_video(vals):
    """[T, H, W, 4] RGBA with R = G = B = v (gray numerator 256 v)."""
    v = np.asarray(vals, dtype=np.uint8)
    out = np.zeros(v.shape + (4,), dtype=np.uint8)
    out[..., 0] = out[..., 1] = out[..., 2] = v
    out[..., 3] = 255
    return out


@pytest.mark.parametrize("n", ost.TAPS)
def test_temporal_impulse_is_the_binomial_row(n):
    T = 9
    vals = np.zeros((T, 2, 3), dtype=np.uint8)
    vals[3] = 100
    g = ost.gray_int(_gray_video(vals))
    for t in range(T):
        k = 3 - t + n
        w = comb(n, k) if 0 <= k <= n else 0
        np.testing.assert_array_equal(ost.temporal_int(g, t, n), w * 25600)


@pytest.mark.parametrize("n", ost.TAPS)
def test_temporal_start_clamp_and_ramp_delay(n):
    T = 8
    const = ost.gray_int(_gray_video(np.full((T, 2, 2), 40, dtype=np.uint8)))
    for t in range(T):
        np.testing.assert_array_equal(ost.temporal_int(const, t, n), (1 << n) * 256 * 40)
    ramp = ost.gray_int(_gray_video(np.array([np.full((2, 2), 10 + 3 * t) for t in range(T)], dtype=np.uint8)))
    for t in range(n, T):
        # the binomial weights are symmetric: a linear signal comes out delayed by n/2
        exp = (1 << n) * 256 * (10 * 2 + 3 * (2 * t - n)) // 2
        np.testing.assert_array_equal(ost.temporal_int(ramp, t, n), exp)


def test_gauss_and_magnitude_integers():
    z = np.zeros((7, 8), dtype=np.int64)
    z[3, 4] = 1
    exp = np.zeros_like(z)
    exp[2:5, 3:6] = np.outer([1, 2, 1], [1, 2, 1])
    np.testing.assert_array_equal(ost.gauss_int(z), exp)
    yy, xx = np.mgrid[0:6, 0:7]
    G = 5 * xx - 3 * yy
    M = ost.magnitude_int(G)
    np.testing.assert_array_equal(M[1:-1, 1:-1], 8 * 5 + 8 * 3)
    np.testing.assert_array_equal(M[1:-1, 0], 4 * 5 + 8 * 3)  # one-sided x at the clamped left edge


@pytest.mark.parametrize("n", ost.TAPS)
def test_integer_chain_equals_the_real_valued_chain(n):
    rng = np.random.default_rng(10 + n)
    fr = rng.integers(0, 256, size=(6, 11, 13, 4), dtype=np.uint8)
    fr[..., 1] = fr[..., 0] // 2 + 60  # correlated channels, some smooth areas
    fr[2:, 4:8, 3:9, :3] = 200
    masks, counts, M_int = ost.chain_volume(fr, n, keep_m=True)
    masks_r, M_r = ost.chain_volume_real(fr, n)
    scale = 65280.0 * (1 << n) * 16
    np.testing.assert_allclose(M_int / scale, M_r, rtol=1e-12, atol=1e-12)
    clear = np.abs(M_r - ost.TAU) > 1e-9
    assert clear.mean() > 0.99
    np.testing.assert_array_equal(masks[clear], masks_r[clear])
    np.testing.assert_array_equal(counts, masks.reshape(6, -1).sum(axis=1))


@pytest.mark.parametrize("n", ost.TAPS)
def test_a_magnitude_exactly_at_the_threshold_is_not_marked(n):
    # gray grows by (77 * 4 + 150 * 10 + 29 * b) per column; with b = 8 that is 2040, and
    # the integer magnitude 2040 * 8 (Sobel) * 16 (3x3 weights) * 2^n (temporal weights)
    # = 261120 * 2^n is the threshold itself at every column two or more from the edges
    def ramp(b):
        x = np.arange(26)
        fr = np.zeros((n + 2, 5, 26, 4), dtype=np.uint8)
        fr[..., 0], fr[..., 1], fr[..., 2], fr[..., 3] = 4 * x, 10 * x, b * x, 255
        return fr
    masks, counts, M = ost.chain_volume(ramp(8), n, keep_m=True)
    assert (M[:, :, 2:-2] == 261120 * 2 ** n).all() and not masks.any() and not counts.any()
    masks_r, M_r = ost.chain_volume_real(ramp(8), n)
    assert (M_r[:, :, 2:-2] == ost.TAU).all() and not masks_r.any()
    masks, _, _ = ost.chain_volume(ramp(9), n)
    assert masks[:, :, 2:-2].all() and not masks[:, :, :2].any() and not masks[:, :, -2:].any()


def test_brute_force_with_exact_rationals():
    rng = np.random.default_rng(3)
    T, H, W, n = 3, 4, 5, 2
    fr = rng.integers(0, 256, size=(T, H, W, 4), dtype=np.uint8)
    masks, counts, _ = ost.chain_volume(fr, n)

    def Y(t, y, x):
        t, y, x = max(t, 0), min(max(y, 0), H - 1), min(max(x, 0), W - 1)
        r, g, b = (int(c) for c in fr[t, y, x, :3])
        return Fraction(77 * r + 150 * g + 29 * b, 65280)

    def z(t, y, x):
        return sum(comb(n, k) * Y(t - n + k, y, x) for k in range(n + 1)) / (1 << n)

    def G(t, y, x):
        y, x = min(max(y, 0), H - 1), min(max(x, 0), W - 1)
        w = (1, 2, 1)
        return sum(w[a] * w[b] * z(t, y + a - 1, x + b - 1) for a in range(3) for b in range(3)) / 16

    for t in range(T):
        for y in range(H):
            for x in range(W):
                gx = sum((1, 2, 1)[d + 1] * (G(t, y + d, x + 1) - G(t, y + d, x - 1)) for d in (-1, 0, 1))
                gy = sum((1, 2, 1)[d + 1] * (G(t, y + 1, x + d) - G(t, y - 1, x + d)) for d in (-1, 0, 1))
                assert masks[t, y, x] == int(abs(gx) + abs(gy) > Fraction(1, 4)), (t, y, x)
    assert counts.tolist() == [int(masks[t].sum()) for t in range(T)]


@pytest.mark.parametrize("W,H,T,x,t,n", [(13, 9, 7, 4, 3, 2), (8, 8, 8, 4, 4, 1), (10, 6, 5, 8, 2, 4)])
def test_clipped_box_reads_by_enumeration(W, H, T, x, t, n):
    total = 0
    for t0 in range(0, T, t):
        for y0 in range(0, H, x):
            for x0 in range(0, W, x):
                pts = {(tt, yy, xx)
                       for tt in range(t0 - n, min(t0 + t, T)) for yy in range(y0 - ost.DX, y0 + x + ost.DX)
                       for xx in range(x0 - ost.DX, x0 + x + ost.DX)
                       if 0 <= tt and 0 <= yy < H and 0 <= xx < W}
                total += len(pts)
    assert ost.box_exact_reads(W, H, T, x, t, n) == total


def test_model_bytes_counts_boxes():
    # 64 x 64 x 32 volume, 16 x 16 x 8 boxes: 4 * 4 * 4 = 64 boxes of 20^2 * (8 + 2) reads
    assert ost.box_model_bytes(64, 64, 32, 16, 8, 2) == 64 * (400 * 10 * 4 + 256 * 8)


@pytest.mark.parametrize("beta,n", [(4096, 2), (16384, 2), (16384, 4), (65536, 1)])
def test_eq6_maximises_data_utilisation(beta, n):
    x6, t6 = opart.eq6_box(beta, ost.DX, n)
    du6 = ost.data_utilisation(x6, t6, n)
    for f in (0.8, 0.9, 1.1, 1.25):
        x = x6 * f
        assert ost.data_utilisation(x, beta / (x * x), n) < du6
