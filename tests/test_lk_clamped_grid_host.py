"""The index design of the tracking kernel's clamped path (CPU only). Points whose 13x13
input patch leaves the frame are tracked on a grid of the clamped rows and columns
within 4 of the point: one half-warp lane per input row for the horizontal Gaussian,
one lane per grid row for the vertical Gaussian (its five taps fetched from the lanes
that hold the clamped rows), one lane per window row for the Sobel and the 7x7 sums
(grid columns selected by index). This test replays that index arithmetic in numpy --
lane by lane, shuffle by shuffle -- for every pixel of tiny and narrow frames, and
checks the window sums against the oracle's clamped definition (Ix, Iy of the smoothed
frame over 8, It the difference of the smoothed frames). Kernel units: the smoothed
frame is 65280 times the oracle's, so A is 65280^2 * 64 and b 65280^2 * 8 times the
oracle's sums."""
import numpy as np
import pytest

from oracle import chain as oc


def clampi(v, lo, hi):
    return lo if v < lo else (hi if v > hi else v)


def grid_sums(fc, fp, p):
    """The five window sums of point p (raster index) the way the clamped path forms them."""
    H, W = fc.shape
    py, px = divmod(p, W)
    r0, c0 = max(py - 4, 0), max(px - 4, 0)
    nr, nc = min(py + 4, H - 1) - r0 + 1, min(px + 4, W - 1) - c0 + 1
    q0 = max(r0 - 2, 0)
    nq = min(r0 + nr - 1 + 2, H - 1) - q0 + 1
    assert nr <= 9 and nc <= 9 and nq <= 13  # grid and input rows fit a half-warp
    # horizontal pass: lane j -> input row q0 + min(j, nq - 1)
    h_c = np.zeros((16, 9))
    h_p = np.zeros((16, 9))
    for lane in range(16):
        y = q0 + min(lane, nq - 1)
        rc, rp = fc[y].astype(np.float64), fp[y].astype(np.float64)
        bc = [rc[clampi(c0 - 2 + j, 0, W - 1)] for j in range(13)]
        bp = [rp[clampi(c0 - 2 + j, 0, W - 1)] for j in range(13)]
        inner = c0 >= 2 and c0 + 10 <= W - 1
        for j in range(9):
            if inner:
                h_c[lane, j] = bc[j] + bc[j + 4] + 4 * (bc[j + 1] + bc[j + 3]) + 6 * bc[j + 2]
                h_p[lane, j] = bp[j] + bp[j + 4] + 4 * (bp[j + 1] + bp[j + 3]) + 6 * bp[j + 2]
            else:
                x = c0 + min(j, nc - 1)
                t = [clampi(x + k, 0, W - 1) for k in (-2, -1, 0, 1, 2)]
                h_c[lane, j] = rc[t[0]] + rc[t[4]] + 4 * (rc[t[1]] + rc[t[3]]) + 6 * rc[t[2]]
                h_p[lane, j] = rp[t[0]] + rp[t[4]] + 4 * (rp[t[1]] + rp[t[3]]) + 6 * rp[t[2]]
    # vertical pass: lane i -> grid row r0 + min(i, nr - 1), taps shuffled from input lanes
    g_c = np.zeros((16, 9))
    g_p = np.zeros((16, 9))
    for lane in range(16):
        y = r0 + min(lane, nr - 1)
        src = [clampi(y + k - 2, 0, H - 1) - q0 for k in range(5)]
        assert all(0 <= s < 16 for s in src)
        for j in range(9):
            a = [h_c[s, j] for s in src]
            b = [h_p[s, j] for s in src]
            g_c[lane, j] = (a[0] + a[4]) + 4 * (a[1] + a[3]) + 6 * a[2]
            g_p[lane, j] = (b[0] + b[4]) + 4 * (b[1] + b[3]) + 6 * b[2]
    # window rows: lane d < 7 -> row dy = d - 3; grid rows and columns by index
    sums = np.zeros(5)
    for lane in range(7):
        qy = clampi(py + lane - 3, 0, H - 1)
        lm, l0, lp = clampi(qy - 1, 0, H - 1) - r0, qy - r0, clampi(qy + 1, 0, H - 1) - r0
        assert all(0 <= v < nr for v in (lm, l0, lp))
        for dx in range(-3, 4):
            qx = clampi(px + dx, 0, W - 1)
            xm, x0, xq = clampi(qx - 1, 0, W - 1) - c0, qx - c0, clampi(qx + 1, 0, W - 1) - c0
            assert all(0 <= v < nc for v in (xm, x0, xq))
            ix = (g_c[lm, xq] - g_c[lm, xm]) + 2 * (g_c[l0, xq] - g_c[l0, xm]) + (g_c[lp, xq] - g_c[lp, xm])
            iy = (g_c[lp, xm] - g_c[lm, xm]) + 2 * (g_c[lp, x0] - g_c[lm, x0]) + (g_c[lp, xq] - g_c[lm, xq])
            it = g_c[l0, x0] - g_p[l0, x0]
            sums += [ix * ix, ix * iy, iy * iy, ix * it, iy * it]
    return sums


def oracle_sums(fc, fp, p):
    """The oracle's clamped 7x7 window sums (gx = Ix / 8, gy = Iy / 8, gt = g_t - g_t-1)."""
    H, W = fc.shape
    maps, _, _ = oc.chain_frame(fc)
    g_prev = oc.gauss_v(oc.gauss_h(oc.convert(fp)))
    py, px = divmod(p, W)
    s = np.zeros(5)
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            q = (clampi(py + dy, 0, H - 1), clampi(px + dx, 0, W - 1))
            gx, gy, gt = maps["ix"][q] / 8, maps["iy"][q] / 8, maps["g"][q] - g_prev[q]
            s += [gx * gx, gx * gy, gy * gy, gx * gt, gy * gt]
    return s


@pytest.mark.parametrize("H,W", [(1, 1), (1, 7), (7, 1), (5, 6), (9, 3), (12, 13), (13, 20)])
def test_clamped_grid_gives_the_clamped_window_sums(H, W):
    rng = np.random.default_rng(H * 100 + W)
    fc = rng.integers(0, 256, (H, W), dtype=np.uint8)
    fp = np.clip(fc.astype(int) + rng.integers(-9, 10, (H, W)), 0, 255).astype(np.uint8)
    scale = 65280.0 ** 2 * np.array([64, 64, 64, 8, 8])
    for p in range(H * W):
        got = grid_sums(fc, fp, p)
        exp = oracle_sums(fc, fp, p) * scale
        tol = 1e-9 * max(1.0, float(np.max(np.abs(exp))))
        assert np.allclose(got, exp, rtol=1e-9, atol=tol), (p, got, exp)
