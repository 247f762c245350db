"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (CPU only).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong
sign, a swapped operand or index, a wrong border rule) fails at least one of them:
closed forms on ramps and impulses, symmetry of a checkerboard, brute force on tiny
maps, a linear solve checked by numpy, and a known translation recovered by tracking.
"""
import itertools

import numpy as np
import pytest

from oracle import chain as oc

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------- Gaussian stages
def test_gauss_constant_frame_stays_constant():
    f = np.full((17, 23), 77, dtype=np.uint8)
    maps, mask, c = oc.chain_frame(f)
    assert np.all(maps["f"] == 77 / 255)
    assert np.all(maps["g1"] == 77 / 255)  # taps sum to exactly one, borders included
    assert np.all(maps["g"] == 77 / 255)


def test_gauss_impulse_response_is_binomial():
    f = np.zeros((13, 15), dtype=np.uint8)
    f[6, 7] = 255
    w = np.array([1, 4, 6, 4, 1]) / 16
    g1 = oc.gauss_h(oc.convert(f))
    exp = np.zeros((13, 15))
    exp[6, 5:10] = w  # horizontal pass touches only the impulse row
    np.testing.assert_allclose(g1, exp, atol=1e-15)
    g = oc.gauss_v(g1)
    exp2 = np.zeros((13, 15))
    exp2[4:9, 5:10] = np.outer(w, w)
    np.testing.assert_allclose(g, exp2, atol=1e-15)


def test_gauss_clamps_its_own_input_at_the_border():
    f = np.zeros((8, 9), dtype=np.uint8)
    f[0, 0] = 255
    g1 = oc.gauss_h(oc.convert(f))
    np.testing.assert_allclose(g1[0, :4], [11 / 16, 5 / 16, 1 / 16, 0], atol=1e-15)
    g = oc.gauss_v(g1)
    np.testing.assert_allclose(g[:4, 0], np.array([11, 5, 1, 0]) / 16 * 11 / 16, atol=1e-15)
    # the bottom-left corner of a frame taller than wide: rows clamp at H - 1, columns at W - 1
    f = np.zeros((20, 3), dtype=np.uint8)
    f[19, 0] = 255
    g1 = oc.gauss_h(oc.convert(f))
    np.testing.assert_allclose(g1[19], [11 / 16, 5 / 16, 1 / 16], atol=1e-15)
    g = oc.gauss_v(g1)
    np.testing.assert_allclose(g[16:, 0], np.array([0, 1, 5, 11]) / 16 * 11 / 16, atol=1e-15)


def test_gauss_passes_commute():
    f = oc.convert(RNG.integers(0, 256, (21, 19), dtype=np.uint8))
    np.testing.assert_allclose(oc.gauss_v(oc.gauss_h(f)), oc.gauss_h(oc.gauss_v(f)),
                               atol=1e-14)


# ---------------------------------------------------------------- ramp closed forms
ALPHA, BETA = 2, 3


def ramp(H=40, W=50):
    y, x = np.mgrid[0:H, 0:W]
    return (ALPHA * x + BETA * y).astype(np.uint8)


def test_sobel_impulse_response_is_the_sobel_kernel():
    # g = a unit impulse at (4, 5): Ix(y, x) = sum_dy s(dy) (g(y+dy, x+1) - g(y+dy, x-1))
    # puts +s on column 4 and -s on column 6 (rows 3..5), Iy the same transposed
    g = np.zeros((9, 11))
    g[4, 5] = 1.0
    ix, iy = oc.sobel(g)
    exp_x = np.zeros_like(g)
    exp_x[3:6, 4], exp_x[3:6, 6] = [1, 2, 1], [-1, -2, -1]
    exp_y = np.zeros_like(g)
    exp_y[3, 4:7], exp_y[5, 4:7] = [1, 2, 1], [-1, -2, -1]
    np.testing.assert_array_equal(ix, exp_x)
    np.testing.assert_array_equal(iy, exp_y)


def test_sobel_on_a_ramp_gives_the_closed_form():
    maps, _, _ = oc.chain_frame(ramp())
    ix, iy = maps["ix"][3:-3, 3:-3], maps["iy"][3:-3, 3:-3]
    np.testing.assert_allclose(ix, 8 * ALPHA / 255, rtol=1e-12)  # x is the column axis
    np.testing.assert_allclose(iy, 8 * BETA / 255, rtol=1e-12)


def test_structure_tensor_and_response_on_a_ramp():
    maps, mask, count = oc.chain_frame(ramp())
    a, b = ALPHA / 255, BETA / 255
    sl = (slice(5, -5), slice(5, -5))
    np.testing.assert_allclose(maps["sxx"][sl], 1600 * a * a, rtol=1e-12)
    np.testing.assert_allclose(maps["sxy"][sl], 1600 * a * b, rtol=1e-12)
    np.testing.assert_allclose(maps["syy"][sl], 1600 * b * b, rtol=1e-12)
    r_exp = -0.04 * (1600 * (a * a + b * b)) ** 2  # det = 0 on a ramp
    np.testing.assert_allclose(maps["r"][sl], r_exp, rtol=1e-9)
    assert r_exp == pytest.approx(-4.0946e-3, rel=1e-3)
    assert not mask[sl].any()


def test_constant_frame_has_no_gradient_no_response_no_corner():
    maps, mask, count = oc.chain_frame(np.full((30, 40), 200, dtype=np.uint8))
    for k in ("ix", "iy", "sxx", "sxy", "syy", "r"):
        assert np.all(maps[k] == 0.0), k
    assert count == 0 and not mask.any()


# ---------------------------------------------------------------- box, Harris
def test_box_impulse_and_corner_clamp():
    m = np.zeros((12, 12))
    m[5, 6] = 1.0
    exp = np.zeros((12, 12))
    exp[3:8, 4:9] = 1.0
    np.testing.assert_array_equal(oc.box5(m), exp)
    m = np.zeros((12, 12))
    m[0, 0] = 1.0
    bx = oc.box5(m)
    assert bx[0, 0] == 9 and bx[0, 1] == 6 and bx[1, 1] == 4 and bx[2, 2] == 1
    assert bx[3, 3] == 0 and bx[0, 3] == 0


def test_harris_hand_value():
    sxx, sxy, syy = np.array([2.0]), np.array([1.0]), np.array([3.0])
    assert oc.harris(sxx, sxy, syy)[0] == pytest.approx(5 - 0.04 * 25, abs=1e-15)
    assert oc.harris(sxx, sxy, syy, k=0.0)[0] == pytest.approx(5.0, abs=1e-15)
    # the off-diagonal enters squared and only once
    assert oc.harris(sxx, -sxy, syy)[0] == oc.harris(sxx, sxy, syy)[0]
    assert oc.harris(syy, sxy, sxx)[0] == oc.harris(sxx, sxy, syy)[0]


# ---------------------------------------------------------------- NMS
def nms_brute(r, thr):
    H, W = r.shape
    mask = np.zeros((H, W), dtype=np.uint8)
    for y, x in itertools.product(range(H), range(W)):
        nb = [r[y + dy, x + dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if 0 <= y + dy < H and 0 <= x + dx < W]
        mask[y, x] = r[y, x] > thr and r[y, x] >= max(nb)
    return mask


@pytest.mark.parametrize("seed", range(6))
def test_nms_matches_brute_force_on_tiny_maps(seed):
    rng = np.random.default_rng(seed)
    H, W = rng.integers(1, 9, size=2)
    r = rng.integers(-3, 4, size=(H, W)).astype(np.float64) * 1e-5  # plateaus and ties
    for thr in (1e-5, 0.0, -1.0):
        mask, count = oc.nms(r, thr)
        exp = nms_brute(r, thr)
        np.testing.assert_array_equal(mask, exp)
        assert count == exp.sum()


def test_nms_threshold_is_strict():
    r = np.full((5, 5), 1e-5)
    r[2, 2] = 2e-5
    mask, c = oc.nms(r, 1e-5)
    assert c == 1 and mask[2, 2] == 1


def _checker(H, W, x0, y0):
    def s(d):
        return np.where(d % 16 == 0, 0, np.where((d // 16) % 2 == 0, 1, -1))
    y, x = np.arange(H), np.arange(W)
    return (110 + 40 * s(y - y0)[:, None] * s(x - x0)[None, :]).astype(np.uint8)


def test_checkerboard_corners_sit_at_the_diagonal_neighbours_of_every_vertex():
    # f = 110 + 40 s(x-x0) s(y-y0) with s(0) = 0: every vertex lies on a zero-contrast
    # cross, R is even about it in x and in y, and its maxima are the four diagonal
    # neighbours (confirmed on this oracle before any GPU code existed).
    H, W, x0, y0 = 96, 128, 8, 8
    maps, mask, count = oc.chain_frame(_checker(H, W, x0, y0))
    got = set(zip(*[a.tolist() for a in np.nonzero(mask)]))
    exp = {(vy + dy, vx + dx) for vx in range(x0, W, 16) for vy in range(y0, H, 16)
           for dx in (-1, 1) for dy in (-1, 1)}
    assert got == exp and count == len(exp) == 192
    r = maps["r"]
    np.testing.assert_allclose(r[y0 - 3:y0 + 4, x0 - 3:x0 + 4], r[y0 - 3:y0 + 4, x0 - 3:x0 + 4][:, ::-1],
                               rtol=1e-12)
    np.testing.assert_allclose(r[y0 - 3:y0 + 4, x0 - 3:x0 + 4], r[y0 - 3:y0 + 4, x0 - 3:x0 + 4][::-1, :],
                               rtol=1e-12)


# ---------------------------------------------------------------- chain wiring
def test_chain_equals_the_stages_composed_one_by_one():
    f = RNG.integers(0, 256, (23, 31), dtype=np.uint8)
    maps, mask, count = oc.chain_frame(f)
    g = oc.gauss_v(oc.gauss_h(oc.convert(f)))
    ix, iy = oc.sobel(g)
    p = oc.products(ix, iy)
    s = [oc.box5(q) for q in p]
    r = oc.harris(*s)
    m2, c2 = oc.nms(r)
    for k, v in zip(("g", "ix", "iy", "sxx", "sxy", "syy", "r"), (g, ix, iy, *s, r)):
        np.testing.assert_array_equal(maps[k], v)
    np.testing.assert_array_equal(mask, m2)
    assert count == c2


def test_chain_volume_matches_frames_and_uses_threads():
    f = RNG.integers(0, 256, (5, 20, 32), dtype=np.uint8)
    masks, counts, r, used = oc.chain_volume(f, W=29, want_r=True)
    assert used >= 1
    for t in range(5):
        maps, m, c = oc.chain_frame(f[t][:, :29].copy())
        np.testing.assert_array_equal(masks[t, :, :29], m)
        assert not masks[t, :, 29:].any()
        assert counts[t] == c
        np.testing.assert_array_equal(r[t], maps["r"])


# ---------------------------------------------------------------- tracking
def test_select_points_orders_by_response_then_raster_index():
    rng = np.random.default_rng(7)
    r = rng.integers(0, 5, size=(9, 11)).astype(np.float64)
    mask = (rng.random((9, 11)) < 0.4).astype(np.uint8)
    cand = [(-r.flat[i], i) for i in range(r.size) if mask.flat[i]]
    exp = [i for _, i in sorted(cand)]
    for K in (1, 5, len(exp), len(exp) + 3):
        got = oc.select_points(r, mask, K)
        assert got.tolist() == exp[:K]


def test_lk_solve_agrees_with_numpy_and_flags_singular_windows():
    rng = np.random.default_rng(3)
    H = W = 9
    ix, iy = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    gp, gc = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    idx = np.array([4 * W + 4], dtype=np.int32)
    u, v, st = oc.lk(gp, gc, ix, iy, idx, win=3)
    sl = (slice(1, 8), slice(1, 8))
    gx, gy, gt = ix[sl] / 8, iy[sl] / 8, (gc - gp)[sl]
    A = np.array([[np.sum(gx * gx), np.sum(gx * gy)], [np.sum(gx * gy), np.sum(gy * gy)]])
    b = np.array([np.sum(gx * gt), np.sum(gy * gt)])
    np.testing.assert_allclose([u[0], v[0]], np.linalg.solve(A, -b), rtol=1e-10)
    assert st[0] == 0
    z = np.zeros((H, W))
    u, v, st = oc.lk(gp, gc, z, z, idx, win=3)
    assert st[0] == 1 and u[0] == 0 and v[0] == 0
    # a rank-one window (gradient along x only) is singular as well
    u, v, st = oc.lk(gp, gc, ix, z, idx, win=3)
    assert st[0] == 1


def _blobs(H, W, dx, dy):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.full((H, W), 100.0)
    for (cx, cy, s, a) in ((30, 28, 5.0, 90), (44, 40, 6.0, -80), (26, 46, 4.5, 70),
                           (50, 22, 5.5, 60)):
        img += a * np.exp(-((x - cx - dx) ** 2 + (y - cy - dy) ** 2) / (2 * s * s))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


@pytest.mark.parametrize("u,v", [(0.6, -0.4), (-0.5, 0.7), (0.0, 0.0)])
def test_lk_recovers_a_known_translation(u, v):
    H, W = 72, 76
    prev, cur = _blobs(H, W, 0, 0), _blobs(H, W, u, v)
    idx, uu, vv, st = oc.track_pair(prev, cur, K=64)
    py, px = idx // W, idx % W
    inner = (px >= 12) & (px < W - 12) & (py >= 12) & (py < H - 12) & (st == 0)
    assert inner.sum() >= 8
    err = np.hypot(uu[inner] - u, vv[inner] - v)
    assert np.median(err) <= 0.1


def test_lk_tracks_slow_checker_patches_of_the_synthetic_video():
    # Ground truth from the generator: every point inside a checker patch (3 px in from
    # its edge, 8 px in from the frame edge) moves with the patch. One linearised LK step
    # is accurate for sub-pixel motion: patches slower than 1 px/frame must come out
    # within 0.25 px/frame (median).
    from synth import video as sv
    spec = sv.VideoSpec(T=6, H=400, W=300, seed=7, n_blobs=16, n_patches=16)
    fr, sc = sv.generate(spec)
    errs = []
    for t in range(1, spec.T):
        idx, u, v, st = oc.track_pair(fr[t - 1], fr[t], K=256)
        py, px = idx // spec.W, idx % spec.W
        X, Y = sc.position(t)
        for i in range(len(idx)):
            if st[i] or not (8 <= px[i] < spec.W - 8 and 8 <= py[i] < spec.H - 8):
                continue
            for o in np.nonzero(sc.kind == 1)[0]:
                dx, dy = (px[i] - X[o]) % spec.W, (py[i] - Y[o]) % spec.H
                if 3 <= dx <= 13 and 3 <= dy <= 13 and np.hypot(sc.vx[o], sc.vy[o]) < 1.0:
                    errs.append(np.hypot(u[i] - sc.vx[o], v[i] - sc.vy[o]))
    assert len(errs) >= 30
    assert np.median(errs) <= 0.25


def test_track_volume_is_track_pair_on_every_frame_pair():
    from synth import video as sv
    fr, _ = sv.generate(sv.VideoSpec(T=4, H=60, W=70, seed=9, n_blobs=6, n_patches=4))
    n, idx, u, v, st, used = oc.track_volume(fr, K=32)
    assert n[0] == 0 and used >= 1
    for t in range(1, 4):
        i2, u2, v2, s2 = oc.track_pair(fr[t - 1], fr[t], K=32)
        assert n[t] == len(i2)
        np.testing.assert_array_equal(idx[t, :n[t]], i2)
        np.testing.assert_array_equal(u[t, :n[t]], u2)
        np.testing.assert_array_equal(v[t, :n[t]], v2)
        np.testing.assert_array_equal(st[t, :n[t]], s2)
