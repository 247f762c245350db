"""Pins of the FP64 reference of the paper's own chain (CPU only): gray weights, the IIR
filter's step response in closed form, the 3x3 Gaussian's impulse response and border
clamp, the gradient of ramps (interior and clamped border), threshold and region sums by
brute force, a ramp whose gradient magnitude is exactly the threshold, the Kalman model
(one frame of constant velocity; the process noise as the integral of white acceleration
over a frame), the filter against the steady state of the discrete algebraic Riccati
equation (scipy's solver), noise-free tracking and pure prediction."""
import numpy as np
import pytest

from oracle import pchain as op


def test_gray_weights_sum_to_one_and_pick_channels():
    v = np.arange(256, dtype=np.uint8)
    rgba = np.stack([v, v, v, np.full_like(v, 7)], axis=-1)[None]
    np.testing.assert_allclose(op.gray(rgba)[0], v / 255.0, rtol=0, atol=1e-15)
    pure = np.array([[[255, 0, 0, 0], [0, 255, 0, 0], [0, 0, 255, 0], [0, 0, 0, 255]]], dtype=np.uint8)
    np.testing.assert_allclose(op.gray(pure)[0], [77 / 256, 150 / 256, 29 / 256, 0.0], atol=1e-15)


def test_iir_step_response_closed_form():
    y = op.iir(None, np.zeros((2, 3)))
    for t in range(1, 30):
        y = op.iir(y, np.ones((2, 3)))
        np.testing.assert_allclose(y, 1.0 - (1.0 - op.ALPHA) ** t, rtol=0, atol=1e-15)
    c = op.iir(None, np.full((2, 2), 0.3))
    for _ in range(5):
        c = op.iir(c, np.full((2, 2), 0.3))
    np.testing.assert_allclose(c, 0.3, atol=1e-15)


def test_gauss3_impulse_constant_and_corner():
    x = np.zeros((7, 9))
    x[3, 4] = 1.0
    exp = np.zeros_like(x)
    exp[2:5, 3:6] = np.outer([1, 2, 1], [1, 2, 1]) / 16.0
    np.testing.assert_allclose(op.gauss3(x), exp, atol=1e-15)
    np.testing.assert_allclose(op.gauss3(np.full((4, 5), 0.7)), 0.7, atol=1e-15)
    c = np.zeros((5, 5))
    c[0, 0] = 1.0
    # corner: the clamped neighbours (-1, *) and (*, -1) read the corner itself
    assert op.gauss3(c)[0, 0] == pytest.approx((0.5 + 0.25) * (0.5 + 0.25))


@pytest.mark.parametrize("a,b", [(0.3, 0.0), (0.0, -0.2), (0.1, 0.05), (0.1, -0.05)])
def test_gradient_of_a_ramp(a, b):
    H, W = 9, 11
    yy, xx = np.mgrid[0:H, 0:W]
    G = a * xx + b * yy
    gx, gy, M = op.gradient(G)
    np.testing.assert_allclose(gx[1:-1, 1:-1], 8 * a, atol=1e-13)
    np.testing.assert_allclose(gy[1:-1, 1:-1], 8 * b, atol=1e-13)
    np.testing.assert_allclose(M[1:-1, 1:-1], 8 * (abs(a) + abs(b)), atol=1e-13)
    # one-sided at the clamped borders: x = 0 sees G(1) - G(0)
    np.testing.assert_allclose(gx[1:-1, 0], 4 * a, atol=1e-13)
    np.testing.assert_allclose(gy[0, 1:-1], 4 * b, atol=1e-13)


def test_threshold_and_regions_by_brute_force():
    rng = np.random.default_rng(5)
    H, W = 13, 10
    M = rng.random((H, W)) * 0.5
    mask, cnt, reg = op.threshold(M)
    assert cnt == int((M > op.TAU).sum())
    exp = np.zeros((16, 3), dtype=np.int64)
    for y in range(H):
        for x in range(W):
            if M[y, x] > op.TAU:
                r = (4 * y // H) * 4 + (4 * x // W)
                exp[r] += [1, x, y]
    np.testing.assert_array_equal(reg, exp)
    np.testing.assert_array_equal(mask, (M > op.TAU).astype(np.uint8))


def _tau_ramp(T, H, W, blue_step):
    """RGBA frames, constant in time and along y, whose gray value grows per column by
    (77 * 4 + 150 * 10 + 29 * blue_step) / (256 * 255). With blue_step = 8 that is 2040 /
    65280 = 1/32, and the Sobel magnitude of the ramp (smoothing leaves it unchanged) is
    8 / 32 = 0.25, the threshold itself, at every column two or more from the edges."""
    x = np.arange(W)
    fr = np.zeros((T, H, W, 4), dtype=np.uint8)
    fr[..., 0], fr[..., 1], fr[..., 2], fr[..., 3] = 4 * x, 10 * x, blue_step * x, 255
    return fr


def test_a_magnitude_exactly_at_the_threshold_is_not_marked():
    masks, counts, _, maps = op.chain_volume(_tau_ramp(3, 5, 26, 8), keep_maps=True)
    assert (maps["M"][:, :, 2:-2] == op.TAU).all()  # exact: every value is a small multiple of 2^-9
    assert counts.tolist() == [0, 0, 0] and not masks.any()
    masks, counts, _, _ = op.chain_volume(_tau_ramp(3, 5, 26, 9), keep_maps=True)  # 2069 / 65280 per column
    assert masks[:, :, 2:-2].all() and not masks[:, :, :2].any() and not masks[:, :, -2:].any()


def test_chain_volume_filters_over_time():
    # a step in time (black, then white frames): the chain's filtered map follows the IIR
    # filter's step response 1 - (1 - alpha)^t at every pixel
    fr = np.zeros((8, 4, 5, 4), dtype=np.uint8)
    fr[1:, ..., :3] = 255
    _, _, _, maps = op.chain_volume(fr, keep_maps=True)
    for t in range(8):
        np.testing.assert_allclose(maps["y"][t], 1.0 - (1.0 - op.ALPHA) ** t if t else 0.0, rtol=0, atol=1e-15)


def test_chain_volume_of_a_constant_video_is_empty():
    fr = np.full((3, 6, 8, 4), 120, dtype=np.uint8)
    masks, counts, regions, maps = op.chain_volume(fr, keep_maps=True)
    assert counts.tolist() == [0, 0, 0] and not masks.any() and not regions.any()
    np.testing.assert_allclose(maps["G"], op.gray(fr[0])[0, 0], atol=1e-15)


def _regions_of(points):
    """[T, 1, 3] region sums of one point per frame (count 1)."""
    return np.array([[[1, x, y]] for x, y in points], dtype=np.int64)


def test_kalman_model_is_constant_velocity_with_white_acceleration():
    F, Q, Hm, R = op.kalman_matrices()
    s = np.array([3.0, -2.0, 0.5, 1.5])
    np.testing.assert_array_equal(F @ s, [3.5, -0.5, 0.5, 1.5])  # one frame at constant velocity
    np.testing.assert_array_equal(Hm @ s, [3.0, -2.0])
    np.testing.assert_array_equal(R, op.KALMAN_R * np.eye(2))
    # the covariance that white acceleration of intensity q adds over one frame:
    # q * integral_0^1 Phi(u) G G' Phi(u)' du, Phi(u) = [[I, u I], [0, I]], G = [0; I]
    # (midpoint rule; its error on these quadratic entries is 1 / (12 m^2))
    m = 4000
    I2, Z2 = np.eye(2), np.zeros((2, 2))
    G = np.vstack([Z2, I2])
    acc = np.zeros((4, 4))
    for u in (np.arange(m) + 0.5) / m:
        Phi = np.block([[I2, u * I2], [Z2, I2]])
        acc += Phi @ G @ G.T @ Phi.T
    np.testing.assert_allclose(Q, op.KALMAN_Q * acc / m, rtol=0, atol=1e-7)


def test_kalman_converges_to_the_dare_steady_state_gain():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    F, Q, Hm, R = op.kalman_matrices()
    # a-priori steady-state covariance of the filter: the DARE of the dual system
    P = scipy_linalg.solve_discrete_are(F.T, Hm.T, Q, R)
    K_ss = P @ Hm.T @ np.linalg.inv(Hm @ P @ Hm.T + R)
    # the filter's gain after many updates, recovered from two runs that differ by a
    # unit measurement step at the last frame: the state moves by K times the step
    rng = np.random.default_rng(1)
    pts = [(50 + rng.normal(), 40 + rng.normal()) for _ in range(400)]
    base = _regions_of(pts)
    s0, _ = op.kalman(base)
    step = base.copy()
    step[-1, 0, 1] += 1  # x of the last measurement + 1
    s1, _ = op.kalman(step)
    np.testing.assert_allclose(s1[-1, 0] - s0[-1, 0], K_ss[:, 0], rtol=1e-9, atol=1e-12)


def test_kalman_is_two_per_axis_filters_from_the_first_frame():
    # the model decouples (F, Q, H, R and the start covariance act on x and y alike): each
    # axis is a 2-state filter [position, velocity] started at its first measurement with
    # variances (r, p0); run here as scalars from the stated model
    q, r, p0 = op.KALMAN_Q, op.KALMAN_R, op.KALMAN_P0
    F = np.array([[1.0, 1.0], [0.0, 1.0]])
    Q = q * np.array([[1 / 3, 1 / 2], [1 / 2, 1.0]])
    rng = np.random.default_rng(4)
    pts = [(30 + 1.5 * t + rng.normal(), 60 - 0.5 * t + rng.normal()) for t in range(40)]
    reg = np.array([[[1, round(x), round(y)]] for x, y in pts], dtype=np.int64)
    reg[17:21, 0] = 0  # a gap: prediction only
    states, status = op.kalman(reg)
    for axis in (0, 1):
        s, P = None, None
        for t in range(40):
            z = reg[t, 0, 1 + axis] if reg[t, 0, 0] else None
            if s is None:
                s, P = np.array([float(z), 0.0]), np.diag([r, p0])
            else:
                s, P = F @ s, F @ P @ F.T + Q
                if z is not None:
                    k = P[:, 0] / (P[0, 0] + r)
                    s = s + k * (z - s[0])
                    P = P - np.outer(k, P[0, :])
            np.testing.assert_allclose(states[t, 0, [axis, axis + 2]], s, rtol=1e-12, atol=1e-12)
    assert status[0, 0] == 1 and (status[17:21, 0] == 2).all()


def test_kalman_tracks_noise_free_constant_velocity_and_predicts_gaps():
    pts = [(10 + 2 * t, 400 - t) for t in range(200)]  # region sums are integer pixel coordinates
    s, st = op.kalman(_regions_of(pts))
    assert st[0, 0] == 1 and (st[1:, 0] == 1).all()
    np.testing.assert_allclose(s[-1, 0], [10 + 2 * 199, 400 - 199, 2.0, -1.0], atol=1e-6)
    reg = _regions_of(pts)
    reg[150:, 0] = 0  # no measurements: pure prediction with the learned velocity
    s2, st2 = op.kalman(reg)
    assert (st2[150:, 0] == 2).all()
    v = s2[149, 0, 2:]
    np.testing.assert_allclose(s2[199, 0, :2], s2[149, 0, :2] + 50 * v, atol=1e-9)
    empty = np.zeros((5, 2, 3), dtype=np.int64)
    s3, st3 = op.kalman(empty)
    assert not st3.any() and not s3.any()
