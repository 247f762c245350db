"""FP64 reference of the paper's own chain (Table II, Table IV): convert RGBA to gray,
IIR filter, Gaussian smoothing, gradient filter, threshold computation -- the fusable set
K1..K5 -- and, after the kernel-to-kernel dependency, a Kalman filter over feature
positions (K6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain definitions, frame by frame in
time order (the IIR filter is a recursion over frames), every stencil clamping its own
input map. The paper names the steps and their dependency types but not their formulas;
the readings taken:
  K1 gray   Y = (77 R + 150 G + 29 B) / (256 * 255): the BT.601 luma weights rounded to
            multiples of 1/256 (they sum to 1); alpha is ignored.
  K2 IIR    y_0 = Y_0, y_t = y_{t-1} + alpha (Y_t - y_{t-1}), alpha = 1/4: a first-order
            temporal low-pass, a point operation over frames (Table II "multi-frame").
  K3 Gauss  G(p) = sum_{dy,dx} w(dy) w(dx) y(clamp(p + (dy, dx))), w = [1, 2, 1] / 4 (3x3).
  K4 grad   gx = sum_dy s(dy) (G(y+dy, x+1) - G(y+dy, x-1)),
            gy = sum_dx s(dx) (G(y+1, x+dx) - G(y-1, x+dx)), s = [1, 2, 1], indices
            clamped on G; M = |gx| + |gy| (Sobel, L1 magnitude).
  K5 thr    mask = M > tau, tau = 0.25 (a point decision, Table IV "thread to thread");
            per frame the mask count and, per region of a 4 x 4 grid (region of (y, x) =
            (4y // H, 4x // W)), the count, sum of x and sum of y of the mask pixels.
  K6 Kalman one track per region: constant-velocity model, state (px, py, vx, vy),
            F = [[I, I], [0, I]], Q = q [[I/3, I/2], [I/2, I]] (white acceleration,
            dt = 1, q = 0.5), measurement z = the region's mask centroid (H = [I 0],
            R = r I, r = 4) in frames where the region has mask pixels. The track starts
            at the first such frame with s = (z, 0, 0), P = diag(r, r, p0, p0), p0 = 100;
            then every frame predicts, and updates when there is a measurement:
            S = H P H' + R, K = P H' S^-1, s += K (z - H s), P = (I - K H) P.
            Status per frame: 0 not started, 1 updated, 2 predicted only.
"""
from __future__ import annotations

import numpy as np

ALPHA = 0.25
TAU = 0.25
GRID = 4
KALMAN_Q = 0.5
KALMAN_R = 4.0
KALMAN_P0 = 100.0


def gray(rgba: np.ndarray) -> np.ndarray:
    """K1: [H, W, 4] u8 -> [H, W] gray in [0, 1]."""
    c = rgba.astype(np.float64)
    return (77.0 * c[..., 0] + 150.0 * c[..., 1] + 29.0 * c[..., 2]) / (256.0 * 255.0)


def iir(y_prev: np.ndarray | None, g: np.ndarray, alpha: float = ALPHA) -> np.ndarray:
    """K2: one step of the first-order temporal low-pass (y_prev None: the first frame)."""
    if y_prev is None:
        return g.copy()
    return y_prev + alpha * (g - y_prev)


def _shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """x(clamp(row + dy), clamp(col + dx)) for every pixel."""
    H, W = x.shape
    ys = np.clip(np.arange(H) + dy, 0, H - 1)
    xs = np.clip(np.arange(W) + dx, 0, W - 1)
    return x[np.ix_(ys, xs)]


def gauss3(y: np.ndarray) -> np.ndarray:
    """K3: 3x3 binomial smoothing, clamp-to-edge."""
    w = {-1: 0.25, 0: 0.5, 1: 0.25}
    out = np.zeros_like(y)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += w[dy] * w[dx] * _shift(y, dy, dx)
    return out


def gradient(G: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """K4: Sobel components on G (clamped) and the L1 magnitude."""
    s = {-1: 1.0, 0: 2.0, 1: 1.0}
    gx = np.zeros_like(G)
    gy = np.zeros_like(G)
    for d in (-1, 0, 1):
        gx += s[d] * (_shift(G, d, 1) - _shift(G, d, -1))
        gy += s[d] * (_shift(G, 1, d) - _shift(G, -1, d))
    return gx, gy, np.abs(gx) + np.abs(gy)


def threshold(M: np.ndarray, tau: float = TAU):
    """K5: mask, count, and per region of the GRID x GRID grid: (count, sum x, sum y)."""
    mask = M > tau
    H, W = M.shape
    regions = np.zeros((GRID * GRID, 3), dtype=np.int64)
    ys, xs = np.nonzero(mask)
    for y, x in zip(ys.tolist(), xs.tolist()):
        r = (GRID * y // H) * GRID + (GRID * x // W)
        regions[r, 0] += 1
        regions[r, 1] += x
        regions[r, 2] += y
    return mask.astype(np.uint8), int(mask.sum()), regions


def chain_volume(frames: np.ndarray, keep_maps: bool = False):
    """K1..K5 over [T, H, W, 4] u8 frames in time order. Returns masks [T, H, W] u8,
    counts [T], regions [T, GRID*GRID, 3] and, with keep_maps, the maps Y, y, G, M."""
    T, H, W, _ = frames.shape
    masks = np.zeros((T, H, W), dtype=np.uint8)
    counts = np.zeros(T, dtype=np.int64)
    regions = np.zeros((T, GRID * GRID, 3), dtype=np.int64)
    maps = {k: np.zeros((T, H, W)) for k in ("Y", "y", "G", "M")} if keep_maps else None
    y = None
    for t in range(T):
        Y = gray(frames[t])
        y = iir(y, Y)
        G = gauss3(y)
        M = gradient(G)[2]
        masks[t], counts[t], regions[t] = threshold(M)
        if keep_maps:
            maps["Y"][t], maps["y"][t], maps["G"][t], maps["M"][t] = Y, y, G, M
    return masks, counts, regions, maps


def kalman_matrices(q: float = KALMAN_Q, r: float = KALMAN_R):
    I2 = np.eye(2)
    F = np.block([[I2, I2], [np.zeros((2, 2)), I2]])
    Q = q * np.block([[I2 / 3.0, I2 / 2.0], [I2 / 2.0, I2]])
    Hm = np.hstack([I2, np.zeros((2, 2))])
    R = r * I2
    return F, Q, Hm, R


def kalman(regions: np.ndarray, q: float = KALMAN_Q, r: float = KALMAN_R, p0: float = KALMAN_P0):
    """K6 over [T, N, 3] region sums (count, sum x, sum y): per track and frame the state
    [T, N, 4] and status [T, N] (0 not started, 1 updated, 2 predicted)."""
    T, N, _ = regions.shape
    F, Q, Hm, R = kalman_matrices(q, r)
    states = np.zeros((T, N, 4))
    status = np.zeros((T, N), dtype=np.int64)
    for n in range(N):
        s = None
        P = None
        for t in range(T):
            cnt, sx, sy = regions[t, n]
            z = np.array([sx / cnt, sy / cnt]) if cnt > 0 else None
            if s is None:
                if z is None:
                    continue
                s = np.array([z[0], z[1], 0.0, 0.0])
                P = np.diag([r, r, p0, p0])
                states[t, n], status[t, n] = s, 1
                continue
            s = F @ s
            P = F @ P @ F.T + Q
            if z is not None:
                S = Hm @ P @ Hm.T + R
                K = P @ Hm.T @ np.linalg.inv(S)
                s = s + K @ (z - Hm @ s)
                P = (np.eye(4) - K @ Hm) @ P
                status[t, n] = 1
            else:
                status[t, n] = 2
            states[t, n] = s
    return states, status
