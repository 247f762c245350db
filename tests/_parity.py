"""Shared helpers of the GPU parity tests: tolerance rules and device buffers."""
from __future__ import annotations

import numpy as np

THRESHOLD = 1e-5
TOL_F32 = 1e-5  # normwise relative error of float maps, FP32 path
TOL_F16 = 2e-3  # FP16 maps


def normwise(gpu: np.ndarray, ref: np.ndarray) -> float:
    """max |gpu - ref| / max |ref|; an all-zero reference uses the absolute error."""
    d = float(np.max(np.abs(gpu.astype(np.float64) - ref))) if ref.size else 0.0
    n = float(np.max(np.abs(ref))) if ref.size else 0.0
    return d / n if n > 0 else d


def exempt_pixels(r: np.ndarray, tol: float, thr: float = THRESHOLD) -> np.ndarray:
    """Pixels whose corner decision float rounding may flip: the oracle response lies
    within tau = tol * max|R| of the threshold, or of one of its in-frame 8-neighbours."""
    H, W = r.shape
    tau = tol * float(np.max(np.abs(r))) if r.size else 0.0
    ex = np.abs(r - thr) <= tau
    pad = np.pad(r, 1, mode="constant", constant_values=np.nan)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            q = pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            with np.errstate(invalid="ignore"):
                ex |= np.abs(r - q) <= tau
    return ex


def check_mask(mask_gpu: np.ndarray, count_gpu: int, mask_ref: np.ndarray, count_ref: int, r_ref: np.ndarray,
               tol: float) -> int:
    """Masks agree except at exempt pixels; counts within the number of exempt mismatches.
    Returns the number of mismatching pixels."""
    mg = mask_gpu.astype(bool)
    mr = mask_ref.astype(bool)
    assert count_gpu == int(mg.sum()), "count differs from the mask's popcount"
    bad = mg != mr
    if bad.any():
        ex = exempt_pixels(r_ref, tol)
        assert not (bad & ~ex).any(), f"{int((bad & ~ex).sum())} non-exempt mask mismatches"
    assert abs(count_gpu - count_ref) <= int(bad.sum())
    return int(bad.sum())


def pitch16(W: int) -> int:
    return (W + 15) // 16 * 16


def pitch4(W: int) -> int:
    return (W + 3) // 4 * 4


def kalman_fp32_bound(states_o: np.ndarray, regions: np.ndarray, W: int, q: float = 0.5, r: float = 4.0,
                      p0: float = 100.0) -> tuple[float, float]:
    """Error budget of the FP32 constant-velocity Kalman filter against the FP64 one
    (positions in px, velocities in px/frame), derived from the filter itself.

    Each step adds rounding errors: the measured centroid z = sum / count (3 roundings of
    |z| <= W), the state update (about 4 roundings of |p| <= W for the position and 3 of
    the largest |v| for the velocity) and the gain computed from an FP32 covariance
    (about 10 roundings of K, times the largest innovation |z - p_predicted|). The error
    then evolves as e_t = A e_{t-1} + d_t with A = (I - K H) F, which is stable (its
    spectral radius at the steady-state gain is 0.66 for q = 0.5, r = 4), so it stays
    below sum_k |A^k| d. The steady-state sum is taken, times a margin of 4 for the
    transient gains and second-order terms."""
    u = 2.0 ** -24
    F = np.array([[1.0, 1.0], [0.0, 1.0]])
    Q = q * np.array([[1 / 3, 1 / 2], [1 / 2, 1.0]])
    Hm = np.array([[1.0, 0.0]])
    P = np.diag([r, p0])
    for _ in range(500):  # Riccati iteration to the steady state
        P = F @ P @ F.T + Q
        K = P @ Hm.T / float((Hm @ P @ Hm.T)[0, 0] + r)
        P = (np.eye(2) - K @ Hm) @ P
    A = (np.eye(2) - K @ Hm) @ F
    S, M = np.zeros((2, 2)), np.eye(2)
    for _ in range(2000):
        S += np.abs(M)
        M = A @ M
    cnt = regions[..., 0]
    with np.errstate(invalid="ignore", divide="ignore"):
        z = np.where(cnt[..., None] > 0, regions[..., 1:] / np.maximum(cnt[..., None], 1), np.nan)
    pred = states_o[:-1, :, :2] + states_o[:-1, :, 2:]
    innov = np.nanmax(np.abs(z[1:] - pred)) if np.isfinite(z[1:] - pred).any() else 0.0
    vmax = float(np.max(np.abs(states_o[..., 2:])))
    k = np.abs(K.ravel())
    d = k * (3 * u * W + 10 * u * innov) + np.array([4 * u * W, 3 * u * vmax])
    b = 4.0 * (S @ d)
    return float(b[0]), float(b[1])
