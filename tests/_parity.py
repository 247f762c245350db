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
