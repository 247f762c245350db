"""Reference of a spatio-temporal fusable set (Table I's spatio-temporal access type) and
of the box traffic that Eq. 3 - Eq. 6 reason about.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). The paper sizes boxes of x * x pixels
by t frames (Sec. VI-E) for fused groups with a temporal halo but gives no stage with a
finite temporal reach; the readings taken:

  K1 gray     Y = (77 R + 150 G + 29 B) / (256 * 255), as in the paper's own chain.
  Kt temporal z_t = sum_k C(n, k) Y_{t-n+k} / 2^n, k = 0..n: the binomial low-pass over the
              current and the n previous frames (one-sided temporal reach dt = n; frames
              before the first clamp to the first). n in {1, 2, 4}.
  K3 Gauss    3x3 binomial, clamp-to-edge (spatial reach 1).
  K4 grad     Sobel, L1 magnitude M = |gx| + |gy|, clamp-to-edge on the smoothed map
              (spatial reach 1).
  K5 thr      mask = M > tau, tau = 0.25; per frame the mask count.

The group's one-sided reaches are dx = 2 (two stencils of radius 1) and dt = n. Every map
is a fixed multiple of an integer: Y of g = 77 R + 150 G + 29 B (scale 65280), z of
sum_k C(n, k) g (scale 65280 * 2^n), the smoothed map of its 3x3 sum with weights
(1,2,1)x(1,2,1) (scale 65280 * 2^n * 16) and M of the unnormalised Sobel of that. So
the definition is carried out here on those integers, exactly, and M > tau is the
integer test M_int > tau * 65280 * 2^n * 16 = 261120 * 2^n. `chain_volume_real` is the
same chain in FP64 on the real values (through `pchain`'s pinned stage functions); the
two agree wherever M is not within rounding of tau.

Box traffic (Sec. VI-D / Eq. 3, with the reading of the halo used throughout: spatial
reach on both sides, temporal reach on the past side): a box of x * x outputs by t frames
reads (x + 2 dx)^2 (t + dt) input pixels and writes x^2 t.
"""
from __future__ import annotations

from math import comb

import numpy as np

from . import pchain

TAU = 0.25
DX = 2  # one-sided spatial reach of the group (Gaussian 1 + Sobel 1)
TAPS = (1, 2, 4)  # supported temporal reaches n


def threshold_int(n: int) -> int:
    """tau in the integer scale of M: 0.25 * 65280 * 2^n * 16."""
    return 261120 << n


def gray_int(rgba: np.ndarray) -> np.ndarray:
    """K1 numerators: [..., 4] u8 -> [...] int64, 77 R + 150 G + 29 B."""
    c = rgba.astype(np.int64)
    return 77 * c[..., 0] + 150 * c[..., 1] + 29 * c[..., 2]


def temporal_int(g: np.ndarray, t: int, n: int) -> np.ndarray:
    """Kt numerators of frame t from the [T, H, W] gray numerators: sum_k C(n, k)
    g[max(t - n + k, 0)]."""
    return sum(comb(n, k) * g[max(t - n + k, 0)] for k in range(n + 1))


def _shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    H, W = x.shape
    ys = np.clip(np.arange(H) + dy, 0, H - 1)
    xs = np.clip(np.arange(W) + dx, 0, W - 1)
    return x[np.ix_(ys, xs)]


def gauss_int(z: np.ndarray) -> np.ndarray:
    """K3 numerators: the 3x3 sum with weights (1,2,1) x (1,2,1), clamped."""
    w = {-1: 1, 0: 2, 1: 1}
    out = np.zeros_like(z)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += w[dy] * w[dx] * _shift(z, dy, dx)
    return out


def magnitude_int(G: np.ndarray) -> np.ndarray:
    """K4 numerators: |gx| + |gy| of the Sobel operator on G, clamped."""
    s = {-1: 1, 0: 2, 1: 1}
    gx = np.zeros_like(G)
    gy = np.zeros_like(G)
    for d in (-1, 0, 1):
        gx += s[d] * (_shift(G, d, 1) - _shift(G, d, -1))
        gy += s[d] * (_shift(G, 1, d) - _shift(G, -1, d))
    return np.abs(gx) + np.abs(gy)


def chain_volume(frames: np.ndarray, n: int, keep_m: bool = False):
    """K1, Kt, K3, K4, K5 over [T, H, W, 4] u8 frames. Returns masks [T, H, W] u8, counts
    [T] and, with keep_m, the integer magnitudes [T, H, W]."""
    assert n in TAPS
    T, H, W, _ = frames.shape
    g = gray_int(frames)
    masks = np.zeros((T, H, W), dtype=np.uint8)
    counts = np.zeros(T, dtype=np.int64)
    ms = np.zeros((T, H, W), dtype=np.int64) if keep_m else None
    thr = threshold_int(n)
    for t in range(T):
        M = magnitude_int(gauss_int(temporal_int(g, t, n)))
        masks[t] = M > thr
        counts[t] = int(masks[t].sum())
        if keep_m:
            ms[t] = M
    return masks, counts, ms


def chain_volume_real(frames: np.ndarray, n: int):
    """The same chain on real values in FP64 (pchain's gray, Gaussian and gradient).
    Returns masks [T, H, W] u8 and the magnitudes M [T, H, W]."""
    T, H, W, _ = frames.shape
    Y = np.stack([pchain.gray(frames[t]) for t in range(T)])
    masks = np.zeros((T, H, W), dtype=np.uint8)
    Ms = np.zeros((T, H, W))
    for t in range(T):
        z = sum(comb(n, k) * Y[max(t - n + k, 0)] for k in range(n + 1)) / 2.0 ** n
        M = pchain.gradient(pchain.gauss3(z))[2]
        Ms[t] = M
        masks[t] = M > TAU
    return masks, Ms


def box_model_bytes(W: int, H: int, T: int, x: int, t: int, n: int, bytes_in: int = 4, bytes_out: int = 1) -> float:
    """Sec. VI-D's fused transfer with B = W H T / (x^2 t) boxes, each reading
    (x + 2 dx)^2 (t + dt) input pixels and writing x^2 t."""
    B = W * H * T / (x * x * t)
    return B * ((x + 2 * DX) ** 2 * (t + n) * bytes_in + x * x * t * bytes_out)


def box_exact_reads(W: int, H: int, T: int, x: int, t: int, n: int) -> int:
    """Input pixels the boxes of the tiling read when halos are clipped at the volume's
    edges (frames before the first and pixels outside the frame are not read): the sum
    over boxes of their clipped input extents."""
    def spans(N, b, r_lo, r_hi):
        return [min(s + b + r_hi, N) - max(s - r_lo, 0) for s in range(0, N, b)]
    cx = sum(spans(W, x, DX, DX))
    cy = sum(spans(H, x, DX, DX))
    ct = sum(spans(T, t, n, 0))
    return cx * cy * ct


def data_utilisation(x: int, t: int, n: int) -> float:
    """Eq. 3 for this group: x^2 t / ((x + 2 dx)^2 (t + dt))."""
    return x * x * t / ((x + 2 * DX) ** 2 * (t + n))
