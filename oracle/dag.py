"""FP64 numpy reference of random kernel DAGs (the learned-cost-model workload).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain definitions, node by node, per
frame, with every stencil clamping its own input map (replicate), as the chain does:
  affine   y = a x + b
  abs      y = |x|
  product  y = min(max(x1 x2, -16), 16)
  stencil  y(p) = sum_{dy, dx} w_r(dy) w_r(dx) x(clamp(p + (dy, dx))),  w_r(k) = C(2r, r+k) / 4^r
  max3     y(p) = max_{|dy|, |dx| <= 1} x(clamp(p + (dy, dx)))
Node 0 is the frame as u8 / 255; the DAG's output is its last node. Sequential semantics
(Sec. III): every node is a whole map.
"""
from __future__ import annotations

from math import comb

import numpy as np


def binomial_weights(r: int) -> np.ndarray:
    return np.array([comb(2 * r, r + k) for k in range(-r, r + 1)], dtype=np.float64) / 4.0 ** r


def _shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """x(clamp(y + dy), clamp(x + dx)) for every pixel."""
    H, W = x.shape
    ys = np.clip(np.arange(H) + dy, 0, H - 1)
    xs = np.clip(np.arange(W) + dx, 0, W - 1)
    return x[np.ix_(ys, xs)]


def stage(kind: int, a_in: np.ndarray, b_in, radius: int, a: float, b: float) -> np.ndarray:
    if kind == 1:
        return a * a_in + b
    if kind == 2:
        return np.abs(a_in)
    if kind == 3:
        return np.clip(a_in * b_in, -16.0, 16.0)
    if kind == 4:
        w = binomial_weights(radius)
        out = np.zeros_like(a_in)
        for iy, dy in enumerate(range(-radius, radius + 1)):
            for ix, dx in enumerate(range(-radius, radius + 1)):
                out += w[iy] * w[ix] * _shift(a_in, dy, dx)
        return out
    if kind == 5:
        out = np.full_like(a_in, -np.inf)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out = np.maximum(out, _shift(a_in, dy, dx))
        return out
    raise ValueError(kind)


def run_frame(rows, frame_u8: np.ndarray) -> list[np.ndarray]:
    """All node maps of one frame [H, W]: nodes[0] = frame / 255, nodes[i] = stage i."""
    nodes = [frame_u8.astype(np.float64) / 255.0]
    for (kind, i1, i2, r, a, b) in rows:
        nodes.append(stage(kind, nodes[i1], nodes[i2] if i2 >= 0 else None, r, a, b))
    return nodes
