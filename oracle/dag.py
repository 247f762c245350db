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


# ------------------------------------------------------------------ FP32 error bound
# Running error analysis of the stage definitions above evaluated in FP32 (unit
# roundoff u = 2^-24), one bound per pixel and node, from the FP64 values: the tolerance
# the GPU's FP32 DAG executor is held to. Each rounding contributes at most u times the
# magnitude it rounds; an input error e passes through a stage as follows:
#   node 0    x = byte * fl(1/255): two roundings, 2u|x|
#   affine    fl(a) fl(x) + fl(b): |a| e + u(2|a x| + |b| + |y|)
#   abs       e (exact)
#   product   |x1| e2 + |x2| e1 + e1 e2 + u(|x1 x2| + ...) ; the clamp to [-16, 16] is
#             1-Lipschitz, so it adds nothing
#   stencil   the (positive, exact dyadic) weights applied to e, plus the dot-product
#             bound of recursive summation over both passes, 2(2r + 1) u sum w |x|
#             (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1)
#   max3      the 3x3 maximum of e (the maximum is 1-Lipschitz in the max norm)
# Terms of second order in u are absorbed by a factor (1 + 2^-10) on every bound.
U32 = 2.0 ** -24


def _stencil_abs(x: np.ndarray, radius: int) -> np.ndarray:
    """The stencil's weights applied to a non-negative map (clamped like the stage)."""
    w = binomial_weights(radius)
    out = np.zeros_like(x)
    for iy, dy in enumerate(range(-radius, radius + 1)):
        for ix, dx in enumerate(range(-radius, radius + 1)):
            out += w[iy] * w[ix] * _shift(x, dy, dx)
    return out


def fp32_error_bounds(rows, frame_u8: np.ndarray) -> list[np.ndarray]:
    """Per-pixel bound of |FP32 result - FP64 result| of every node of one frame."""
    nodes = run_frame(rows, frame_u8)
    grow = 1.0 + 2.0 ** -10
    err = [2.0 * U32 * np.abs(nodes[0]) * grow]
    for i, (kind, i1, i2, r, a, b) in enumerate(rows, start=1):
        x, e = np.abs(nodes[i1]), err[i1]
        y = np.abs(nodes[i])
        if kind == 1:
            bound = abs(a) * e + U32 * (2.0 * abs(a) * x + abs(b) + y)
        elif kind == 2:
            bound = e.copy()
        elif kind == 3:
            x2, e2 = np.abs(nodes[i2]), err[i2]
            exact = x * e2 + x2 * e + e * e2
            bound = exact + U32 * (x * x2 + exact)
        elif kind == 4:
            bound = _stencil_abs(e, r) + 2 * (2 * r + 1) * U32 * _stencil_abs(x + e, r)
        elif kind == 5:
            bound = np.full_like(e, 0.0)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    bound = np.maximum(bound, _shift(e, dy, dx))
        else:
            raise ValueError(kind)
        err.append(bound * grow)
    return err
