"""Brute-force partitioner and the paper's traffic model, restated plainly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. VI: a chain of n kernels can be cut into contiguous groups in 2^(n-1) ways
(three kernels give the four partitions listed there), there are n(n+1)/2 candidate
groups (Fig. 5), and the chosen partition minimises the summed cost of its groups
subject to every algorithm being covered exactly once. This module enumerates every
partition and evaluates each one; no dynamic programming, no pruning.

Cost of a group is the traffic model of Sec. VI-D, under these readings of the text:
  * radii are one-sided; a stage that reads (2*rx+1) x (2*ry+1) x rt pixels (Alg. 2)
    needs a spatial halo on both sides and a temporal halo on the past side only;
  * a fused group's halo is the SUM of its stages' radii (chained stencils grow their
    halos), not the maximum Alg. 2 takes;
  * traffic is counted in bytes: each map has channels x element size per pixel;
  * one box of x*y*t outputs reads (x+2Rx)(y+2Ry)(t+Rt) input pixels and writes x*y*t
    output pixels; there are B = N*M*T / (x*y*t) boxes (Sec. V, Fig. 3).
With 1-byte point stages this gives Transfer_serial = 2 n B x y t (Sec. VI-D).
"""
from __future__ import annotations

import dataclasses
import itertools


@dataclasses.dataclass(frozen=True)
class Stage:
    name: str
    rx: int  # one-sided radius along columns
    ry: int  # one-sided radius along rows
    rt: int  # frames in the past
    in_bytes: float  # bytes per pixel of all input maps
    out_bytes: float  # bytes per pixel of all output maps


def harris_chain(elem_bytes: int = 4) -> list[Stage]:
    """The 8-stage Harris chain with float maps of `elem_bytes` bytes per channel."""
    e = elem_bytes
    return [
        Stage("convert", 0, 0, 0, 1, 1 * e),
        Stage("gauss_h", 2, 0, 0, 1 * e, 1 * e),
        Stage("gauss_v", 0, 2, 0, 1 * e, 1 * e),
        Stage("sobel", 1, 1, 0, 1 * e, 2 * e),
        Stage("products", 0, 0, 0, 2 * e, 3 * e),
        Stage("box5", 2, 2, 0, 3 * e, 3 * e),
        Stage("harris", 0, 0, 0, 3 * e, 1 * e),
        Stage("nms", 1, 1, 0, 1 * e, 1),
    ]


def candidate_groups(n: int) -> list[tuple[int, int]]:
    """All contiguous groups (a, b), 0 <= a <= b < n."""
    return [(a, b) for a in range(n) for b in range(a, n)]


def groups_of(n: int, cuts: int) -> list[tuple[int, int]]:
    """Groups of a partition; bit i of `cuts` = a cut between stage i and i+1."""
    out, a = [], 0
    for i in range(n - 1):
        if cuts >> i & 1:
            out.append((a, i))
            a = i + 1
    out.append((a, n - 1))
    return out


def all_partitions(n: int) -> list[list[tuple[int, int]]]:
    """Every contiguous partition, by listing every subset of the n-1 cut points."""
    parts = []
    for chosen in itertools.product((0, 1), repeat=n - 1):
        cuts = sum(bit << i for i, bit in enumerate(chosen))
        parts.append(groups_of(n, cuts))
    return parts


def halo(stages: list[Stage], a: int, b: int) -> tuple[int, int, int]:
    return (sum(s.rx for s in stages[a:b + 1]), sum(s.ry for s in stages[a:b + 1]),
            sum(s.rt for s in stages[a:b + 1]))


def group_traffic(stages, a, b, N, M, T, box) -> float:
    """Bytes one fused group moves between global memory and the chip."""
    x, y, t = box
    Rx, Ry, Rt = halo(stages, a, b)
    boxes = N * M * T / (x * y * t)
    per_box = (x + 2 * Rx) * (y + 2 * Ry) * (t + Rt) * stages[a].in_bytes \
        + x * y * t * stages[b].out_bytes
    return boxes * per_box


def group_onchip(stages, a, b, box) -> float:
    """On-chip bytes a fused group holds per box: each stage keeps its (2ry+1)-row
    window of its input maps over the full halo-extended box width, for t frames."""
    x, _, t = box
    Rx, _, Rt = halo(stages, a, b)
    return (x + 2 * Rx) * (t + Rt) * sum((2 * s.ry + 1) * s.in_bytes for s in stages[a:b + 1])


def data_utilisation(box, radii) -> float:
    """Eq. 3 with two-sided spatial and one-sided temporal halo."""
    x, y, t = box
    rx, ry, rt = radii
    return x * y * t / ((x + 2 * rx) * (y + 2 * ry) * (t + rt))


def partition_cost(stages, groups, N, M, T, box) -> float:
    return sum(group_traffic(stages, a, b, N, M, T, box) for a, b in groups)


def feasible(stages, groups, box, onchip_limit) -> bool:
    return all(group_onchip(stages, a, b, box) <= onchip_limit for a, b in groups)


def brute_force_best(stages, N, M, T, box, onchip_limit=float("inf")):
    """(groups, cost) of the cheapest feasible partition; ties go to the first one met in
    enumeration order (fewest cuts among the lowest cut indices first is NOT assumed)."""
    best = None
    for g in all_partitions(len(stages)):
        if not feasible(stages, g, box, onchip_limit):
            continue
        c = partition_cost(stages, g, N, M, T, box)
        if best is None or c < best[1]:
            best = (g, c)
    return best


def eq6_box(beta: float, dx: float, dt: float) -> tuple[float, float]:
    """Closed form of Eq. 6: x = y = (2 beta dx / dt)^(1/3), t = 2^(-2/3) beta^(1/3) (dt/dx)^(2/3)."""
    x = (2.0 * beta * dx / dt) ** (1.0 / 3.0)
    t = 2.0 ** (-2.0 / 3.0) * beta ** (1.0 / 3.0) * (dt / dx) ** (2.0 / 3.0)
    return x, t
