"""Seeded random kernel DAGs for the learned cost model (no arithmetic of the method).

A DAG is a list of stages in topological order; node 0 is the input frame and stage i
(1-based) writes node i. Each stage reads one or two earlier nodes:
  * "affine"   y = a x + b                     (point operation)
  * "abs"      y = |x|                         (point operation)
  * "product"  y = clamp(x1 x2, -16, 16)       (point operation, two inputs)
  * "stencil"  separable binomial smoothing of radius r in 0..3 (rectangular operation)
  * "max3"     3x3 maximum                      (rectangular operation)
The output of the DAG is its last node. Stage kinds, inputs and parameters are drawn
from splitmix64 counters of the seed, like the video generator.
"""
from __future__ import annotations

import dataclasses

from .video import uniforms

KINDS = ("affine", "abs", "product", "stencil", "max3")
KIND_CODE = {"affine": 1, "abs": 2, "product": 3, "stencil": 4, "max3": 5}


@dataclasses.dataclass(frozen=True)
class GStage:
    kind: str
    in1: int
    in2: int = -1  # product only
    radius: int = 0  # stencil: 0..3, max3: 1
    a: float = 1.0  # affine
    b: float = 0.0


def radius_of(s: GStage) -> int:
    return s.radius if s.kind == "stencil" else (1 if s.kind == "max3" else 0)


def random_dag(seed: int, n_min: int = 12, n_max: int = 24) -> list[GStage]:
    u = uniforms(seed, 7, 1 + 8 * n_max)
    n = n_min + int(u[0] * (n_max - n_min + 1))
    stages: list[GStage] = []
    for i in range(1, n + 1):
        v = u[1 + 8 * (i - 1): 1 + 8 * i]
        k = v[0]
        kind = "affine" if k < 0.2 else "abs" if k < 0.3 else "product" if k < 0.5 else "stencil" if k < 0.85 else "max3"
        # first input: the previous node most of the time, else any earlier node
        in1 = i - 1 if v[1] < 0.7 else int(v[2] * i)
        in2 = int(v[3] * i) if kind == "product" else -1
        radius = int(v[4] * 4) if kind == "stencil" else (1 if kind == "max3" else 0)
        a = -1.5 + 3.0 * v[5]
        b = -1.0 + 2.0 * v[6]
        stages.append(GStage(kind, in1, in2, radius, a, b))
    return stages


def to_array(stages: list[GStage]):
    """(kind, in1, in2, radius, a, b) rows for the C ABI / the oracle."""
    return [(KIND_CODE[s.kind], s.in1, s.in2, s.radius, s.a, s.b) for s in stages]


def deep_dag(seed: int, n_min: int = 14, n_max: int = 24) -> list[GStage]:
    """A DAG whose fused halos outgrow shared memory: stencils of radius 2-3 make up half
    the stages, and products take their second input from the first quarter of the DAG
    (long skip connections), so early point stages are read far downstream."""
    u = uniforms(seed, 11, 1 + 8 * n_max)
    n = n_min + int(u[0] * (n_max - n_min + 1))
    stages: list[GStage] = []
    for i in range(1, n + 1):
        v = u[1 + 8 * (i - 1): 1 + 8 * i]
        k = v[0]
        kind = "affine" if k < 0.2 else "abs" if k < 0.3 else "product" if k < 0.5 else "stencil" if k < 0.95 else "max3"
        in1 = i - 1 if v[1] < 0.8 else int(v[2] * i)
        in2 = int(v[3] * max(1, i // 4)) if kind == "product" else -1
        radius = 2 + int(v[4] * 2) if kind == "stencil" else (1 if kind == "max3" else 0)
        a = -1.5 + 3.0 * v[5]
        b = -1.0 + 2.0 * v[6]
        stages.append(GStage(kind, in1, in2, radius, a, b))
    return stages
