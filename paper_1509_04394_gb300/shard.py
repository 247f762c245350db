"""Frame-range sharding of one video over processes (one per GPU), merged on the host.

Every result of the hot path for frame t depends on frame t alone, except the tracking
step (the Lucas-Kanade step of the temporal set, after the kernel-to-kernel cut of
Sec. V-A c), which also reads frame t - 1: the path's temporal reach is one frame. A
process that owns the frames [t0, t1) therefore runs the path over [s0, t1), s0 =
max(t0 - 1, 0), and keeps the results of [t0, t1); the leading frame is read only for its
successor's tracking (its own results, computed without a predecessor, are dropped).
The kept results of all processes, in rank order, are the whole video's, element for
element. No data crosses between processes while the path runs; the results are
gathered once at the end.

Host logic only: the device work of a shard is an ordinary kf_track call on the view
frames[s0:t1].
"""
from __future__ import annotations

import numpy as np

HALO_FRAMES = 1  # frames before a shard that its first owned frame's tracking reads


def frame_ranges(T: int, world: int) -> list[tuple[int, int]]:
    """Contiguous owned ranges [t0, t1) covering [0, T) in rank order; the first T % world
    ranks own one frame more than the rest (ranks past T own nothing)."""
    if T < 0 or world < 1:
        raise ValueError("need T >= 0 and world >= 1")
    base, extra = divmod(T, world)
    out, t0 = [], 0
    for r in range(world):
        t1 = t0 + base + (1 if r < extra else 0)
        out.append((t0, t1))
        t0 = t1
    return out


def span(T: int, world: int, rank: int) -> tuple[int, int, int]:
    """(s0, t0, t1): rank `rank` owns [t0, t1) and runs the path over [s0, t1). An empty
    range runs nothing (s0 = t0 = t1)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    t0, t1 = frame_ranges(T, world)[rank]
    s0 = t0 if t0 == t1 else max(t0 - HALO_FRAMES, 0)
    return s0, t0, t1


def keep(results: dict, s0: int, t0: int) -> dict:
    """The owned rows of a shard's per-frame results (arrays indexed by frame first, over
    the run range [s0, t1))."""
    d = t0 - s0
    return {k: np.asarray(a)[d:] for k, a in results.items()}


def merge(parts: list[dict]) -> dict:
    """Concatenate the kept results of the shards, in rank order, along the frame axis.
    Shards that own no frame may be empty dicts."""
    parts = [p for p in parts if p]
    if not parts:
        return {}
    keys = parts[0].keys()
    if any(p.keys() != keys for p in parts):
        raise ValueError("shards hold different result fields")
    return {k: np.concatenate([p[k] for p in parts], axis=0) for k in keys}


def gather_merge(kept: dict, rank: int, world: int, dst: int = 0):
    """Gather every rank's kept results to rank `dst` over the default process group and
    merge them there (returns the merged dict on `dst`, None elsewhere). One collective,
    after the path has run."""
    if world == 1:
        return merge([kept])
    import torch.distributed as dist
    box = [None] * world if rank == dst else None
    dist.gather_object(kept, box, dst=dst)
    return merge(box) if rank == dst else None
