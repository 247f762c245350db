"""Autotuning results kept across runs: a JSON file of measured choices, each keyed by
what the measurement depends on (the tuned call, the frame shape, the precision, the
device's name and the candidates tried). A hit applies the stored choice to the context
without measuring; a miss measures through the library and stores the result.

Host logic only; the measurement itself is the library's (kf_tune_chunk_rows times
every candidate with CUDA events on the device).
"""
from __future__ import annotations

import json
import os
import tempfile


class TuneCache:
    """A JSON object of key -> result, rewritten atomically on every store. A missing or
    unreadable file starts an empty cache."""

    def __init__(self, path: str):
        self.path = path
        self.entries: dict = {}
        try:
            with open(path) as fh:
                data = json.load(fh)
            if isinstance(data, dict):
                self.entries = data
        except (OSError, ValueError):
            pass

    @staticmethod
    def key(call: str, **fields) -> str:
        return call + "|" + "|".join(f"{k}={fields[k]}" for k in sorted(fields))

    def get(self, key: str):
        return self.entries.get(key)

    def put(self, key: str, value) -> None:
        self.entries[key] = value
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune-", suffix=".json")
        try:
            with os.fdopen(fd, "w") as fh:
                json.dump(self.entries, fh, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def chunk_rows(ctx, frames, W: int, mask, counts, cache: TuneCache, device_name: str, precision: int,
               candidates=(100, 200, 400, 800), reps: int = 3, stream=None, tune=None) -> tuple[int, bool]:
    """The executor's chunk height (rows per warp job) for this frame shape on this device:
    from the cache, else measured by kf_tune_chunk_rows on `frames` and stored. Either way
    the context is left set to it. Returns (rows, whether it came from the cache).
    `tune` replaces the measurement (same arguments and result as K.kf_tune_chunk_rows)."""
    from . import kfuse as K
    T, H, _ = frames.shape
    key = TuneCache.key("chunk_rows", W=int(W), H=int(H), precision=int(precision), device=str(device_name),
                        candidates=",".join(str(int(c)) for c in candidates))
    hit = cache.get(key)
    if hit is not None:
        rows = int(hit["rows"])
        K.kf_set_chunk_rows(ctx, rows)
        return rows, True
    rows, ms = (tune or K.kf_tune_chunk_rows)(ctx, frames, W, mask, counts, list(candidates), reps, stream)
    cache.put(key, {"rows": int(rows), "ms": float(ms), "frames": int(T)})
    return int(rows), False


def batch_rows(ctx, videos, cache: TuneCache, device_name: str, precision: int, candidates=(100, 160, 200, 267, 400),
               sample_frames: int = 64, reps: int = 3, stream=None, tune=None) -> list[int]:
    """The tile height of every video of a batch: one chunk_rows() measurement per distinct
    frame shape, on the first `sample_frames` frames of the first video of that shape
    (the per-frame cost of a shape does not depend on the video's length), reused from the
    cache when present. videos: list of (frames [T, H, P] CUDA tensor, W). Returns one
    height per video, in order. The context is left at the last measured height."""
    rows_of: dict[tuple[int, int], int] = {}
    out = []
    for frames, W in videos:
        shape = (int(W), int(frames.shape[1]))
        if shape not in rows_of:
            f = frames[:sample_frames]
            mask = counts = None
            if tune is None:  # the library's measurement writes a mask and counts
                import torch
                mask = torch.zeros_like(f)
                counts = torch.zeros(f.shape[0], dtype=torch.int32, device=f.device)
            rows_of[shape], _ = chunk_rows(ctx, f, W, mask, counts, cache, device_name, precision, candidates, reps,
                                           stream, tune)
        out.append(rows_of[shape])
    return out


def batch_launch(ctx, videos, masks, counts, workspace, tracks, row_choices, cache: TuneCache, device_name: str,
                 warp_candidates=(0, 10), reps: int = 3, stream=None, time_batch=None) -> tuple[list[int], int, bool]:
    """The tile heights and resident warps per SM of a batch, measured on the batch itself:
    every (tile-height assignment, warps per SM) pair is built as a batch, replayed once
    untimed and `reps` times under CUDA events, and destroyed; the fastest pair is kept in
    the cache under the batch's shape mix. row_choices: candidate assignments, each one
    height per video (e.g. the per-shape standalone choices of batch_rows, and uniform
    heights). Returns (heights, warps per SM, whether it came from the cache).
    `time_batch(rows, warps)` replaces the measurement (returns ms per replay)."""
    from collections import Counter
    mix = Counter((int(W), int(f.shape[1]), int(f.shape[0])) for f, W in videos)
    key = TuneCache.key("batch_launch", mix=";".join(f"{n}x{w}x{h}x{t}" for (w, h, t), n in sorted(mix.items())),
                        rows="/".join(",".join(str(int(r)) for r in rc) for rc in row_choices),
                        track=int(tracks is not None), device=str(device_name),
                        warps=",".join(str(int(c)) for c in warp_candidates))
    hit = cache.get(key)
    if hit is not None:
        return [int(r) for r in hit["rows"]], int(hit["warps_per_sm"]), True

    def measure(rows, warps: int) -> float:
        import torch
        from . import kfuse as K
        b = K.kf_batch_create(ctx, [f for f, _ in videos], [w for _, w in videos], masks, counts, workspace, tracks,
                              chunk_rows=rows, warps_per_sm=warps)
        try:
            K.kf_batch_run(b, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s = stream or torch.cuda.current_stream()
            e0.record(s)
            for _ in range(reps):
                K.kf_batch_run(b, stream)
            e1.record(s)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps
        finally:
            K.kf_batch_destroy(b)
    timings = []
    for i, rc in enumerate(row_choices):
        for w in warp_candidates:
            timings.append((float((time_batch or measure)(list(rc), int(w))), i, int(w)))
    ms, i, w = min(timings)
    cache.put(key, {"rows": [int(r) for r in row_choices[i]], "warps_per_sm": w, "ms": ms,
                    "all_ms": [[t, j, x] for t, j, x in timings]})
    return [int(r) for r in row_choices[i]], w, False


def batch_warps(ctx, videos, masks, counts, workspace, tracks, rows, cache: TuneCache, device_name: str,
                candidates=(0, 10, 8), reps: int = 3, stream=None, time_batch=None) -> tuple[int, bool]:
    """Resident warps per SM of a batch's persistent launch (0 = as many as fit): each
    candidate's batch is created, replayed once untimed and `reps` times under CUDA events,
    and destroyed; the fastest is kept in the cache under the batch's shape mix. Returns
    (warps per SM, whether it came from the cache). `time_batch(warps)` replaces the
    measurement (returns ms per replay)."""
    from collections import Counter
    mix = Counter((int(W), int(f.shape[1]), int(f.shape[0])) for f, W in videos)
    key = TuneCache.key("batch_warps", mix=";".join(f"{n}x{w}x{h}x{t}" for (w, h, t), n in sorted(mix.items())),
                        rows=",".join(str(int(r)) for r in rows), track=int(tracks is not None),
                        device=str(device_name), candidates=",".join(str(int(c)) for c in candidates))
    hit = cache.get(key)
    if hit is not None:
        return int(hit["warps_per_sm"]), True

    def measure(warps: int) -> float:
        import torch
        from . import kfuse as K
        b = K.kf_batch_create(ctx, [f for f, _ in videos], [w for _, w in videos], masks, counts, workspace, tracks,
                              chunk_rows=rows, warps_per_sm=warps)
        try:
            K.kf_batch_run(b, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s = stream or torch.cuda.current_stream()
            e0.record(s)
            for _ in range(reps):
                K.kf_batch_run(b, stream)
            e1.record(s)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps
        finally:
            K.kf_batch_destroy(b)
    timings = {int(c): float((time_batch or measure)(int(c))) for c in candidates}
    best = min(timings, key=lambda c: (timings[c], c))
    cache.put(key, {"warps_per_sm": best, "ms": timings[best], "all_ms": {str(k): v for k, v in timings.items()}})
    return best, False
