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
