"""The autotuning cache (CPU only): a miss measures and stores, a hit applies the stored
chunk height to the context without measuring, every field of the key separates
entries, and an unreadable file starts an empty cache. The measurement is replaced by a
stand-in with the library tuner's arguments and result."""
import json

import numpy as np
import pytest

from paper_1509_04394_gb300 import build as kbuild
from paper_1509_04394_gb300 import kfuse as K
from paper_1509_04394_gb300 import tuning


@pytest.fixture()
def ctx():
    kbuild.build()
    c = K.kf_create(-1)
    K.kf_add_harris_chain(c)
    yield c
    K.kf_destroy(c)


def _tuner(rows, calls):
    def tune(ctx, frames, W, mask, counts, candidates, reps, stream):
        calls.append((frames.shape, W, tuple(candidates), reps))
        K.kf_set_chunk_rows(ctx, rows)  # as the library's tuner leaves the context
        return rows, 1.25
    return tune


def _no_tune(*a):
    raise AssertionError("measured on a cache hit")


def test_miss_measures_and_stores_then_hit_applies(ctx, tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    frames = np.zeros((5, 48, 64), dtype=np.uint8)
    calls = []
    rows, cached = tuning.chunk_rows(ctx, frames, 60, None, None, tuning.TuneCache(path), "GB300", K.KF_PREC_F32,
                                     tune=_tuner(400, calls))
    assert (rows, cached) == (400, False) and calls == [((5, 48, 64), 60, (100, 200, 400, 800), 3)]
    stored = json.load(open(path))
    assert list(stored.values()) == [{"rows": 400, "ms": 1.25, "frames": 5}]
    # a later run: the stored height is applied without measuring
    K.kf_set_chunk_rows(ctx, 100)
    rows, cached = tuning.chunk_rows(ctx, frames, 60, None, None, tuning.TuneCache(path), "GB300", K.KF_PREC_F32,
                                     tune=_no_tune)
    assert (rows, cached) == (400, True)
    ref = K.kf_create(-1)
    K.kf_add_harris_chain(ref)
    K.kf_set_chunk_rows(ref, 400)
    # the executor's tile height enters the traffic model: equal once the context holds 400 rows
    assert K.kf_group_traffic(ctx, 0, 7, 60, 48, 5) == K.kf_group_traffic(ref, 0, 7, 60, 48, 5)
    K.kf_destroy(ref)


@pytest.mark.parametrize("change", ["W", "H", "device", "precision", "candidates"])
def test_every_key_field_separates_entries(ctx, tmp_path, change):
    path = str(tmp_path / "tune.json")
    base = dict(W=60, H=48, device="GB300", precision=K.KF_PREC_F32, candidates=(100, 200, 400, 800))
    calls = []

    def run(p):
        frames = np.zeros((3, p["H"], 64), dtype=np.uint8)
        return tuning.chunk_rows(ctx, frames, p["W"], None, None, tuning.TuneCache(path), p["device"], p["precision"],
                                 candidates=p["candidates"], tune=_tuner(200, calls))
    run(base)
    other = dict(base)
    other[change] = {"W": 61, "H": 50, "device": "other", "precision": K.KF_PREC_F16, "candidates": (100, 200)}[change]
    assert run(other)[1] is False and len(calls) == 2
    assert run(base)[1] is True and run(other)[1] is True and len(calls) == 2


def test_unreadable_file_starts_empty(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    c = tuning.TuneCache(str(path))
    assert c.entries == {}
    c.put("k", {"rows": 1})
    assert json.loads(path.read_text()) == {"k": {"rows": 1}}
    path.write_text("[1, 2]")  # valid JSON, not an object
    assert tuning.TuneCache(str(path)).entries == {}


def test_batch_rows_measures_each_shape_once(ctx, tmp_path):
    """A batch's tile heights: one measurement per distinct frame shape (on a prefix of its
    first video), shared by every video of that shape and reused from the cache later."""
    path = str(tmp_path / "tune.json")
    calls = []

    def tune(c, frames, W, mask, counts, cands, reps, stream):
        calls.append((int(W), frames.shape[1], frames.shape[0]))
        return {60: 160, 90: 267}[int(W)], 1.0
    vids = [(np.zeros((100, 48, 64), np.uint8), 60), (np.zeros((7, 40, 96), np.uint8), 90),
            (np.zeros((30, 48, 64), np.uint8), 60)]
    rows = tuning.batch_rows(ctx, vids, tuning.TuneCache(path), "GB300", K.KF_PREC_F32, sample_frames=64, tune=tune)
    assert rows == [160, 267, 160]
    assert calls == [(60, 48, 64), (90, 40, 7)]
    rows2 = tuning.batch_rows(ctx, vids, tuning.TuneCache(path), "GB300", K.KF_PREC_F32, tune=_no_tune)
    assert rows2 == rows and len(calls) == 2


def test_batch_warps_keeps_the_fastest_and_caches_it(tmp_path):
    """The persistent launch's warps per SM: every candidate timed once, the fastest kept
    (ties to the smaller setting), stored under the batch's shape mix and tile heights."""
    path = str(tmp_path / "tune.json")
    vids = [(np.zeros((10, 48, 64), np.uint8), 60), (np.zeros((10, 48, 64), np.uint8), 60),
            (np.zeros((4, 40, 96), np.uint8), 90)]
    seen = []

    def time_batch(w):
        seen.append(w)
        return {0: 5.0, 10: 4.0, 8: 4.0}[w]
    best, cached = tuning.batch_warps(None, vids, None, None, None, None, [200, 200, 100], tuning.TuneCache(path), "GB300",
                                      candidates=(0, 10, 8), time_batch=time_batch)
    assert (best, cached) == (8, False) and seen == [0, 10, 8]
    best, cached = tuning.batch_warps(None, vids, None, None, None, None, [200, 200, 100], tuning.TuneCache(path), "GB300",
                                      candidates=(0, 10, 8), time_batch=lambda w: pytest.fail("measured again"))
    assert (best, cached) == (8, True)
    # another tile-height choice is another entry
    best, cached = tuning.batch_warps(None, vids, None, None, None, None, [100, 100, 100], tuning.TuneCache(path),
                                      "GB300", candidates=(0, 10, 8), time_batch=lambda w: {0: 1.0, 10: 2.0, 8: 3.0}[w])
    assert (best, cached) == (0, False)


def test_batch_launch_picks_the_fastest_assignment_and_caches_it(tmp_path):
    """Tile heights and warps per SM measured on the batch itself: every pair of a
    candidate assignment and a warps setting timed once, the fastest kept and stored."""
    path = str(tmp_path / "tune.json")
    vids = [(np.zeros((10, 48, 64), np.uint8), 60), (np.zeros((4, 40, 96), np.uint8), 90)]
    choices = [[100, 160], [200, 200], [267, 267]]
    seen = []

    def time_batch(rows, w):
        seen.append((tuple(rows), w))
        return {(200, 200): 3.0, (100, 160): 4.0, (267, 267): 3.5}[tuple(rows)] + (0.5 if w else 0.0)
    rows, w, cached = tuning.batch_launch(None, vids, None, None, None, None, choices, tuning.TuneCache(path), "GB300",
                                          warp_candidates=(0, 10), time_batch=time_batch)
    assert (rows, w, cached) == ([200, 200], 0, False) and len(seen) == 6
    rows, w, cached = tuning.batch_launch(None, vids, None, None, None, None, choices, tuning.TuneCache(path), "GB300",
                                          warp_candidates=(0, 10), time_batch=lambda r, w: pytest.fail("again"))
    assert (rows, w, cached) == ([200, 200], 0, True)
