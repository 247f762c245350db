"""Frame-range sharding of one video over processes, merged on the host (CPU only): the
ranges cover the video in balanced contiguous pieces, a path with a one-frame temporal
reach merges to the whole-video result only with the one-frame halo, two gloo ranks
running the oracle on their shards merge to the oracle's whole-video tracking, and the
benchmark's ranks render their ranges of one video."""
import os
import socket

import numpy as np
import pytest

from paper_1509_04394_gb300 import shard

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("T", [0, 1, 2, 7, 1000, 1001])
@pytest.mark.parametrize("world", [1, 2, 3, 8, 13])
def test_ranges_cover_the_video_in_balanced_pieces(T, world):
    rs = shard.frame_ranges(T, world)
    assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == T
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    sizes = [t1 - t0 for t0, t1 in rs]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    for r, (t0, t1) in enumerate(rs):
        s0, u0, u1 = shard.span(T, world, r)
        assert (u0, u1) == (t0, t1)
        assert s0 == (t0 if t0 == t1 or t0 == 0 else t0 - 1)


def _one_frame_reach(frames):
    """A stand-in path: result t = 3 f_t + f_(t-1); the run's first frame has no
    predecessor (as the tracking step, whose first frame has no points)."""
    out = 3 * frames.astype(np.int64)
    out[1:] += frames[:-1]
    return {"r": out, "first": np.arange(len(frames)) == 0}


@pytest.mark.parametrize("T,world", [(10, 3), (5, 5), (3, 4), (1, 2), (64, 8)])
def test_one_frame_halo_gives_the_whole_video(T, world):
    frames = np.random.default_rng(T * 31 + world).integers(0, 256, size=(T, 4, 6))
    whole = _one_frame_reach(frames)
    parts = []
    for r in range(world):
        s0, t0, t1 = shard.span(T, world, r)
        parts.append(shard.keep(_one_frame_reach(frames[s0:t1]), s0, t0) if t1 > t0 else {})
    merged = shard.merge(parts)
    assert merged.keys() == whole.keys()
    for k in whole:
        assert np.array_equal(merged[k], whole[k])
    # without the halo frame every later shard's first frame loses its predecessor
    if world > 1 and T > world:
        no_halo = shard.merge([_one_frame_reach(frames[t0:t1]) for t0, t1 in shard.frame_ranges(T, world)])
        assert not np.array_equal(no_halo["r"], whole["r"])


def test_bad_arguments():
    with pytest.raises(ValueError):
        shard.frame_ranges(5, 0)
    with pytest.raises(ValueError):
        shard.frame_ranges(-1, 2)
    with pytest.raises(ValueError):
        shard.span(5, 2, 2)
    with pytest.raises(ValueError):
        shard.merge([{"a": np.zeros(1)}, {"b": np.zeros(1)}])
    assert shard.merge([{}, {}]) == {}


# ------------------------------------------------------------------ two gloo ranks
SPEC = dict(T=9, H=40, W=52, seed=17, n_blobs=6, n_patches=4)
KP = 16


def _oracle_results(frames, W):
    from oracle import chain as oc
    masks, counts, _, _ = oc.chain_volume(frames, W, nthreads=1)
    n, idx, u, v, st, _ = oc.track_volume(frames, W, K=KP, nthreads=1)
    return {"mask": masks, "counts": counts, "n_points": n, "idx": idx, "u": u, "v": v, "status": st}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from synth import video as sv
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = sv.VideoSpec(**SPEC)
    s0, t0, t1 = shard.span(spec.T, world, rank)
    frames, _ = sv.generate(spec, pitch=sv.pitch_for(spec.W), frames=range(s0, t1))
    kept = shard.keep(_oracle_results(frames, spec.W), s0, t0)
    merged = shard.gather_merge(kept, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, merged))


def test_two_ranks_merge_to_the_whole_video_tracking():
    from oracle import chain as oc
    from synth import video as sv
    oc.build()  # once, before the ranks start
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] is None
    spec = sv.VideoSpec(**SPEC)
    frames, _ = sv.generate(spec, pitch=sv.pitch_for(spec.W))
    whole = _oracle_results(frames, spec.W)
    merged = res[0]
    assert int(whole["n_points"][5]) > 0  # rank 1's first owned frame tracks points
    for k in whole:
        assert np.array_equal(merged[k], whole[k]), k


def test_benchmark_ranks_render_their_ranges_of_one_video():
    import bench
    from synth import video as sv
    world, T = 3, 4
    P = sv.pitch_for(bench.SPEC.W)
    whole, _ = sv.generate(bench.SPEC, pitch=P, frames=range(world * T))
    owned = []
    for r in range(world):
        fr, P2, own = bench.make_video(r, world, T)
        assert P2 == P and own == T and len(fr) == T + (1 if r else 0)
        assert np.array_equal(fr, whole[max(r * T - 1, 0):(r + 1) * T])
        owned.append(fr[len(fr) - own:])
    assert np.array_equal(np.concatenate(owned), whole)
    # one rank: the single-GPU workload's own first frames
    fr, _, own = bench.make_video(0, 1, 2)
    assert own == 2 and np.array_equal(fr, whole[:2])
