"""Batched form: uneven videos through one persistent launch replayed from a CUDA graph.

Every video's mask, counts and tracks must equal, bit for bit, what kf_run (full
fusion) and kf_track give for that video alone, on two replays of the graph, and agree
with the FP64 oracle on every frame (masks and counts under the exemption rule, tracks
by the tracking parity rule); a batch with one video of each shape of the 48-video
workload is checked against the oracle on sampled frames; the autotuner must return one
of its candidates and keep it in the context.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import chain as oc  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402
from tests._parity import TOL_F32, check_mask  # noqa: E402
from tests._track_parity import check_frame  # noqa: E402

SHAPES = [(3, 64, 100), (5, 40, 300), (2, 130, 77), (4, 96, 150), (1, 20, 20), (2, 7, 3)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def _videos(dev):
    out = []
    for i, (T, H, W) in enumerate(SHAPES):
        fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=60 + i, n_blobs=6, n_patches=4), pitch=sv.pitch_for(W))
        out.append((torch.from_numpy(fr).to(dev), W))
    return out


def _check_against_oracle(fr, W, mask, counts, tracks, frames):
    """Masks and counts of the listed frames against the oracle; with tracks, each listed
    frame t >= 1 also by the tracking parity rule against the pair (t - 1, t)."""
    checked = 0
    for t in frames:
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        check_mask(mask[t, :, :W], int(counts[t]), m_ref, c_ref, maps["r"], TOL_F32)
        if tracks is not None and t >= 1:
            checked += check_frame(fr, t, W, tracks, tracks["idx"].shape[1])
    return checked


@pytest.mark.parametrize("track", [False, True])
def test_batch_equals_per_video_runs(dev, track):
    ctx = K.Context(0)
    vids = _videos(dev)
    KP = 16
    masks = [torch.full_like(f, 5) for f, _ in vids]
    counts = [torch.full((f.shape[0],), -1, dtype=torch.int32, device=dev) for f, _ in vids]
    tracks = None
    if track:
        tracks = []
        for f, _ in vids:
            T = f.shape[0]
            tracks.append((KP, torch.full((T,), -1, dtype=torch.int32, device=dev),
                           torch.full((T, KP), -1, dtype=torch.int32, device=dev),
                           torch.zeros((T, KP), device=dev), torch.zeros((T, KP), device=dev),
                           torch.full((T, KP), -1, dtype=torch.int32, device=dev)))
    ws = torch.empty(K.kf_batch_workspace_bytes(ctx.h, [f for f, _ in vids], [w for _, w in vids], KP if track else 0),
                     dtype=torch.uint8, device=dev)
    b = K.kf_batch_create(ctx.h, [f for f, _ in vids], [w for _, w in vids], masks, counts, ws, tracks)
    try:
        for rep in range(2):
            if rep:
                for m in masks:
                    m.fill_(5)
            K.kf_batch_run(b)
            torch.cuda.synchronize()
            assert K.kf_device_error(ctx.h) == 0
            for i, (f, W) in enumerate(vids):
                T = f.shape[0]
                m_ref = torch.zeros_like(f)
                c_ref = torch.zeros(T, dtype=torch.int32, device=dev)
                if track:
                    n_r = torch.zeros(T, dtype=torch.int32, device=dev)
                    i_r = torch.zeros((T, KP), dtype=torch.int32, device=dev)
                    u_r, v_r = torch.zeros((T, KP), device=dev), torch.zeros((T, KP), device=dev)
                    s_r = torch.zeros((T, KP), dtype=torch.int32, device=dev)
                    wst = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, f.shape[1], T), dtype=torch.uint8, device=dev)
                    K.kf_track(ctx.h, f, W, m_ref, c_ref, KP, n_r, i_r, u_r, v_r, s_r, wst)
                    _, n_b, i_b, u_b, v_b, s_b = tracks[i]
                    assert torch.equal(n_b, n_r), i
                    for t in range(1, T):
                        n = int(n_r[t])
                        assert torch.equal(i_b[t, :n], i_r[t, :n]), (i, t)
                        assert torch.equal(u_b[t, :n], u_r[t, :n]) and torch.equal(v_b[t, :n], v_r[t, :n]), (i, t)
                        assert torch.equal(s_b[t, :n], s_r[t, :n]), (i, t)
                else:
                    K.kf_run(ctx.h, 0, f, W, m_ref, c_ref, None)
                assert torch.equal(masks[i][:, :, :W], m_ref[:, :, :W]), i
                assert torch.all(masks[i][:, :, W:] == 5), i
                assert torch.equal(counts[i], c_ref), i
                if rep == 0:  # every frame of every video against the oracle
                    tr = None
                    if track:
                        _, n_b, i_b, u_b, v_b, s_b = tracks[i]
                        tr = dict(n=n_b.cpu().numpy(), idx=i_b.cpu().numpy(), u=u_b.cpu().numpy(),
                                  v=v_b.cpu().numpy(), st=s_b.cpu().numpy())
                    _check_against_oracle(f.cpu().numpy(), W, masks[i].cpu().numpy(), counts[i].cpu().numpy(), tr,
                                          range(T))
    finally:
        K.kf_batch_destroy(b)


def test_autotuner_picks_a_candidate(dev):
    ctx = K.Context(0)
    fr, _ = sv.generate(sv.VideoSpec(T=8, H=200, W=300, seed=70), pitch=sv.pitch_for(300))
    f = torch.from_numpy(fr).to(dev)
    m = torch.zeros_like(f)
    c = torch.zeros(8, dtype=torch.int32, device=dev)
    best, ms = K.kf_tune_chunk_rows(ctx.h, f, 300, m, c, [32, 100, 200], reps=2)
    assert best in (32, 100, 200) and ms > 0
    m2 = torch.zeros_like(f)
    c2 = torch.zeros_like(c)
    K.kf_set_chunk_rows(ctx.h, 200)
    K.kf_run(ctx.h, 0, f, 300, m2, c2, None)
    assert torch.equal(m, m2) and torch.equal(c, c2)


def test_batch_of_the_48_video_shapes_matches_the_oracle(dev):
    """One video of each shape of the 48-video workload (192x432x600, 480x640x300,
    800x600x1000, 1080x1920x120; each cycling its first 32 generated frames, as the
    workload does) in one batch with 256 points per frame; sampled frames of every video
    (including the seam where a video's frames wrap) against the oracle."""
    ctx = K.Context(0)
    KP = 256
    hosts, vids, masks, counts, tracks = [], [], [], [], []
    for i, (H, W, T) in enumerate([(192, 432, 600), (480, 640, 300), (800, 600, 1000), (1080, 1920, 120)]):
        P = sv.pitch_for(W)
        base, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=1000 + 16 * i), pitch=P, frames=range(32))
        fr = np.concatenate([base] * ((T + 31) // 32))[:T]
        hosts.append((fr, W))
        f = torch.from_numpy(fr).to(dev)
        vids.append(f)
        masks.append(torch.zeros_like(f))
        counts.append(torch.zeros(T, dtype=torch.int32, device=dev))
        tracks.append((KP, torch.zeros(T, dtype=torch.int32, device=dev),
                       torch.zeros((T, KP), dtype=torch.int32, device=dev), torch.zeros((T, KP), device=dev),
                       torch.zeros((T, KP), device=dev), torch.zeros((T, KP), dtype=torch.int32, device=dev)))
    Ws = [w for _, w in hosts]
    ws = torch.empty(K.kf_batch_workspace_bytes(ctx.h, vids, Ws, KP), dtype=torch.uint8, device=dev)
    b = K.kf_batch_create(ctx.h, vids, Ws, masks, counts, ws, tracks)
    try:
        K.kf_batch_run(b)
        torch.cuda.synchronize()
        assert K.kf_device_error(ctx.h) == 0
    finally:
        K.kf_batch_destroy(b)
    checked = 0
    for (fr, W), m, c, tr in zip(hosts, masks, counts, tracks):
        T = fr.shape[0]
        _, n_b, i_b, u_b, v_b, s_b = tr
        tr_np = dict(n=n_b.cpu().numpy(), idx=i_b.cpu().numpy(), u=u_b.cpu().numpy(), v=v_b.cpu().numpy(),
                     st=s_b.cpu().numpy())
        assert tr_np["n"][0] == 0
        checked += _check_against_oracle(fr, W, m.cpu().numpy(), c.cpu().numpy(), tr_np, (1, 32, T // 2, T - 1))
    assert checked >= 4 * 4 * 100


def test_batch_with_per_video_tiles_and_fewer_warps_gives_the_same_bits(dev):
    """kf_batch_create_ex: each video with its own tile height, the launch capped at 3
    resident warps per SM, the queue in longest-job-first order: every result equals the
    video's own kf_track (tile heights never change the bits)."""
    ctx = K.Context(0)
    vids = _videos(dev)
    KP = 16
    masks = [torch.zeros_like(f) for f, _ in vids]
    counts = [torch.zeros((f.shape[0],), dtype=torch.int32, device=dev) for f, _ in vids]
    tracks = [(KP, torch.zeros((f.shape[0],), dtype=torch.int32, device=dev),
               torch.full((f.shape[0], KP), -1, dtype=torch.int32, device=dev), torch.zeros((f.shape[0], KP), device=dev),
               torch.zeros((f.shape[0], KP), device=dev), torch.zeros((f.shape[0], KP), dtype=torch.int32, device=dev))
              for f, _ in vids]
    ws = torch.empty(K.kf_batch_workspace_bytes(ctx.h, [f for f, _ in vids], [w for _, w in vids], KP),
                     dtype=torch.uint8, device=dev)
    rows = [37, 100, 5, 200, 1, 3]
    b = K.kf_batch_create(ctx.h, [f for f, _ in vids], [w for _, w in vids], masks, counts, ws, tracks,
                          chunk_rows=rows, warps_per_sm=3)
    try:
        K.kf_batch_run(b)
        torch.cuda.synchronize()
        assert K.kf_device_error(ctx.h) == 0
    finally:
        K.kf_batch_destroy(b)
    for i, (f, W) in enumerate(vids):
        T = f.shape[0]
        m_r, c_r = torch.zeros_like(f), torch.zeros(T, dtype=torch.int32, device=dev)
        n_r = torch.zeros(T, dtype=torch.int32, device=dev)
        i_r = torch.full((T, KP), -1, dtype=torch.int32, device=dev)
        u_r, v_r = torch.zeros((T, KP), device=dev), torch.zeros((T, KP), device=dev)
        s_r = torch.zeros((T, KP), dtype=torch.int32, device=dev)
        wst = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, f.shape[1], T), dtype=torch.uint8, device=dev)
        K.kf_track(ctx.h, f, W, m_r, c_r, KP, n_r, i_r, u_r, v_r, s_r, wst)
        assert torch.equal(masks[i][:, :, :W], m_r[:, :, :W]) and torch.equal(counts[i], c_r), i
        _, n_b, i_b, u_b, v_b, s_b = tracks[i]
        assert torch.equal(n_b, n_r), i
        for t in range(1, T):
            n = int(n_r[t])
            assert torch.equal(i_b[t, :n], i_r[t, :n]) and torch.equal(u_b[t, :n], u_r[t, :n]), (i, t)
    with pytest.raises(K.KfuseError):  # a tile height below 1
        K.kf_batch_create(ctx.h, [f for f, _ in vids], [w for _, w in vids], masks, counts, ws, tracks,
                          chunk_rows=[0] * len(vids))
