"""Frame-range shards of one video, each run by kf_track on the view of its frames plus
the one frame before them, merge on the host to the whole-video kf_track bit for bit
(mask, counts, points, velocities, status). The shards run one after another on one
GPU, as separate processes would run them on separate GPUs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from paper_1509_04394_gb300 import shard  # noqa: E402
from synth import video as sv  # noqa: E402

KP = 64


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def track(ctx, frames, W, dev):
    """kf_track over a device video (any contiguous run of frames); host results."""
    T, H, P = frames.shape
    mask = torch.zeros_like(frames)
    counts = torch.full((T,), -1, dtype=torch.int32, device=dev)
    n = torch.full((T,), -1, dtype=torch.int32, device=dev)
    idx = torch.full((T, KP), -1, dtype=torch.int32, device=dev)
    u = torch.zeros((T, KP), dtype=torch.float32, device=dev)
    v = torch.zeros((T, KP), dtype=torch.float32, device=dev)
    st = torch.full((T, KP), -1, dtype=torch.int32, device=dev)
    ws = torch.empty(max(K.kf_track_workspace_bytes(ctx.h, W, H, T), 256), dtype=torch.uint8, device=dev)
    K.kf_track(ctx.h, frames, W, mask, counts, KP, n, idx, u, v, st, ws)
    assert K.kf_device_error(ctx.h) == 0
    return {k: t.cpu().numpy() for k, t in
            dict(mask=mask, counts=counts, n_points=n, idx=idx, u=u, v=v, status=st).items()}


@pytest.mark.parametrize("spec,world", [
    (sv.VideoSpec(T=23, H=192, W=432, seed=41), 3),
    (sv.VideoSpec(T=23, H=192, W=432, seed=41), 7),
    (sv.VideoSpec(T=11, H=96, W=600, seed=42, n_blobs=12, n_patches=8), 4),
])
def test_frame_shards_merge_to_the_whole_video(dev, spec, world):
    fr, _ = sv.generate(spec, pitch=sv.pitch_for(spec.W))
    frames = torch.from_numpy(fr).to(dev)
    ctx = K.Context(0)
    whole = track(ctx, frames, spec.W, dev)
    assert int(whole["n_points"][1:].min()) > 0
    parts = []
    for r in range(world):
        s0, t0, t1 = shard.span(spec.T, world, r)
        view = frames[s0:t1]  # a contiguous view: 16-byte aligned since the pitch is
        parts.append(shard.keep(track(ctx, view, spec.W, dev), s0, t0))
    merged = shard.merge(parts)
    for k in whole:
        assert np.array_equal(merged[k], whole[k]), k
