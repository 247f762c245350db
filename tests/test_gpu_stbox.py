"""GPU parity of the spatio-temporal box group (integer chain: bit-exact masks and counts
against the reference) over box shapes, temporal reaches, ragged and tiny volumes, and
sampled frames of the full 1024 x 1024 x 1000 workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import stbox as ost  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def rgba_video(T, H, W, seed, frames=None):
    spec = sv.VideoSpec(T=T, H=H, W=W, seed=seed, n_blobs=max(2, H * W // 4000), n_patches=max(2, H * W // 6000))
    g, _ = sv.generate(spec, frames=frames if frames is not None else range(T))
    P = (W + 3) // 4 * 4
    out = np.zeros((g.shape[0], H, P, 4), dtype=np.uint8)
    out[:, :, :W] = sv.rgba_of(g)
    return out


def run(dev, fr, W, n, x, t):
    T, H = fr.shape[:2]
    ctx = K.Context(0)
    frames = torch.from_numpy(fr).to(dev)
    mp = (W + 15) // 16 * 16
    mask = torch.full((T, H, mp), 7, dtype=torch.uint8, device=dev)
    counts = torch.full((T,), -1, dtype=torch.int32, device=dev)
    K.kf_st_run(ctx.h, frames, W, mask, counts, n, x, t)
    torch.cuda.synchronize()
    assert K.kf_device_error(ctx.h) == 0
    m = mask.cpu().numpy()
    assert (m[:, :, W:] == 7).all()  # pitch padding untouched
    return m[:, :, :W], counts.cpu().numpy()


@pytest.mark.parametrize("n", ost.TAPS)
@pytest.mark.parametrize("x,t", [(8, 1), (16, 3), (32, 4), (48, 7), (64, 2)])
def test_masks_and_counts_bit_exact(dev, n, x, t):
    T, H, W = 9, 75, 110  # several boxes, ragged in every axis
    fr = rgba_video(T, H, W, seed=20 + n)
    m, c = run(dev, fr, W, n, x, t)
    mo, co, _ = ost.chain_volume(fr[:, :, :W], n)
    assert mo.sum() > 0
    np.testing.assert_array_equal(m, mo)
    np.testing.assert_array_equal(c, co)


@pytest.mark.parametrize("T,H,W,x,t", [(1, 3, 5, 8, 1), (2, 8, 8, 8, 5), (3, 1, 17, 16, 2), (6, 40, 4, 64, 6),
                                       (5, 98, 100, 96, 2), (4, 50, 101, 48, 3)])
def test_tiny_and_single_box_volumes(dev, T, H, W, x, t):
    n = 4 if x == 96 else 2
    fr = rgba_video(T, H, W, seed=T * 31 + W)
    m, c = run(dev, fr, W, n, x, t)
    mo, co, _ = ost.chain_volume(fr[:, :, :W], n)
    np.testing.assert_array_equal(m, mo)
    np.testing.assert_array_equal(c, co)


def test_empty_video_and_rejections(dev):
    ctx = K.Context(0)
    fr = torch.zeros((0, 8, 8, 4), dtype=torch.uint8, device=dev)
    K.kf_st_run(ctx.h, fr, 8, torch.zeros((0, 8, 16), dtype=torch.uint8, device=dev),
                torch.zeros(0, dtype=torch.int32, device=dev), 2, 8, 4)
    fr = torch.zeros((2, 8, 8, 4), dtype=torch.uint8, device=dev)
    mask = torch.zeros((2, 8, 16), dtype=torch.uint8, device=dev)
    counts = torch.zeros(2, dtype=torch.int32, device=dev)
    for n, x, t in [(3, 8, 1), (2, 12, 1), (2, 8, 0), (2, 128, 1), (1, 24, 1)]:  # bad reach, side, depth
        with pytest.raises(K.KfuseError):
            K.kf_st_run(ctx.h, fr, 8, mask, counts, n, x, t)


def test_full_size_sampled_frames(dev):
    """1024 x 1024 x 1000 in the bench's box (32 x 32 x 16, n = 2): frames sampled across
    the volume (box starts, ends and interiors) against the reference of each frame from
    its own n previous frames."""
    T, H, W, n = 1000, 1024, 1024, 2
    fr = rgba_video(T, H, W, seed=7)
    ctx = K.Context(0)
    frames = torch.from_numpy(fr).to(dev)
    mask = torch.zeros((T, H, W), dtype=torch.uint8, device=dev)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_st_run(ctx.h, frames, W, mask, counts, n, 32, 16)
    torch.cuda.synchronize()
    assert K.kf_device_error(ctx.h) == 0
    cnt = counts.cpu().numpy()
    for f in (0, 1, 15, 16, 17, 500, 511, 999):
        lo = max(f - n, 0)
        mo, co, _ = ost.chain_volume(fr[lo:f + 1], n)
        np.testing.assert_array_equal(mask[f].cpu().numpy(), mo[-1])
        assert cnt[f] == co[-1]
    # every count equals its mask's
    np.testing.assert_array_equal(cnt, mask.view(T, -1).sum(dim=1, dtype=torch.int64).cpu().numpy())


def test_box_tuner_returns_the_fastest_candidate_and_the_same_results(dev):
    T, H, W, n = 20, 96, 128, 2
    fr = rgba_video(T, H, W, seed=31)
    ctx = K.Context(0)
    frames = torch.from_numpy(fr).to(dev)
    mask = torch.zeros((T, H, W), dtype=torch.uint8, device=dev)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    boxes = [(16, 8), (32, 4), (32, 16), (64, 2)]
    x, t, ms = K.kf_st_tune(ctx.h, frames, W, mask, counts, n, boxes, reps=2)
    assert (x, t) in boxes and ms > 0
    torch.cuda.synchronize()
    m, c = run(dev, fr, W, n, x, t)
    np.testing.assert_array_equal(mask.cpu().numpy(), m)
    np.testing.assert_array_equal(counts.cpu().numpy(), c)
    with pytest.raises(K.KfuseError):  # an unsupported side
        K.kf_st_tune(ctx.h, frames, W, mask, counts, n, [(24, 4)])
