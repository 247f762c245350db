"""The bounded-wait timeout path, run on the GPU without a fault.

Every wait of the chain kernels and of the spatio-temporal box kernel for staged input
is bounded. Lowering the bound to 0 polls (kf_set_wait_polls) makes each first wait
expire at once: the kernel records KF_DEVERR_TIMEOUT in the context's error word, waits
with the full bound for the copies it issued, and ends its job. The call itself
succeeds, the host reads the timeout from kf_device_error, the outputs of the expired
jobs stay unwritten, and with the default bound restored the same context gives the
full, correct results again.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402

DEVERR_TIMEOUT = 1
DEFAULT_POLLS = 1 << 22


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def test_chain_wait_expires_and_the_context_recovers(dev):
    T, H, W = 4, 120, 300
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=91, n_blobs=8, n_patches=4), pitch=sv.pitch_for(W))
    frames = torch.from_numpy(fr).to(dev)
    ctx = K.Context(0)
    ref_m, ref_c = torch.zeros_like(frames), torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, 0, frames, W, ref_m, ref_c, None)
    assert K.kf_device_error(ctx.h) == 0 and int(ref_c.sum()) > 0

    K.kf_set_wait_polls(ctx.h, 0)
    mask = torch.full_like(frames, 7)
    counts = torch.full((T,), -1, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, 0, frames, W, mask, counts, None)  # enqueued and returned: no host error
    assert K.kf_device_error(ctx.h) == DEVERR_TIMEOUT
    assert torch.all(mask == 7)  # every job ended at its first wait: no output row written
    assert torch.all(counts == 0)  # zeroed by the call, nothing added
    assert K.kf_device_error(ctx.h) == 0  # reading the word cleared it

    # the unfused sequence and the tracking path take the same way out
    cuts = 127
    ws = torch.empty(K.kf_workspace_bytes(ctx.h, cuts, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_run(ctx.h, cuts, frames, W, mask, counts, ws)
    assert K.kf_device_error(ctx.h) == DEVERR_TIMEOUT
    Kp = 16
    n_pts = torch.zeros(T, dtype=torch.int32, device=dev)
    idx = torch.zeros((T, Kp), dtype=torch.int32, device=dev)
    u, v = torch.zeros((T, Kp), device=dev), torch.zeros((T, Kp), device=dev)
    st = torch.zeros((T, Kp), dtype=torch.int32, device=dev)
    wst = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_track(ctx.h, frames, W, mask, counts, Kp, n_pts, idx, u, v, st, wst)
    assert K.kf_device_error(ctx.h) == DEVERR_TIMEOUT
    assert torch.all(n_pts == 0)  # no corner reached the selection

    K.kf_set_wait_polls(ctx.h, DEFAULT_POLLS)
    for c in (0, cuts):
        mask.fill_(7)
        K.kf_run(ctx.h, c, frames, W, mask, counts, ws)
        assert K.kf_device_error(ctx.h) == 0
        assert torch.equal(mask[:, :, :W], ref_m[:, :, :W]) and torch.equal(counts, ref_c)
    K.kf_track(ctx.h, frames, W, mask, counts, Kp, n_pts, idx, u, v, st, wst)
    assert K.kf_device_error(ctx.h) == 0
    assert torch.equal(counts, ref_c) and int(n_pts[1]) == min(Kp, int(ref_c[1]))


def test_box_kernel_wait_expires_and_the_context_recovers(dev):
    T, H, W = 6, 64, 80
    g, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=92, n_blobs=4, n_patches=2))
    fr = np.zeros((T, H, W, 4), dtype=np.uint8)
    fr[:] = sv.rgba_of(g)
    frames = torch.from_numpy(fr).to(dev)
    ctx = K.Context(0)
    mp = (W + 15) // 16 * 16
    ref_m = torch.zeros((T, H, mp), dtype=torch.uint8, device=dev)
    ref_c = torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_st_run(ctx.h, frames, W, ref_m, ref_c, 2, 16, 3)
    assert K.kf_device_error(ctx.h) == 0 and int(ref_c.sum()) > 0

    K.kf_set_wait_polls(ctx.h, 0)
    mask = torch.full((T, H, mp), 7, dtype=torch.uint8, device=dev)
    counts = torch.full((T,), -1, dtype=torch.int32, device=dev)
    K.kf_st_run(ctx.h, frames, W, mask, counts, 2, 16, 3)
    assert K.kf_device_error(ctx.h) == DEVERR_TIMEOUT
    assert torch.all(mask == 7)  # every box ended at its first frame's wait

    K.kf_set_wait_polls(ctx.h, DEFAULT_POLLS)
    K.kf_st_run(ctx.h, frames, W, mask, counts, 2, 16, 3)
    assert K.kf_device_error(ctx.h) == 0
    assert torch.equal(mask[:, :, :W], ref_m[:, :, :W]) and torch.equal(counts, ref_c)
