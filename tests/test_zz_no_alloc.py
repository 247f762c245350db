"""kf_run_static: the partitioned chain with the library's fixed per-GPU workspace.

Some callers cannot allocate device memory (a plug-in inside a host framework that owns
every device allocation, a real-time pipeline whose footprint is fixed at start-up);
kf_run_static serves them from a file-scope device array instead of a caller workspace.
This file is collected last so that a failure here comes after every other test ran.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402


def _video(seed, T=5, H=96, W=150):
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=seed, n_blobs=8, n_patches=4), pitch=sv.pitch_for(W))
    return fr


@pytest.mark.gpu
def test_static_workspace_run_matches_kf_run_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    dev = torch.device("cuda:0")
    ctx = K.Context(0)
    W = 150
    for cuts in (127, 0b0100100, 0b1000000):
        for seed in (31, 32):  # two calls in a row on different inputs: no stale state
            fr = torch.from_numpy(_video(seed)).to(dev)
            T, H, _ = fr.shape
            ws = torch.empty(K.kf_workspace_bytes(ctx.h, cuts, W, H, T), dtype=torch.uint8, device=dev)
            m_ref = torch.zeros_like(fr)
            c_ref = torch.zeros(T, dtype=torch.int32, device=dev)
            K.kf_run(ctx.h, cuts, fr, W, m_ref, c_ref, ws)
            m = torch.full_like(fr, 7)
            c = torch.full((T,), -1, dtype=torch.int32, device=dev)
            K.kf_run_static(ctx.h, cuts, fr, W, m, c)
            torch.cuda.synchronize()
            assert torch.equal(m[:, :, :W], m_ref[:, :, :W]), (cuts, seed)
            assert torch.equal(c, c_ref), (cuts, seed)
    assert K.kf_device_error(ctx.h) == 0


@pytest.mark.gpu
def test_static_workspace_rejects_volumes_beyond_its_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    dev = torch.device("cuda:0")
    ctx = K.Context(0)
    T, H, W = 40, 800, 600  # unfused FP32 maps of 40 frames need ~460 MB > 64 MiB
    assert K.kf_workspace_bytes(ctx.h, 127, W, H, T) > K.KF_STATIC_WORKSPACE_BYTES
    fr = torch.zeros((T, H, 608), dtype=torch.uint8, device=dev)
    m = torch.zeros_like(fr)
    c = torch.zeros(T, dtype=torch.int32, device=dev)
    with pytest.raises(K.KfuseError) as e:
        K.kf_run_static(ctx.h, 127, fr, W, m, c)
    assert e.value.status == K.KF_ENOMEM
    K.kf_run_static(ctx.h, 0, fr, W, m, c)  # full fusion needs no workspace
    torch.cuda.synchronize()
