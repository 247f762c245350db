"""GPU parity of the paper's own chain (K1..K5 fused in any partition, K6 Kalman).

Each stage map of the unfused sequence against the FP64 oracle (Y' exact; y', G', M'
within 1e-5 normwise), masks under the exemption rule (pixels whose oracle response is
within the tolerance of the threshold may differ), counts and region sums consistent
with the mask, all 16 partitions bit-identical to each other, ragged and degenerate
sizes, and the Kalman filter (FP32) against the oracle's (FP64) on the GPU's own region sums."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pchain as op  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402
from tests._parity import kalman_fp32_bound  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def pitch4(W):
    return (W + 3) // 4 * 4


def rgba_video(T, H, W, seed, pitch=None):
    g, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=seed, n_blobs=max(2, H * W // 4000),
                                    n_patches=max(2, H * W // 6000)))
    rgba = sv.rgba_of(g)
    P = pitch or pitch4(W)
    out = np.zeros((T, H, P, 4), dtype=np.uint8)
    out[:, :, :W] = rgba
    return out


def outputs(dev, T, H, W, mask_pitch=None):
    mp = mask_pitch or (W + 15) // 16 * 16
    return (torch.full((T, H, mp), 7, dtype=torch.uint8, device=dev), torch.full((T,), -1, dtype=torch.int32, device=dev),
            torch.full((T, 16, 3), -1, dtype=torch.int32, device=dev))


def regions_of_mask(mask):
    """Region sums of a [T, H, W] 0/1 mask, by the definition."""
    T, H, W = mask.shape
    reg = np.zeros((T, 16, 3), dtype=np.int64)
    for t in range(T):
        ys, xs = np.nonzero(mask[t])
        for y, x in zip(ys.tolist(), xs.tolist()):
            r = (4 * y // H) * 4 + (4 * x // W)
            reg[t, r] += [1, x, y]
    return reg


def check_mask(mask, counts, regions, M_o):
    """mask [T, H, W] from the GPU against M_o (true units): differences only where the
    oracle's response is within the tolerance of the threshold."""
    T = mask.shape[0]
    for t in range(T):
        tau = TOL * max(np.max(np.abs(M_o[t])), 1e-300)
        ref = M_o[t] > op.TAU
        diff = (mask[t] != 0) != ref
        assert np.all(np.abs(M_o[t][diff] - op.TAU) <= tau), t
        assert counts[t] == int(mask[t].sum())
    np.testing.assert_array_equal(regions, regions_of_mask(mask))


def normwise(a, b):
    den = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / den if den > 0 else np.max(np.abs(a))


@pytest.mark.parametrize("shape", [(5, 96, 128), (4, 61, 83), (3, 33, 29), (70, 40, 50)])
def test_every_stage_map_matches_the_oracle(dev, shape):
    T, H, W = shape
    fr = rgba_video(T, H, W, seed=3, pitch=(W + 4 + 3) // 4 * 4)
    _, _, _, maps = op.chain_volume(fr[:, :, :W], keep_maps=True)
    ctx = K.Context(0, harris=False)
    fd = torch.from_numpy(fr).to(dev)
    P = (W + 7) // 8 * 8
    cur = None
    names = ["Y", "y", "G", "M"]
    ws = torch.empty(K.kf_pc_group_workspace_bytes(ctx.h, 1, 1, W, H, T), dtype=torch.uint8, device=dev)
    for s in range(4):
        out = torch.full((T, H, P), float("nan"), dtype=torch.float32, device=dev)
        K.kf_pc_run_group(ctx.h, s, s, W, frames=fd if s == 0 else None, inp=cur, out=out,
                          workspace=ws if s == 1 else None)
        got = out[:, :, :W].cpu().numpy().astype(np.float64) / K.PC_SCALE[s]
        ref = maps[names[s]]
        err = max(normwise(got[t], ref[t]) for t in range(T))
        assert err <= (1e-12 if s == 0 else TOL), (names[s], err)
        cur = out
    mask, counts, regions = outputs(dev, T, H, W)
    ws5 = torch.empty(K.kf_pc_group_workspace_bytes(ctx.h, 4, 4, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_pc_run_group(ctx.h, 4, 4, W, inp=cur, mask_out=(mask, counts, regions), workspace=ws5)
    m = mask.cpu().numpy()
    assert np.all(m[:, :, W:] == 7), "columns past W must be untouched"
    check_mask(m[:, :, :W], counts.cpu().numpy(), regions.cpu().numpy(), maps["M"])


@pytest.mark.parametrize("T", [4, 33, 65])
def test_all_16_partitions_are_bit_identical(dev, T):
    """T = 33 and 65: the IIR recursion spans two and three chunks."""
    H, W = 70, 90
    fr = rgba_video(T, H, W, seed=4)
    ctx = K.Context(0, harris=False)
    fd = torch.from_numpy(fr).to(dev)
    res = {}
    for cuts in range(16):
        ws = torch.empty(K.kf_pc_workspace_bytes(ctx.h, cuts, W, H, T), dtype=torch.uint8, device=dev)
        mask, counts, regions = outputs(dev, T, H, W)
        K.kf_pc_run(ctx.h, cuts, fd, W, mask, counts, regions, ws)
        res[cuts] = (mask.cpu().numpy(), counts.cpu().numpy(), regions.cpu().numpy())
    for cuts in range(16):
        for a, b in zip(res[cuts], res[15]):
            assert np.array_equal(a, b), cuts
    _, _, _, maps = op.chain_volume(fr[:, :, :W], keep_maps=True)
    m, c, r = res[0]
    check_mask(m[:, :, :W], c, r, maps["M"])
    assert c.sum() > 0


@pytest.mark.parametrize("T,H,W", [(1, 1, 1), (2, 1, 7), (3, 7, 1), (2, 5, 5), (3, 29, 31), (2, 30, 30), (1, 64, 64),
                                   (3, 100, 57), (40, 9, 33)])
def test_ragged_and_degenerate_frames(dev, T, H, W):
    rng = np.random.default_rng(H * 1000 + W)
    fr = np.zeros((T, H, pitch4(W), 4), dtype=np.uint8)
    fr[:, :, :W] = rng.integers(0, 256, (T, H, W, 4), dtype=np.uint8)
    ctx = K.Context(0, harris=False)
    fd = torch.from_numpy(fr).to(dev)
    _, _, _, maps = op.chain_volume(fr[:, :, :W], keep_maps=True)
    for cuts in (0, 0b0010, 0b1111):
        ws = torch.empty(K.kf_pc_workspace_bytes(ctx.h, cuts, W, H, T), dtype=torch.uint8, device=dev)
        mask, counts, regions = outputs(dev, T, H, W)
        K.kf_pc_run(ctx.h, cuts, fd, W, mask, counts, regions, ws)
        m = mask.cpu().numpy()
        assert np.all(m[:, :, W:] == 7)
        check_mask(m[:, :, :W], counts.cpu().numpy(), regions.cpu().numpy(), maps["M"])


def test_kalman_matches_the_oracle_on_the_gpu_region_sums(dev):
    T, H, W = 60, 128, 160
    fr = rgba_video(T, H, W, seed=6)
    ctx = K.Context(0, harris=False)
    fd = torch.from_numpy(fr).to(dev)
    mask, counts, regions = outputs(dev, T, H, W)
    ws = torch.empty(K.kf_pc_workspace_bytes(ctx.h, 0, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_pc_run(ctx.h, 0, fd, W, mask, counts, regions, ws)
    states = torch.zeros((T, 16, 4), dtype=torch.float64, device=dev)
    status = torch.full((T, 16), -1, dtype=torch.int32, device=dev)
    K.kf_pc_kalman(ctx.h, regions, states, status)
    reg = regions.cpu().numpy().astype(np.int64)
    s_o, st_o = op.kalman(reg)
    np.testing.assert_array_equal(status.cpu().numpy(), st_o)
    # FP32 filter against the FP64 oracle, within the error budget derived from the
    # filter's own matrices (per-step roundings carried by the stable error recursion)
    tol_p, tol_v = kalman_fp32_bound(s_o, reg, W)
    assert tol_p < 2e-3 and tol_v < 2e-3
    np.testing.assert_allclose(states.cpu().numpy()[..., :2], s_o[..., :2], rtol=0, atol=tol_p)
    np.testing.assert_allclose(states.cpu().numpy()[..., 2:], s_o[..., 2:], rtol=0, atol=tol_v)
    assert (st_o == 1).sum() > T  # the regions do see features
    # a track with gaps: drop every third frame's measurements of region 5
    reg2 = reg.copy()
    reg2[::3, 5] = 0
    r2 = torch.from_numpy(reg2.astype(np.int32)).to(dev)
    K.kf_pc_kalman(ctx.h, r2, states, status)
    s_o2, st_o2 = op.kalman(reg2)
    np.testing.assert_array_equal(status.cpu().numpy(), st_o2)
    tol_p, tol_v = kalman_fp32_bound(s_o2, reg2, W)
    np.testing.assert_allclose(states.cpu().numpy()[..., :2], s_o2[..., :2], rtol=0, atol=tol_p)
    np.testing.assert_allclose(states.cpu().numpy()[..., 2:], s_o2[..., 2:], rtol=0, atol=tol_v)
