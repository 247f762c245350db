"""GPU parity of the fused chain against the FP64 oracle, through the C ABI.

* every stage map of the unfused sequence (Sec. III) vs the oracle's map;
* every one of the 128 partitions (Sec. VI) bit-identical to the unfused sequence in
  FP32 (stages 1-4 are exact and later stages share one device function);
* masks and counts vs the oracle under the exemption rule for float-decided pixels;
* ragged and degenerate sizes, chunking, FP16 maps, and the full-size workload on
  sampled frames in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import chain as oc  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402
from tests._parity import (TOL_F16, TOL_F32, check_mask, normwise, pitch16)  # noqa: E402

MAP_KEYS = (("f",), ("g1",), ("g",), ("ix", "iy"), ("pxx", "pxy", "pyy"), ("sxx", "sxy", "syy"), ("r",))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def frames_of(spec, n=None, pitch=None):
    fr, _ = sv.generate(spec, pitch=pitch or pitch16(spec.W), frames=range(n or spec.T))
    return fr


def random_frames(T, H, W, seed):
    rng = np.random.default_rng(seed)
    fr = np.zeros((T, H, pitch16(W)), dtype=np.uint8)
    # smooth-ish content with corners: blocky noise plus a ramp
    base = rng.integers(0, 256, size=(T, (H + 3) // 4, (W + 3) // 4), dtype=np.uint8)
    big = np.repeat(np.repeat(base, 4, axis=1), 4, axis=2)[:, :H, :W]
    fr[:, :, :W] = big
    return fr


def map_dtypes(prec, s):
    """(kf dtype, torch dtype) of the map written by 0-based stage s."""
    if prec == K.KF_PREC_F32:
        return K.KF_DT_F32, torch.float32
    return (K.KF_DT_U16, torch.uint16) if s <= 2 else (K.KF_DT_F16, torch.float16)


def as_f64(t):
    if t.dtype == torch.uint16:  # barebones dtype: reinterpret and widen
        return (t.view(torch.int16).to(torch.int32) & 0xFFFF).double().cpu().numpy()
    return t.double().cpu().numpy()


def run_unfused_maps(ctx_h, prec, fr_dev, W):
    """Each stage as its own kernel; returns the list of output map planes per stage."""
    T, H, _ = fr_dev.shape
    cur, cur_dt, outs = [fr_dev], K.KF_DT_U8, []
    for s in range(7):
        dt, tdt = map_dtypes(prec, s)
        out = [torch.empty((T, H, pitch16(W)), dtype=tdt, device=fr_dev.device) for _ in range(K.MAP_CHANNELS[s + 1])]
        K.kf_run_group(ctx_h, s, s, cur, cur_dt, out, dt, W)
        outs.append(out)
        cur, cur_dt = out, dt
    mask = torch.zeros((T, H, pitch16(W)), dtype=torch.uint8, device=fr_dev.device)
    counts = torch.full((T,), -7, dtype=torch.int32, device=fr_dev.device)
    K.kf_run_group(ctx_h, 7, 7, cur, cur_dt, [mask], K.KF_DT_U8, W, counts)
    return outs, mask, counts


@pytest.mark.parametrize("shape", [(3, 192, 432), (2, 45, 61), (2, 13, 130)])
def test_every_stage_map_matches_the_oracle_fp32(dev, shape):
    T, H, W = shape
    fr = frames_of(sv.VideoSpec(T=T, H=H, W=W, seed=11, n_blobs=8, n_patches=4)) if H > 20 else \
        random_frames(T, H, W, 5)
    ctx = K.Context(0)
    outs, mask, counts = run_unfused_maps(ctx.h, K.KF_PREC_F32, torch.from_numpy(fr).to(dev), W)
    torch.cuda.synchronize()
    for t in range(T):
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        for s in range(7):
            scale = K.kf_map_scale(ctx.h, s)
            for c, key in enumerate(MAP_KEYS[s]):
                got = as_f64(outs[s][c][t, :, :W]) * scale
                err = normwise(got, maps[key])
                bound = 1e-12 if s <= 3 else TOL_F32  # stages 1-4 are exact integers in FP32
                assert err <= bound, (s, key, t, err)
        check_mask(mask[t, :, :W].cpu().numpy(), int(counts[t]), m_ref, c_ref, maps["r"], TOL_F32)


@pytest.mark.parametrize("T,H,W", [(2, 70, 203), (3, 41, 150)])
def test_all_128_partitions_are_bit_identical_to_the_unfused_chain(dev, T, H, W):
    """(3, 41, 150): the last strip of most groups is a half strip run for two frames by
    one warp, and with T odd the last pair has one frame."""
    fr = frames_of(sv.VideoSpec(T=T, H=H, W=W, seed=12, n_blobs=10, n_patches=6))
    ctx = K.Context(0)
    fd = torch.from_numpy(fr).to(dev)
    results = {}
    for cuts in range(128):
        ws_b = K.kf_workspace_bytes(ctx.h, cuts, W, H, T)
        ws = torch.empty(max(ws_b, 1), dtype=torch.uint8, device=dev)
        mask = torch.zeros((T, H, pitch16(W)), dtype=torch.uint8, device=dev)
        counts = torch.zeros(T, dtype=torch.int32, device=dev)
        K.kf_run(ctx.h, cuts, fd, W, mask, counts, ws if ws_b else None)
        results[cuts] = (mask.cpu().numpy(), counts.cpu().numpy())
    assert K.kf_device_error(ctx.h) == 0
    ref_m, ref_c = results[127]
    for cuts, (m, c) in results.items():
        assert np.array_equal(m, ref_m), cuts
        assert np.array_equal(c, ref_c), cuts
    # and the unfused result is right
    for t in range(T):
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        check_mask(ref_m[t, :, :W], int(ref_c[t]), m_ref, c_ref, maps["r"], TOL_F32)
    # R through a fused group [0..6] equals R through the unfused stages, bit for bit
    outs, _, _ = run_unfused_maps(ctx.h, K.KF_PREC_F32, fd, W)
    r = torch.empty((T, H, pitch16(W)), dtype=torch.float32, device=dev)
    K.kf_run_group(ctx.h, 0, 6, [fd], K.KF_DT_U8, [r], K.KF_DT_F32, W)
    assert torch.equal(r[:, :, :W], outs[6][0][:, :, :W])


@pytest.mark.parametrize("H,W", [(1, 1), (1, 7), (7, 1), (2, 3), (3, 2), (5, 5), (9, 127), (6, 128), (11, 129),
                                 (33, 4), (4, 33), (17, 300)])
def test_ragged_and_degenerate_frames(dev, H, W):
    T = 2
    fr = random_frames(T, H, W, H * 1000 + W)
    ctx = K.Context(0)
    fd = torch.from_numpy(fr).to(dev)
    for cuts in (0, 127, 0b0100100):
        ws_b = K.kf_workspace_bytes(ctx.h, cuts, W, H, T)
        ws = torch.empty(max(ws_b, 1), dtype=torch.uint8, device=dev)
        mask = torch.full((T, H, pitch16(W)), 9, dtype=torch.uint8, device=dev)
        counts = torch.zeros(T, dtype=torch.int32, device=dev)
        K.kf_run(ctx.h, cuts, fd, W, mask, counts, ws if ws_b else None)
        assert K.kf_device_error(ctx.h) == 0
        m = mask.cpu().numpy()
        assert np.all(m[:, :, W:] == 9), "columns past W must be untouched"
        for t in range(T):
            maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
            check_mask(m[t, :, :W], int(counts[t]), m_ref, c_ref, maps["r"], TOL_F32)


def test_zero_frames_is_a_no_op(dev):
    ctx = K.Context(0)
    fd = torch.zeros((0, 8, 16), dtype=torch.uint8, device=dev)
    mask = torch.zeros((0, 8, 16), dtype=torch.uint8, device=dev)
    counts = torch.zeros(1, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, 0, fd, 8, mask, counts, None)
    torch.cuda.synchronize()


@pytest.mark.parametrize("rows", [1, 2, 3, 7, 64, 1000])
def test_chunking_does_not_change_the_result(dev, rows):
    T, H, W = 2, 96, 200
    fr = frames_of(sv.VideoSpec(T=T, H=H, W=W, seed=13, n_blobs=10, n_patches=6))
    fd = torch.from_numpy(fr).to(dev)
    res = []
    for r in (200, rows):
        ctx = K.Context(0)
        K.kf_set_chunk_rows(ctx.h, r)
        r_map = torch.empty((T, H, pitch16(W)), dtype=torch.float32, device=dev)
        K.kf_run_group(ctx.h, 0, 6, [fd], K.KF_DT_U8, [r_map], K.KF_DT_F32, W)
        mask = torch.zeros((T, H, pitch16(W)), dtype=torch.uint8, device=dev)
        counts = torch.zeros(T, dtype=torch.int32, device=dev)
        K.kf_run(ctx.h, 0, fd, W, mask, counts, None)
        res.append((r_map.cpu(), mask.cpu(), counts.cpu()))
    assert torch.equal(res[0][0][:, :, :W], res[1][0][:, :, :W])
    assert torch.equal(res[0][1], res[1][1]) and torch.equal(res[0][2], res[1][2])


def test_fp16_maps_stay_within_2e_3(dev):
    """16-bit maps between every pair of stages: uint16 maps of stages 1-3 are exact,
    FP16 maps of stages 4-7 stay within 2e-3 normwise of the FP64 oracle."""
    T, H, W = 3, 192, 432
    fr = frames_of(sv.VideoSpec(T=T, H=H, W=W, seed=14))
    ctx = K.Context(0, precision=K.KF_PREC_F16)
    fd = torch.from_numpy(fr).to(dev)
    outs, mask, counts = run_unfused_maps(ctx.h, K.KF_PREC_F16, fd, W)
    worst = {}
    for t in range(T):
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        for s in range(7):
            scale = K.kf_map_scale(ctx.h, s)
            for c, key in enumerate(MAP_KEYS[s]):
                got = as_f64(outs[s][c][t, :, :W]) * scale
                err = normwise(got, maps[key])
                worst[key] = max(worst.get(key, 0.0), err)
                assert err <= (1e-12 if s <= 2 else TOL_F16), (s, key, err)
        check_mask(mask[t, :, :W].cpu().numpy(), int(counts[t]), m_ref, c_ref, maps["r"], TOL_F16)
    print("fp16 unfused normwise errors:", {k: f"{v:.2e}" for k, v in worst.items()})
    # every partition in FP16 stays within tolerance of the oracle
    for cuts in (0, 127, 0b1000000, 0b0010100):
        ws_b = K.kf_workspace_bytes(ctx.h, cuts, W, H, T)
        ws = torch.empty(max(ws_b, 1), dtype=torch.uint8, device=dev)
        m2 = torch.zeros((T, H, pitch16(W)), dtype=torch.uint8, device=dev)
        c2 = torch.zeros(T, dtype=torch.int32, device=dev)
        K.kf_run(ctx.h, cuts, fd, W, m2, c2, ws if ws_b else None)
        for t in range(T):
            maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy(), want_maps=True)
            check_mask(m2[t, :, :W].cpu().numpy(), int(c2[t]), m_ref, c_ref, maps["r"], TOL_F16)


def test_full_size_workload_on_sampled_frames(dev):
    """The 1000 x 800 x 600 volume in the benchmark's launch configuration; the oracle
    checks a sample of frames one by one."""
    spec = sv.HSDV_800x600x1000
    P = pitch16(spec.W)
    sample = [0, 1, 499, 998, 999]
    fr_s, _ = sv.generate(spec, pitch=P, frames=sample)
    full = torch.zeros((spec.T, spec.H, P), dtype=torch.uint8, device=dev)
    # the other frames are random content: only sampled frames are checked
    full.random_(0, 256)
    for i, t in enumerate(sample):
        full[t] = torch.from_numpy(fr_s[i]).to(dev)
    ctx = K.Context(0)
    cuts, _ = K.kf_plan(ctx.h, spec.W, spec.H, spec.T)
    assert cuts == 0
    mask = torch.zeros_like(full)
    counts = torch.zeros(spec.T, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, cuts, full, spec.W, mask, counts, None)
    assert K.kf_device_error(ctx.h) == 0
    for i, t in enumerate(sample):
        maps, m_ref, c_ref = oc.chain_frame(fr_s[i][:, :spec.W].copy())
        check_mask(mask[t, :, :spec.W].cpu().numpy(), int(counts[t]), m_ref, c_ref, maps["r"], TOL_F32)


def test_measured_planner_times_every_partition(dev):
    """kf_plan_measured: a median time for every candidate, the least one returned, the
    outputs those of a correct run; a workspace too small for some candidate is refused
    before any work."""
    T, H, W = 6, 96, 150
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=17, n_blobs=6, n_patches=4), pitch=pitch16(W))
    f = torch.from_numpy(fr).to(dev)
    ctx = K.Context(0)
    m_ref, c_ref = torch.zeros_like(f), torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, 0, f, W, m_ref, c_ref, None)
    ws = torch.empty(max(K.kf_workspace_bytes(ctx.h, c, W, H, T) for c in range(128)), dtype=torch.uint8, device=dev)
    mask, counts = torch.zeros_like(f), torch.zeros(T, dtype=torch.int32, device=dev)
    best, ms, all_ms = K.kf_plan_measured(ctx.h, f, W, mask, counts, ws, reps=3)
    assert 0 <= best < 128 and ms > 0 and np.all(all_ms > 0)
    assert all_ms[best] == ms and ms == all_ms.min()
    assert torch.equal(mask, m_ref) and torch.equal(counts, c_ref)
    best2, ms2, all2 = K.kf_plan_measured(ctx.h, f, W, mask, counts, ws, candidates=[127, 0, 8], reps=2)
    assert best2 in (127, 0, 8) and len(all2) == 3 and ms2 == all2.min()
    small = torch.empty(256, dtype=torch.uint8, device=dev)
    with pytest.raises(K.KfuseError) as e:
        K.kf_plan_measured(ctx.h, f, W, mask, counts, small, candidates=[0, 127], reps=1)
    assert e.value.status == K.KF_ENOMEM


@pytest.mark.parametrize("cuts", [0, 0b0000100, 0b0001000, 0b0010000, 127])
def test_fp16_tiles_match_the_oracle(dev, cuts):
    """KF_PREC_F16_TILES: 16-bit maps between groups, and FP16 row-pair sums of the box on
    chip in the groups that form the products and the response (here full fusion and
    the groups [4..8], [5..8]); masks and counts within the FP16 exemption rule."""
    T, H, W = 3, 150, 237
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=29, n_blobs=10, n_patches=6), pitch=pitch16(W))
    fd = torch.from_numpy(fr).to(dev)
    ctx = K.Context(0, precision=K.KF_PREC_F16_TILES)
    ws_b = K.kf_workspace_bytes(ctx.h, cuts, W, H, T)
    ws = torch.empty(max(ws_b, 1), dtype=torch.uint8, device=dev)
    mask = torch.zeros((T, H, pitch16(W)), dtype=torch.uint8, device=dev)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, cuts, fd, W, mask, counts, ws if ws_b else None)
    assert K.kf_device_error(ctx.h) == 0
    for t in range(T):
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy(), want_maps=True)
        check_mask(mask[t, :, :W].cpu().numpy(), int(counts[t]), m_ref, c_ref, maps["r"], TOL_F16)
    assert int(counts.sum()) > 0
