"""GPU parity of the tracking stages (corner selection + one Lucas-Kanade step).

The CUDA path ranks corners by its FP32 response, the oracle by FP64: the selected sets
must agree except for corners whose oracle response is within the FP32 tolerance of the
K-th response (where the two precisions may order them differently). Velocities of the
common points agree within 2e-3 px/frame (relative to the window's conditioning), status
flags agree away from the singularity threshold, and slow checker patches of the
synthetic video are tracked within 0.25 px/frame of the generator's motion.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import chain as oc  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import video as sv  # noqa: E402
from tests._parity import TOL_F16, TOL_F32, check_mask  # noqa: E402
from tests._track_parity import check_frame  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


def run_track(dev, fr, W, Kp=256, precision=None):
    T, H, P = fr.shape
    ctx = K.Context(0) if precision is None else K.Context(0, precision=precision)
    frames = torch.from_numpy(fr).to(dev)
    mask = torch.zeros_like(frames)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    n = torch.full((T,), -1, dtype=torch.int32, device=dev)
    idx = torch.full((T, Kp), -1, dtype=torch.int32, device=dev)
    u = torch.zeros((T, Kp), dtype=torch.float32, device=dev)
    v = torch.zeros((T, Kp), dtype=torch.float32, device=dev)
    st = torch.full((T, Kp), -1, dtype=torch.int32, device=dev)
    ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_track(ctx.h, frames, W, mask, counts, Kp, n, idx, u, v, st, ws)
    assert K.kf_device_error(ctx.h) == 0
    out = dict(mask=mask.cpu().numpy(), counts=counts.cpu().numpy(), n=n.cpu().numpy(), idx=idx.cpu().numpy(),
               u=u.cpu().numpy(), v=v.cpu().numpy(), st=st.cpu().numpy())
    # the chain part equals kf_run's full fusion bit for bit
    m2 = torch.zeros_like(frames)
    c2 = torch.zeros(T, dtype=torch.int32, device=dev)
    K.kf_run(ctx.h, 0, frames, W, m2, c2, None)
    assert np.array_equal(out["mask"], m2.cpu().numpy()) and np.array_equal(out["counts"], c2.cpu().numpy())
    return out


@pytest.mark.parametrize("shape,Kp", [((4, 192, 432), 256), ((3, 77, 130), 64), ((3, 40, 50), 1024), ((3, 96, 150), 1),
                                      ((5, 120, 600), 256)])
def test_tracking_matches_the_oracle(dev, shape, Kp):
    T, H, W = shape
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=41, n_blobs=12, n_patches=8), pitch=sv.pitch_for(W))
    out = run_track(dev, fr, W, Kp)
    assert out["n"][0] == 0
    checked = sum(check_frame(fr, t, W, out, Kp) for t in range(1, T))
    assert checked >= min(Kp, 5)


def test_full_size_tracking_in_the_benchmark_configuration(dev):
    """The benchmark's timed step itself: kf_track over the whole 1000 x 800 x 600 volume
    (seed 3, 64 blobs, 32 patches; 256 points per frame) in the launch configuration the
    benchmark times (the chain with corner lists, then selection and LK). The oracle checks
    sampled frame pairs one by one: masks and counts under the exemption rule, the
    selected points up to FP32 near-ties at the K-th response, velocities within the
    conditioning-scaled tolerance."""
    spec = sv.HSDV_800x600x1000
    W = spec.W
    fr, _ = sv.generate(spec, pitch=sv.pitch_for(W))
    out = run_track(dev, fr, W, 256)
    assert out["n"][0] == 0
    checked = 0
    for t in (1, 2, 499, 998, 999):
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        check_mask(out["mask"][t, :, :W], int(out["counts"][t]), m_ref, c_ref, maps["r"], TOL_F32)
        assert out["n"][t] == min(256, int(out["counts"][t]))
        checked += check_frame(fr, t, W, out, 256)
    assert checked >= 5 * 200


@pytest.mark.parametrize("shape,sample", [((5, 120, 600), (1, 2, 3, 4)), ((1000, 800, 600), (1, 2, 499, 998, 999))])
def test_fp16_form_of_the_tracking_step(dev, shape, sample):
    """The FP16-tile form (KF_PREC_F16_TILES): the fused chain keeps the box's row-pair
    sums in FP16 on chip; masks and counts within the FP16 exemption rule (2e-3 of the
    frame's largest response), selected points up to near-ties or exempt corner decisions
    within the same tolerance, velocities by the FP32 rule (LK reads the frames, not the
    response). The full size is the
    benchmark's volume, checked on sampled frame pairs."""
    T, H, W = shape
    if T == 1000:
        spec = sv.HSDV_800x600x1000
        fr, _ = sv.generate(spec, pitch=sv.pitch_for(W))
    else:
        fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=43, n_blobs=12, n_patches=8), pitch=sv.pitch_for(W))
    out = run_track(dev, fr, W, 256, precision=K.KF_PREC_F16_TILES)
    assert out["n"][0] == 0
    checked = 0
    for t in sample:
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        check_mask(out["mask"][t, :, :W], int(out["counts"][t]), m_ref, c_ref, maps["r"], TOL_F16)
        assert out["n"][t] == min(256, int(out["counts"][t]))
        checked += check_frame(fr, t, W, out, 256, tol=TOL_F16, exempt_corners=True)
    assert checked >= len(sample) * 150


@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (5, 7), (12, 12), (9, 30), (30, 9), (13, 13)])
def test_tracking_on_frames_smaller_than_the_lk_window(dev, H, W):
    """Frames no larger than LK's 13 x 13 input patch: every point takes the clamped path
    (half-warp 9 x 9 grids with every frame access clamped); masks, counts, points and
    velocities against the oracle."""
    rng = np.random.default_rng(H * 100 + W)
    T, Kp = 4, 16
    fr = np.zeros((T, H, sv.pitch_for(W)), dtype=np.uint8)
    base = rng.integers(0, 256, (H, W), dtype=np.uint8)
    for t in range(T):  # a slowly drifting texture, so consecutive frames are related
        fr[t, :, :W] = np.roll(base, t % 2, axis=1) // 2 + rng.integers(0, 64, (H, W), dtype=np.uint8)
    out = run_track(dev, fr, W, Kp)
    assert out["n"][0] == 0
    for t in range(1, T):
        maps, m_ref, c_ref = oc.chain_frame(fr[t][:, :W].copy())
        check_mask(out["mask"][t, :, :W], int(out["counts"][t]), m_ref, c_ref, maps["r"], TOL_F32)
        check_frame(fr, t, W, out, Kp)


def test_constant_video_has_no_points_and_a_single_frame_has_no_tracks(dev):
    fr = np.full((3, 40, 64), 90, dtype=np.uint8)
    out = run_track(dev, fr, 64)
    assert out["counts"].tolist() == [0, 0, 0] and out["n"].tolist() == [0, 0, 0]
    fr1, _ = sv.generate(sv.VideoSpec(T=1, H=64, W=80, seed=3, n_blobs=6, n_patches=4), pitch=80)
    out1 = run_track(dev, fr1, 80)
    assert out1["n"].tolist() == [0] and out1["counts"][0] > 0


def test_slow_checker_patches_are_tracked_to_their_true_motion(dev):
    spec = sv.VideoSpec(T=6, H=400, W=300, seed=7, n_blobs=16, n_patches=16)
    fr, sc = sv.generate(spec, pitch=sv.pitch_for(spec.W))
    out = run_track(dev, fr, spec.W)
    errs = []
    for t in range(1, spec.T):
        n = int(out["n"][t])
        idx = out["idx"][t, :n]
        py, px = idx // spec.W, idx % spec.W
        X, Y = sc.position(t)
        for i in range(n):
            if out["st"][t, i] or not (8 <= px[i] < spec.W - 8 and 8 <= py[i] < spec.H - 8):
                continue
            for o in np.nonzero(sc.kind == 1)[0]:
                dx, dy = (px[i] - X[o]) % spec.W, (py[i] - Y[o]) % spec.H
                if 3 <= dx <= 13 and 3 <= dy <= 13 and np.hypot(sc.vx[o], sc.vy[o]) < 1.0:
                    errs.append(np.hypot(out["u"][t, i] - sc.vx[o], out["v"][t, i] - sc.vy[o]))
    assert len(errs) >= 30
    assert np.median(errs) <= 0.25


def kth_bucket(frame, W, Kp):
    """(candidates, keys in the FP32 exponent bucket of the Kp-th strongest) of one frame,
    from the oracle's responses: which of the selection's paths the frame takes."""
    maps, m, _ = oc.chain_frame(frame[:, :W].copy())
    r = np.sort(maps["r"].ravel()[np.flatnonzero(m.ravel())].astype(np.float32))[::-1]
    if len(r) <= Kp:
        return len(r), 0
    e = r.view(np.uint32) >> 23
    return len(r), int(np.sum(e == e[Kp - 1]))


@pytest.mark.parametrize("H,W,Kp", [(480, 640, 256), (720, 960, 1024), (720, 960, 7)])
def test_selection_with_many_candidates(dev, H, W, Kp):
    """Noise frames: about 3% of pixels are corner candidates, so the 480 x 640 frames'
    lists (~9k keys) are selected from shared memory and the 720 x 960 frames' (~21k
    keys) from global memory; at K = 1024 the K-th key's exponent bucket holds more keys
    than the 2048 the selection gathers on chip, so its digits are found over all keys."""
    rng = np.random.default_rng(H + Kp)
    fr = rng.integers(0, 256, (3, H, W), dtype=np.uint8)
    out = run_track(dev, fr, W, Kp)
    assert out["counts"][1] > (10240 if H == 720 else 5000)
    if Kp == 1024:
        assert kth_bucket(fr[1], W, Kp)[1] > 2048
    checked = sum(check_frame(fr, t, W, out, Kp) for t in range(1, 3))
    assert checked >= min(Kp, 5)


@pytest.mark.parametrize("Kp", [256, 1024])
def test_selection_when_the_kth_bucket_holds_every_key(dev, Kp):
    """A moving checkerboard: thousands of corners of one response, all in the K-th key's
    exponent bucket (more than the selection gathers on chip) while the frame's keys fit
    in shared memory; the raster index decides among equal responses."""
    T, H, W, sq = 3, 480, 640, 16
    fr = np.zeros((T, H, sv.pitch_for(W)), np.uint8)
    y, x = np.mgrid[0:H, 0:W]
    for t in range(T):
        fr[t, :, :W] = (((x + t) // sq + y // sq) % 2 * 200 + 20).astype(np.uint8)
    n, in_bucket = kth_bucket(fr[1], W, Kp)
    assert n <= 10240 and in_bucket > 2048
    out = run_track(dev, fr, W, Kp)
    checked = sum(check_frame(fr, t, W, out, Kp) for t in range(1, T))
    assert checked >= 5


def test_step_is_the_same_at_every_tile_height_and_the_tuner_keeps_the_fastest(dev):
    """kf_track's chain launch takes its jobs by SM kind from counters in the workspace:
    whatever the tile height (so the job count and the mix of kinds per wave), the step
    gives the same masks, counts and tracks; kf_tune_track_rows returns one of its
    candidates and leaves the context on it."""
    T, H, W, Kp = 6, 150, 300, 32
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=17, n_blobs=10, n_patches=6), pitch=sv.pitch_for(W))
    ctx = K.Context(0)
    frames = torch.from_numpy(fr).to(dev)
    mask = torch.zeros_like(frames)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    n = torch.zeros(T, dtype=torch.int32, device=dev)
    idx = torch.zeros((T, Kp), dtype=torch.int32, device=dev)
    u, v = torch.zeros((T, Kp), device=dev), torch.zeros((T, Kp), device=dev)
    st = torch.zeros((T, Kp), dtype=torch.int32, device=dev)
    ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
    ref = None
    for rows in (16, 48, 200, 7):
        K.kf_set_chunk_rows(ctx.h, rows)
        mask.fill_(3)
        idx.fill_(-2)
        K.kf_track(ctx.h, frames, W, mask, counts, Kp, n, idx, u, v, st, ws)
        got = [t.cpu().clone() for t in (mask, counts, n, idx, u, v, st)]
        assert K.kf_device_error(ctx.h) == 0
        if ref is None:
            ref = got
        else:
            for a, b in zip(got, ref):
                assert torch.equal(a, b), rows
    best, ms = K.kf_tune_track_rows(ctx.h, frames, W, mask, counts, Kp, n, idx, u, v, st, ws, [24, 64, 160], reps=2)
    assert best in (24, 64, 160) and ms > 0
    K.kf_track(ctx.h, frames, W, mask, counts, Kp, n, idx, u, v, st, ws)
    for a, b in zip([t.cpu() for t in (mask, counts, n, idx, u, v, st)], ref):
        assert torch.equal(a, b)


def test_kernel_timing_counts_every_launch(dev):
    """With timing on, kf_track records one event pair per kernel it launches (the chain
    with corner lists, selection, LK) and kf_run one per fused group; the record clears."""
    fr, _ = sv.generate(sv.VideoSpec(T=3, H=96, W=160, seed=5, n_blobs=6, n_patches=4), pitch=sv.pitch_for(160))
    T, H, P = fr.shape
    ctx = K.Context(0)
    frames = torch.from_numpy(fr).to(dev)
    mask = torch.zeros_like(frames)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    n = torch.zeros(T, dtype=torch.int32, device=dev)
    idx = torch.zeros((T, 16), dtype=torch.int32, device=dev)
    u, v = torch.zeros((T, 16), device=dev), torch.zeros((T, 16), device=dev)
    st = torch.zeros((T, 16), dtype=torch.int32, device=dev)
    ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, 160, H, T), dtype=torch.uint8, device=dev)
    K.kf_track(ctx.h, frames, 160, mask, counts, 16, n, idx, u, v, st, ws)  # untimed
    K.kf_set_kernel_timing(ctx.h, True)
    for _ in range(2):
        K.kf_track(ctx.h, frames, 160, mask, counts, 16, n, idx, u, v, st, ws)
    cuts = 0b1000100  # three groups
    wsr = torch.empty(K.kf_workspace_bytes(ctx.h, cuts, 160, H, T), dtype=torch.uint8, device=dev)
    K.kf_run(ctx.h, cuts, frames, 160, mask, counts, wsr)
    kt = K.kf_kernel_times(ctx.h)
    assert {k: c for k, (c, _) in kt.items() if c} == {"group": 3, "chain_corners": 2, "select": 2, "lk": 2}
    assert all(ms > 0 for c, ms in kt.values() if c)
    assert all(c == 0 for c, _ in K.kf_kernel_times(ctx.h).values())
    K.kf_set_kernel_timing(ctx.h, False)
    K.kf_track(ctx.h, frames, 160, mask, counts, 16, n, idx, u, v, st, ws)
    assert all(c == 0 for c, _ in K.kf_kernel_times(ctx.h).values())


@pytest.mark.parametrize("chunk", [1, 3, 7, 100])
def test_host_pipelined_call_equals_kf_track(dev, chunk):
    """kf_track_host (host frames in, host results out, chunks overlapped on copy
    streams) gives what kf_track gives, bit for bit, in host and device buffers."""
    T, H, W, Kp = 9, 80, 150, 32
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=8, n_blobs=8, n_patches=6), pitch=sv.pitch_for(W))
    ref = run_track(dev, fr, W, Kp)
    ctx = K.Context(0)
    P = fr.shape[2]

    def bufs(device, pin):
        d = dict(frames=torch.zeros((T, H, P), dtype=torch.uint8, device=device),
                 mask=torch.full((T, H, P), 5, dtype=torch.uint8, device=device),
                 counts=torch.full((T,), -1, dtype=torch.int32, device=device),
                 n_points=torch.full((T,), -1, dtype=torch.int32, device=device),
                 idx=torch.full((T, Kp), -1, dtype=torch.int32, device=device),
                 u=torch.zeros((T, Kp), dtype=torch.float32, device=device),
                 v=torch.zeros((T, Kp), dtype=torch.float32, device=device),
                 status=torch.full((T, Kp), -1, dtype=torch.int32, device=device))
        return {k: t.pin_memory() for k, t in d.items()} if pin else d
    host, devb = bufs("cpu", True), bufs(dev, False)
    host["frames"].copy_(torch.from_numpy(fr))
    ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_track_host(ctx.h, host, devb, W, Kp, ws, chunk=chunk, mask_format=K.KF_MASK_BYTES)
    torch.cuda.synchronize()
    assert K.kf_device_error(ctx.h) == 0
    names = dict(mask="mask", counts="counts", n_points="n", idx="idx", u="u", v="v", status="st")
    for k, r in names.items():
        got, exp = host[k].numpy(), ref[r]
        if k == "mask":  # the pitch padding is not written by either call
            got, exp = got[..., :W], exp[..., :W]
        assert np.array_equal(got, exp), k
        assert np.array_equal(host[k].numpy(), devb[k].cpu().numpy()), k


def test_host_call_timeline_and_chunk_tile_height(dev):
    """With timing on, kf_track_host records each chunk's copy in, chain, mask packing and
    copy out, two selections and two LK steps (the frames up to the first chunk end at or
    past T/2, then the rest) and the six copies of the counts and tracks; the timeline
    puts each chunk's chain after its copy in, the first tracking after the chains of its
    frames and the second after every chain. Its results do not depend on the tile height
    of the chunk launches (kf_set_host_chunk_rows)."""
    T, H, W, Kp = 9, 80, 150, 16
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=12, n_blobs=8, n_patches=6), pitch=sv.pitch_for(W))
    ctx = K.Context(0)
    P = fr.shape[2]
    S = ((W * H + 7) // 8 + 15) // 16 * 16

    def run(rows, timing):
        devb = dict(frames=torch.zeros((T, H, P), dtype=torch.uint8, device=dev),
                    mask=torch.zeros((T, H, P), dtype=torch.uint8, device=dev),
                    counts=torch.zeros(T, dtype=torch.int32, device=dev),
                    n_points=torch.zeros(T, dtype=torch.int32, device=dev),
                    idx=torch.zeros((T, Kp), dtype=torch.int32, device=dev), u=torch.zeros((T, Kp), device=dev),
                    v=torch.zeros((T, Kp), device=dev), status=torch.zeros((T, Kp), dtype=torch.int32, device=dev))
        host = {k: torch.empty_like(t, device="cpu").pin_memory() for k, t in devb.items()}
        host["mask"] = torch.zeros((T, S), dtype=torch.uint8).pin_memory()
        host["frames"].copy_(torch.from_numpy(fr))
        ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
        K.kf_set_host_chunk_rows(ctx.h, rows)
        K.kf_set_kernel_timing(ctx.h, timing)
        K.kf_track_host(ctx.h, host, devb, W, Kp, ws, chunk=3, mask_format=K.KF_MASK_BITS)
        torch.cuda.synchronize()
        tl = K.kf_kernel_timeline(ctx.h) if timing else []
        K.kf_set_kernel_timing(ctx.h, False)
        assert K.kf_device_error(ctx.h) == 0
        return {k: t.numpy().copy() for k, t in host.items() if k != "frames"}, tl

    ref, _ = run(0, False)
    got, tl = run(8, True)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    kinds = [k for k, _, _ in tl]
    n_chunks = kinds.count("copy_in")
    for k in ("chain_corners", "pack"):
        assert kinds.count(k) == n_chunks, k
    # 9 frames in chunks of 3: [0, 1), [1, 4), [4, 7), [7, 8), [8, 9); the first tracking
    # covers [0, 4), after the first two chains
    assert n_chunks == 5
    assert kinds.count("select") == 2 and kinds.count("lk") == 2
    assert kinds.count("copy_out") == n_chunks + 6
    assert all(0.0 <= a <= b for _, a, b in tl)
    ins = [(a, b) for k, a, b in tl if k == "copy_in"]
    chains = [(a, b) for k, a, b in tl if k == "chain_corners"]
    assert all(c[0] >= i[1] for i, c in zip(ins, chains))
    sel = [a for k, a, _ in tl if k == "select"]
    assert sel[0] >= max(b for _, b in chains[:2])
    assert sel[1] >= max(b for _, b in chains)
    assert K.kf_kernel_timeline(ctx.h) == []
    with pytest.raises(K.KfuseError):
        K.kf_set_host_chunk_rows(ctx.h, -1)


@pytest.mark.parametrize("W,chunk", [(150, 4), (600, 3), (37, 100)])
def test_host_call_with_bit_packed_masks(dev, W, chunk):
    """KF_MASK_BITS: the host receives each frame's mask as H * W bits in raster order
    (LSB first), packed on the device and copied out; the rest as with bytes."""
    T, H, Kp = 7, 40, 16
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=9, n_blobs=6, n_patches=4), pitch=sv.pitch_for(W))
    ref = run_track(dev, fr, W, Kp)
    ctx = K.Context(0)
    P = fr.shape[2]
    S = ((W * H + 7) // 8 + 15) // 16 * 16
    devb = dict(frames=torch.zeros((T, H, P), dtype=torch.uint8, device=dev),
                mask=torch.zeros((T, H, P), dtype=torch.uint8, device=dev),
                counts=torch.zeros(T, dtype=torch.int32, device=dev),
                n_points=torch.full((T,), -1, dtype=torch.int32, device=dev),
                idx=torch.full((T, Kp), -1, dtype=torch.int32, device=dev), u=torch.zeros((T, Kp), device=dev),
                v=torch.zeros((T, Kp), device=dev), status=torch.full((T, Kp), -1, dtype=torch.int32, device=dev))
    host = {k: torch.empty_like(t, device="cpu").pin_memory() for k, t in devb.items()}
    host["mask"] = torch.full((T, S), 0xAB, dtype=torch.uint8).pin_memory()
    host["frames"].copy_(torch.from_numpy(fr))
    ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
    K.kf_track_host(ctx.h, host, devb, W, Kp, ws, chunk=chunk, mask_format=K.KF_MASK_BITS)
    torch.cuda.synchronize()
    assert K.kf_device_error(ctx.h) == 0
    exp = np.packbits(ref["mask"][..., :W].reshape(T, -1), axis=1, bitorder="little")
    got = host["mask"].numpy()
    nbytes = (W * H + 7) // 8
    np.testing.assert_array_equal(got[:, :nbytes], exp)
    words = (nbytes + 3) // 4 * 4
    assert (got[:, nbytes:words] == 0).all() and (got[:, words:] == 0xAB).all()
    for k, r in dict(counts="counts", n_points="n", idx="idx", u="u", v="v", status="st").items():
        assert np.array_equal(host[k].numpy(), ref[r]), k
    # a pageable host mask gets the same packed mask (the copies are then synchronous)
    host["mask"] = torch.zeros((T, S), dtype=torch.uint8)
    K.kf_track_host(ctx.h, host, devb, W, Kp, ws, chunk=chunk, mask_format=K.KF_MASK_BITS)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host["mask"].numpy()[:, :nbytes], exp)


def test_host_call_rejects_bad_arguments_before_any_work(dev):
    T, H, W, Kp = 3, 32, 64, 8
    P = sv.pitch_for(W)
    ctx = K.Context(0)
    devb = dict(frames=torch.zeros((T, H, P), dtype=torch.uint8, device=dev),
                mask=torch.zeros((T, H, P), dtype=torch.uint8, device=dev),
                counts=torch.zeros(T, dtype=torch.int32, device=dev), n_points=torch.zeros(T, dtype=torch.int32, device=dev),
                idx=torch.zeros((T, Kp), dtype=torch.int32, device=dev), u=torch.zeros((T, Kp), device=dev),
                v=torch.zeros((T, Kp), device=dev), status=torch.zeros((T, Kp), dtype=torch.int32, device=dev))
    host = {k: torch.empty_like(t, device="cpu").pin_memory() for k, t in devb.items()}
    ws = torch.empty(K.kf_track_workspace_bytes(ctx.h, W, H, T), dtype=torch.uint8, device=dev)
    with pytest.raises(K.KfuseError):  # unknown mask format
        K.kf_track_host(ctx.h, host, devb, W, Kp, ws, chunk=2, mask_format=7)
    with pytest.raises(K.KfuseError):  # empty chunks
        K.kf_track_host(ctx.h, host, devb, W, Kp, ws, chunk=0)
    packed = dict(host, mask=torch.zeros((T, 8), dtype=torch.uint8).pin_memory())  # < ceil(W H / 8) bytes a frame
    with pytest.raises(K.KfuseError):
        K.kf_track_host(ctx.h, packed, devb, W, Kp, ws, chunk=2, mask_format=K.KF_MASK_BITS)
    torch.cuda.synchronize()
    assert K.kf_device_error(ctx.h) == 0
