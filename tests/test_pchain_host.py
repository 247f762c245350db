"""Host-side checks of the paper's own chain (CPU only): the traffic model restated
plainly for every partition (tiles of 128 x 32 input, row halo = number of spatial
stages in the group, column halo one lane of 4), the planner's choice, workspace sizes,
and argument rejection on a host-only context."""
import itertools

import pytest

from paper_1509_04394_gb300 import kfuse as K


@pytest.fixture
def hctx():
    h = K.kf_create(-1)
    yield h
    K.kf_destroy(h)


def groups_of(cuts):
    a, out = 0, []
    for i in range(5):
        if i == 4 or (cuts >> i) & 1:
            out.append((a, i))
            a = i + 1
    return out


def expected_bytes(cuts, W, H, T):
    in_b = [4, 4, 4, 4, 4]   # input of stage k: RGBA (k = 0) or an FP32 map
    out_b = [4, 4, 4, 4, 1]  # output of stage k: FP32 map, or the u8 mask
    tot = 0.0
    for a, b in groups_of(cuts):
        halo = sum(1 for s in (2, 3) if a <= s <= b)
        hc = 4 if halo else 0  # tiles of 128 x 32 input; the column halo is one lane (4 columns)
        rf = 128 * 32 / ((128 - 2 * hc) * (32 - 2 * halo))
        tot += W * H * T * (in_b[a] * rf + out_b[b])
        if a <= 1 <= b:  # the chunked IIR recursion (chunks of 32 frames)
            nc = -(-T // 32)
            hw = W * H
            tot += (nc - 1) * 32 * hw * in_b[a] + (nc - 1) * hw * 4        # local end states
            tot += hw * in_b[a] + (nc - 1) * hw * 4 + nc * hw * 4          # carry
            tot += nc * hw * 4 * rf                                          # start states, with halo
    return tot + T * 4 * (1 + 3 * 16)


@pytest.mark.parametrize("cuts", range(16))
def test_traffic_model_of_every_partition(hctx, cuts):
    W, H, T = 1024, 1024, 1000
    assert K.kf_pc_traffic(hctx, cuts, W, H, T) == pytest.approx(expected_bytes(cuts, W, H, T), rel=1e-12)


def test_plan_is_full_fusion_and_orders_the_papers_partitions(hctx):
    for W, H in ((256, 256), (512, 512), (1024, 1024), (600, 800)):
        cuts, b = K.kf_pc_plan(hctx, W, H, 1000)
        assert cuts == 0 and b == pytest.approx(expected_bytes(0, W, H, 1000))
        full, two, none = (K.kf_pc_traffic(hctx, c, W, H, 1000) for c in (0, 0b0010, 0b1111))
        assert full < two < none
        assert min(K.kf_pc_traffic(hctx, c, W, H, 1000) for c in range(16)) == b


def test_workspace_sizes(hctx):
    T = 70  # three chunks of 32 frames
    plane = -(-(1024 * 512 * T * 4) // 256) * 256  # pitch round_up(1020, 8) = 1024
    state = -(-(3 * 512 * 1024 * 4) // 256) * 256
    slots = -(-(T * 32 * 49 * 4) // 256) * 256  # 32 partial copies of the 49 per-frame sums
    assert K.kf_pc_workspace_bytes(hctx, 0, 1020, 512, T) == state + slots
    assert K.kf_pc_workspace_bytes(hctx, 0b0010, 1020, 512, T) == state + slots + plane
    for c in (0b0011, 0b1111):
        assert K.kf_pc_workspace_bytes(hctx, c, 1020, 512, T) == state + slots + 2 * plane
    for a, b in [(0, 1), (1, 1), (1, 3)]:
        assert K.kf_pc_group_workspace_bytes(hctx, a, b, 1020, 512, T) == state
    assert K.kf_pc_group_workspace_bytes(hctx, 0, 4, 1020, 512, T) == state + slots
    for a, b in [(2, 4), (4, 4)]:
        assert K.kf_pc_group_workspace_bytes(hctx, a, b, 1020, 512, T) == slots
    for a, b in [(0, 0), (2, 3), (3, 3)]:
        assert K.kf_pc_group_workspace_bytes(hctx, a, b, 1020, 512, T) == 0


def test_argument_rejection(hctx):
    L = K._lib()
    with pytest.raises(K.KfuseError):
        K.kf_pc_traffic(hctx, 16, 8, 8, 1)
    with pytest.raises(K.KfuseError):
        K.kf_pc_traffic(hctx, 0, 0, 8, 1)
    v = K.kf_pc_video(0, 8, 8, 1, 8)
    assert L.kf_pc_run(hctx, 0, K.ctypes.byref(v), None, None, 0, None) == K.KF_EINVAL
    # region sums would pass 2^31: rejected before any launch
    big = K.kf_pc_video(16, 40000, 40000, 1, 40000)
    assert L.kf_pc_run_group(hctx, 1, 2, K.ctypes.byref(big), 16, 40000, 16, 40000, None, 256, 1 << 40,
                             None) == K.KF_EINVAL
    odd = K.kf_pc_video(16, 62, 32, 2, 62)  # pitch not a multiple of 4 pixels
    assert L.kf_pc_run(hctx, 0, K.ctypes.byref(odd), None, None, 0, None) == K.KF_EINVAL
    ok = K.kf_pc_video(16, 64, 32, 2, 64)
    assert L.kf_pc_run_group(hctx, 2, 3, K.ctypes.byref(ok), 16, 64, 16, 64, None, None, 0, None) == K.KF_ESTATE
    # a group holding the IIR filter without its chunk-state workspace
    assert L.kf_pc_run_group(hctx, 1, 2, K.ctypes.byref(ok), 16, 64, 16, 64, None, None, 0, None) == K.KF_EINVAL
    assert L.kf_pc_run_group(hctx, 1, 2, K.ctypes.byref(ok), 16, 64, 16, 64, None, 256, 16, None) == K.KF_ENOMEM
    assert L.kf_pc_kalman(hctx, 16, 5, 16, 16, 16, None) == K.KF_ESTATE
    assert L.kf_pc_kalman(hctx, 16, -1, 16, 16, 16, None) == K.KF_EINVAL
