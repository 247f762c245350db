"""Pins of the brute-force partitioner and traffic model (CPU only).

Golden values come from the paper: the four partitions of three kernels (Sec. VI),
the n(n+1)/2 candidate groups (Fig. 5), Transfer_serial = 2nBxyt (Sec. VI-D), the
data-utilisation ratio (Eq. 3) and the closed-form box of Eq. 6, also as the minimiser of
the traffic model itself; the unfused Harris chain's bytes per pixel and one fused
group's on-chip bytes counted by hand; feasibility requires every group to fit.
"""
import os

import numpy as np
import pytest

from oracle import partition as op

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_three_kernels_have_the_four_partitions_listed_in_the_paper():
    gold = set()
    for ln in _read("partitions_of_three_kernels.txt"):
        groups = tuple(tuple(int(k) - 1 for k in g.split()) for g in ln.split("|"))
        gold.add(tuple((g[0], g[-1]) for g in groups))
    got = {tuple(p) for p in op.all_partitions(3)}
    assert got == gold


def test_partition_and_candidate_group_counts():
    for ln in _read("counts.txt"):
        n, parts, groups = map(int, ln.split())
        assert len(op.all_partitions(n)) == parts
        cand = op.candidate_groups(n)
        assert len(cand) == len(set(cand)) == groups  # every contiguous range once
        assert all(0 <= a <= b < n for a, b in cand)
        # every partition covers each kernel exactly once (Fig. 5 constraint)
        for p in op.all_partitions(n):
            cover = np.zeros(n, dtype=int)
            for a, b in p:
                cover[a:b + 1] += 1
            assert np.all(cover == 1)


def test_serial_transfer_is_2nBxyt_for_point_stages():
    n = 5
    stages = [op.Stage(f"k{i}", 0, 0, 0, 1, 1) for i in range(n)]
    N, M, T, box = 256, 256, 1000, (32, 32, 8)
    B = N * M * T / (box[0] * box[1] * box[2])
    unfused = [(i, i) for i in range(n)]
    assert op.partition_cost(stages, unfused, N, M, T, box) == pytest.approx(
        2 * n * B * box[0] * box[1] * box[2])
    # fusing point stages leaves only the first read and the last write: 2Bxyt
    assert op.partition_cost(stages, [(0, n - 1)], N, M, T, box) == pytest.approx(
        2 * B * box[0] * box[1] * box[2])


def test_fused_halo_term_grows_with_the_summed_radius():
    stages = [op.Stage("a", 1, 1, 0, 1, 1), op.Stage("b", 2, 2, 0, 1, 1)]
    N, M, T, box = 64, 64, 4, (16, 16, 1)
    B = N * M * T / 256
    got = op.group_traffic(stages, 0, 1, N, M, T, box)
    assert got == pytest.approx(B * ((16 + 6) * (16 + 6) + 256))


def test_data_utilisation_eq3():
    assert op.data_utilisation((32, 32, 16), (0, 0, 0)) == 1.0
    assert op.data_utilisation((32, 32, 16), (1, 1, 1)) == pytest.approx(
        32 * 32 * 16 / (34 * 34 * 17))


@pytest.mark.parametrize("beta,dx,dt", [(48 * 1024, 1, 1), (96 * 1024, 2, 1), (20000, 3, 2)])
def test_eq6_is_the_minimiser_of_eq5(beta, dx, dt):
    # V = (x + 2 dx)^2 (t + dt) with x^2 t = beta (two-sided spatial, one-sided temporal)
    x_cf, t_cf = op.eq6_box(beta, dx, dt)
    xs = np.linspace(1.0, 200.0, 400001)
    V = (xs + 2 * dx) ** 2 * (beta / xs ** 2 + dt)
    x_num = xs[np.argmin(V)]
    assert x_cf == pytest.approx(x_num, rel=1e-3)
    assert t_cf == pytest.approx(beta / x_cf ** 2, rel=1e-12)


@pytest.mark.parametrize("beta,dx,dt", [(48 * 1024, 1, 1), (20000, 3, 2)])
def test_traffic_model_is_minimised_at_the_eq6_box(beta, dx, dt):
    # one spatio-temporal stage, no output bytes: at a fixed box volume beta the model's
    # traffic is (boxes = const / beta) x the box's input, so its minimum is Eq. 6's box
    st = [op.Stage("st", dx, dx, dt, 1, 0)]
    xs = np.linspace(2.0, 150.0, 60001)
    cost = [op.group_traffic(st, 0, 0, 512, 512, 64, (x, x, beta / x ** 2)) for x in xs]
    assert op.eq6_box(beta, dx, dt)[0] == pytest.approx(xs[int(np.argmin(cost))], rel=2e-3)


@pytest.mark.parametrize("e,total", [(4, 98), (2, 50)])
def test_unfused_harris_chain_bytes_per_pixel(e, total):
    # FP32 maps: reads 1 + 4 + 4 + 4 + 8 + 12 + 12 + 4 = 49, writes 4 + 4 + 4 + 8 + 12 + 12
    # + 4 + 1 = 49 (Sobel writes Ix and Iy, products and sums three maps, the mask one
    # byte); 16-bit maps: 25 + 25
    assert sum(s.in_bytes + s.out_bytes for s in op.harris_chain(e)) == total


def test_onchip_bytes_of_the_fused_harris_chain_by_hand():
    # halo 0+2+0+1+0+2+0+1 = 6 columns a side; rows held x bytes: convert 1 x 1, Gaussian-H
    # 1 x 4, Gaussian-V 5 x 4, Sobel 3 x 4, products 1 x 8, box 5 x 12, Harris 1 x 12,
    # NMS 3 x 4 = 129 bytes per column of the (116 + 12)-wide box, one frame
    assert op.group_onchip(op.harris_chain(4), 0, 7, (116, 64, 1)) == (116 + 12) * 129


def test_onchip_bytes_of_a_spatio_temporal_stage_by_hand():
    # rx = ry = 1, rt = 2, 4-byte input: (16 + 2) columns x (8 + 2) frames (the temporal
    # halo on the past side only) x 3 rows x 4 bytes
    st = [op.Stage("st", 1, 1, 2, 4, 1)]
    assert op.group_onchip(st, 0, 0, (16, 16, 8)) == 18 * 10 * 3 * 4


def test_a_partition_is_feasible_only_if_every_group_fits():
    st, box = op.harris_chain(4), (116, 64, 1)
    small, big = op.group_onchip(st, 0, 0, box), op.group_onchip(st, 1, 7, box)
    assert small < big
    assert op.feasible(st, [(0, 0), (1, 7)], box, big)
    assert not op.feasible(st, [(0, 0), (1, 7)], box, big - 1)


def test_brute_force_prefers_full_fusion_for_the_harris_chain_on_large_boxes():
    st = op.harris_chain(4)
    g, c = op.brute_force_best(st, 600, 800, 10, (116, 64, 1))
    assert g == [(0, 7)]
    unfused = op.partition_cost(st, [(i, i) for i in range(8)], 600, 800, 10, (116, 64, 1))
    assert unfused > 40 * c


def test_onchip_limit_forces_cuts():
    st = op.harris_chain(4)
    box = (116, 64, 1)
    full = op.group_onchip(st, 0, 7, box)
    g, _ = op.brute_force_best(st, 600, 800, 10, box, onchip_limit=full - 1)
    assert len(g) >= 2
    assert op.feasible(st, g, box, full - 1)


def _paper_chain():
    """The paper's K1..K5 (Table II / IV) as stages of the Sec. VI-D model: RGBA in (4
    bytes), float maps between stages, a byte mask out; K2 reads the previous frame's
    filtered value (one-sided temporal reach 1), K3 and K4 are 3x3 stencils."""
    return [op.Stage("gray", 0, 0, 0, 4, 4), op.Stage("iir", 0, 0, 1, 4, 4), op.Stage("gauss3", 1, 1, 0, 4, 4),
            op.Stage("gradient", 1, 1, 0, 4, 4), op.Stage("threshold", 0, 0, 0, 4, 1)]


def test_paper_chain_box_traffic_by_hand():
    st, N, M, T = _paper_chain(), 256, 256, 1000
    px = N * M * T

    def per_px(groups, box):
        return op.partition_cost(st, groups, N, M, T, box) / px
    none, two, full = [(i, i) for i in range(5)], [(0, 1), (2, 4)], [(0, 4)]
    # box [8, 8, 8]: halo reads (8 + 2 rx)(8 + 2 ry)(8 + rt) / 512 of the input bytes
    assert per_px(none, (8, 8, 8)) == pytest.approx((4 + 4) + (4 * 9 / 8 + 4) + 2 * (4 * 100 / 64 + 4) + (4 + 1))
    assert per_px(two, (8, 8, 8)) == pytest.approx((4 * 9 / 8 + 4) + (4 * 144 / 64 + 1))
    assert per_px(full, (8, 8, 8)) == pytest.approx(4 * 144 * 9 / (64 * 8) + 1)
    # fused traffic falls as the box grows (Fig. 12a); without halos No Fusion's would not
    # change (the paper's "constant"), with them it falls too, towards 2 reads + writes
    boxes = [(8, 8, 8), (16, 16, 8), (32, 32, 16), (64, 64, 32)]
    for groups in (two, full):
        seq = [per_px(groups, b) for b in boxes]
        assert all(a > b for a, b in zip(seq, seq[1:]))
    assert per_px(full, (64, 64, 32)) < per_px(two, (64, 64, 32)) < per_px(none, (64, 64, 32))
