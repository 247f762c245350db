"""Pins of the recompute-vs-store plan reference (CPU only): Sec. VI-D's serial and fused
transfer for a chain of point stages, a three-stage DAG worked by hand with and without
recomputing its first node, a 3x3 maximum's halo by hand, stores and members by their definitions, and the brute
force's minimum against every plan listed by hand."""
import pytest

from oracle import dag_plan as odp

AFF, ABS, PROD, STEN, MAX3 = 1, 2, 3, 4, 5
TILE = odp.TX * odp.TY


def chain(n):
    return [(AFF, i - 1, -1, 0, 1.5, 0.1) for i in range(1, n + 1)]


@pytest.mark.parametrize("n", [1, 2, 5])
def test_point_chain_serial_and_fused(n):
    W, H, T = 64, 32, 3
    rows = chain(n)
    allcut = (1 << (n - 1)) - 1
    # every stage stored and read back: frame 1 B in, then 4 B out and 4 B in per cut
    assert odp.plan_traffic(rows, allcut, set(), W, H, T) == W * H * T * (1 + 4 + (n - 1) * 8)
    assert odp.plan_traffic(rows, 0, set(), W, H, T) == W * H * T * (1 + 4)


def test_hand_worked_recompute():
    # 1 = affine(frame), 2 = 3x3 binomial(1), 3 = product(2, 1); cut between 2 and 3
    rows = [(AFF, 0, -1, 0, 2.0, 0.0), (STEN, 1, -1, 1, 0, 0), (PROD, 2, 1, 0, 0, 0)]
    # stored 1: group [1,2] reads the frame with halo 1, stores 1 and 2; group [3] reads both
    g1 = (odp.TX + 2) * (odp.TY + 2) * 1 + 2 * TILE * 4
    g2 = 2 * TILE * 4 + TILE * 4
    assert odp.plan_traffic(rows, 0b10, set(), odp.TX, odp.TY, 1) == g1 + g2
    # node 1 recomputed by group [3] from the frame (halo 0) instead of stored and read
    g1x = (odp.TX + 2) * (odp.TY + 2) * 1 + TILE * 4
    g2x = TILE * 1 + TILE * 4 + TILE * 4
    assert odp.plan_traffic(rows, 0b10, {1}, odp.TX, odp.TY, 1) == g1x + g2x
    assert odp.group_members(rows, 3, 3, {1}) == {1, 3}
    assert odp.stored(rows, 1, 2, {1}, 1) is False and odp.stored(rows, 1, 2, {1}, 2) is True
    assert odp.stored(rows, 1, 2, set(), 1) is True
    # the output is never inlined; an inlined node only later groups need is dropped from
    # its own range (node 2 here) and recomputed where it is read
    assert not odp.valid(rows, 0, {3})
    assert odp.group_members(rows, 1, 2, {2}) == {1}
    assert odp.group_members(rows, 3, 3, {2}) == {2, 3}


def test_hand_worked_max3():
    # 1 = 3x3 max(frame), 2 = affine(1): the max reads the frame with a halo of 1
    rows = [(MAX3, 0, -1, 1, 0, 0), (AFF, 1, -1, 0, 1.0, 0.0)]
    fused = (odp.TX + 2) * (odp.TY + 2) * 1 + TILE * 4
    assert odp.plan_traffic(rows, 0, set(), odp.TX, odp.TY, 1) == fused
    assert odp.plan_traffic(rows, 1, set(), odp.TX, odp.TY, 1) == fused + TILE * 4 * 2
    # frame slot, node 1's slot; node 2 reuses the frame's: 2 slots of (TX + 2)(TY + 2)
    assert odp.onchip_bytes(rows, 1, 2, set()) == 2 * (odp.TX + 2) * (odp.TY + 2) * 4


def test_inlined_node_not_needed_by_its_range_is_not_computed_there():
    # 1 = affine(frame); 2 = affine(frame); 3 = product(1, 2); cut after 1 and after 2
    rows = [(AFF, 0, -1, 0, 1.0, 0.0), (AFF, 0, -1, 0, 3.0, 0.0), (PROD, 1, 2, 0, 0, 0)]
    assert odp.group_members(rows, 1, 1, {1}) == set()
    assert odp.group_members(rows, 3, 3, {1, 2}) == {1, 2, 3}
    t = odp.plan_traffic(rows, 0b11, {1, 2}, odp.TX, odp.TY, 1)
    # groups [1] and [2] compute nothing; group [3] reads the frame once and stores 3
    assert t == TILE * 1 + TILE * 4


def test_inlined_nodes_are_recomputed_through_inlined_inputs():
    # 1 = affine(frame), 2 = affine(1), 3 = affine(2), a cut after every stage, 1 and 2
    # inlined: group [3] recomputes 2 and, through it, 1 from the frame
    rows = chain(3)
    assert odp.group_members(rows, 3, 3, {1, 2}) == {1, 2, 3}
    assert odp.plan_traffic(rows, 0b11, {1, 2}, odp.TX, odp.TY, 1) == TILE * 1 + TILE * 4


def test_brute_force_is_the_minimum_over_listed_plans():
    rows = [(AFF, 0, -1, 0, 2.0, 0.0), (STEN, 1, -1, 2, 0, 0), (MAX3, 2, -1, 1, 0, 0), (PROD, 3, 1, 0, 0, 0)]
    W, H, T = 64, 32, 1
    lim = 14000
    feas = lambda r, a, b, X: odp.onchip_bytes(r, a, b, X) <= lim  # noqa: E731
    best = odp.brute_force(rows, W, H, T, feas)
    plans = [(c, X) for c in range(8) for X in (set(), {1}, {2}, {3}, {1, 2}, {1, 3}, {2, 3}, {1, 2, 3})]
    costs = [odp.plan_traffic(rows, c, X, W, H, T) for c, X in plans
             if all(feas(rows, a, b, X) for a, b in odp.ranges(4, c))]
    assert best[0] == min(costs)


def test_onchip_bytes_by_hand():
    # one 3x3 binomial of the frame: frame tile with halo 1 and the output tile, both in
    # slots of (TX + 2)(TY + 2) floats
    rows = [(STEN, 0, -1, 1, 0, 0)]
    assert odp.onchip_bytes(rows, 1, 1, set()) == 2 * (odp.TX + 2) * (odp.TY + 2) * 4
    # a chain of two point stages: the frame's slot is freed once node 1 has taken its
    # own, node 2 then reuses it -> 2 slots of TX * TY floats
    rows = chain(2)
    assert odp.onchip_bytes(rows, 1, 2, set()) == 2 * TILE * 4
