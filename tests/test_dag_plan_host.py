"""Recompute-vs-store plans of kernel DAGs on the host (CPU only; the library loads
without a GPU): traffic and on-chip bytes of plans with inlined nodes against the
reference, the planner against brute force under on-chip limits, never worse than the
best contiguous partition, the learned-cost form, and argument checks."""
import random

import numpy as np
import pytest

from oracle import dag_plan as odp
from paper_1509_04394_gb300 import build as kbuild
from paper_1509_04394_gb300 import kfuse as K
from synth import dags as sd

W, H, T = 1920, 1080, 4


@pytest.fixture(scope="module")
def ctx():
    kbuild.build()
    c = K.kf_create(-1)
    yield c
    K.kf_destroy(c)


def test_plan_traffic_and_onchip_equal_the_reference(ctx):
    rng = random.Random(3)
    for seed in range(4000, 4012):
        rows = sd.to_array(sd.random_dag(seed, 5, 11))
        n = len(rows)
        dag = K.kf_dag_create(ctx, rows)
        for _ in range(12):
            cuts, xm = rng.randrange(1 << (n - 1)), rng.randrange(1 << (n - 1))
            X = {j + 1 for j in range(n - 1) if xm >> j & 1}
            t, m = K.kf_dag_xplan_traffic(dag, cuts, xm, W, H, T)
            assert t == pytest.approx(odp.plan_traffic(rows, cuts, X, W, H, T), rel=1e-12)
            assert m == max(odp.onchip_bytes(rows, a, b, X) for a, b in odp.ranges(n, cuts))
        # no inlining: the contiguous partition's traffic, group by group
        cuts = rng.randrange(1 << (n - 1))
        exp = sum(K.kf_dag_group_info(dag, a - 1, b - 1, W, H, T)[2] for a, b in odp.ranges(n, cuts))
        assert K.kf_dag_xplan_traffic(dag, cuts, 0, W, H, T)[0] == pytest.approx(exp, rel=1e-12)
        K.kf_dag_destroy(dag)


@pytest.mark.parametrize("seed", [4100, 4103, 4107, 4111, 4117])
@pytest.mark.parametrize("limit", [7000, 12000, 40000])
def test_planner_equals_brute_force(ctx, seed, limit):
    rows = sd.to_array(sd.random_dag(seed, 5, 6))
    dag = K.kf_dag_create(ctx, rows)
    Wp, Hp, Tp = 64, 32, 2
    bf = odp.brute_force(rows, Wp, Hp, Tp, feasible=lambda r, a, b, X: odp.onchip_bytes(r, a, b, X) <= limit)
    if bf is None:
        with pytest.raises(K.KfuseError):
            K.kf_dag_plan_recompute(dag, Wp, Hp, Tp, limit)
    else:
        cuts, xm, cost = K.kf_dag_plan_recompute(dag, Wp, Hp, Tp, limit)
        assert cost == pytest.approx(bf[0], rel=1e-12)
        X = {j + 1 for j in range(len(rows) - 1) if xm >> j & 1}
        assert odp.plan_traffic(rows, cuts, X, Wp, Hp, Tp) == pytest.approx(cost, rel=1e-12)
    K.kf_dag_destroy(dag)


def test_recompute_wins_where_a_cut_separates_a_cheap_node_from_its_late_reader(ctx):
    # 1 = affine(frame), 2..4 = 7x7 binomials, 5 = product(4, 1): with a limit that forbids
    # full fusion, recomputing node 1 from the frame beats storing and reading it back
    rows = [(1, 0, -1, 0, 2.0, 0.0), (4, 1, -1, 3, 0, 0), (4, 2, -1, 3, 0, 0), (4, 3, -1, 3, 0, 0), (3, 4, 1, 0, 0, 0)]
    dag = K.kf_dag_create(ctx, rows)
    full = odp.onchip_bytes(rows, 1, 5, set())
    limit = full - 1
    cuts, xm, cost = K.kf_dag_plan_recompute(dag, 64, 32, 1, limit)
    assert xm & 1
    contiguous = min(odp.plan_traffic(rows, c, set(), 64, 32, 1) for c in range(16)
                     if all(odp.onchip_bytes(rows, a, b, set()) <= limit for a, b in odp.ranges(5, c)))
    assert cost < contiguous
    K.kf_dag_destroy(dag)


def test_never_worse_than_the_best_contiguous_partition(ctx):
    for seed in list(range(4000, 4006)) + list(range(5000, 5006)):
        rows = sd.to_array(sd.random_dag(seed) if seed < 5000 else sd.deep_dag(seed))
        n = len(rows)
        dag = K.kf_dag_create(ctx, rows)
        for limit in (0, 60000):
            lim = limit or 200 * 1024
            costs = []
            for a in range(n):
                for b in range(a, n):
                    _, oc, tr = K.kf_dag_group_info(dag, a, b, W, H, T)
                    costs.append(tr if oc <= lim else -1)
            _, best_contiguous = K.kf_dag_plan(dag, costs)
            cuts, xm, cost = K.kf_dag_plan_recompute(dag, W, H, T, limit)
            assert cost <= best_contiguous * (1 + 1e-12)
            t, m = K.kf_dag_xplan_traffic(dag, cuts, xm, W, H, T)
            assert t == pytest.approx(cost, rel=1e-12) and m <= lim
        K.kf_dag_destroy(dag)


def test_learned_cost_plans(ctx):
    rows = sd.to_array(sd.random_dag(4021))
    n = len(rows)
    dag = K.kf_dag_create(ctx, rows)
    with pytest.raises(K.KfuseError):  # no model trained or set
        K.kf_dag_plan_recompute(dag, W, H, T, model=ctx)
    rng = np.random.default_rng(8)
    p = rng.normal(scale=0.2, size=K.KF_MLP_NPARAMS).astype(np.float32)
    norm = np.concatenate([rng.normal(size=K.KF_NFEAT), rng.uniform(0.5, 2.0, K.KF_NFEAT), [0.3], [1.7]]).astype(np.float32)
    K.kf_costmodel_set(ctx, p, norm)
    feats, groups = [], []
    for a in range(n):
        for b in range(a, n):
            f, oc, _ = K.kf_dag_group_info(dag, a, b, W, H, T)
            feats.append(f)
            groups.append(oc <= 200 * 1024)
    pred = K.kf_costmodel_predict(ctx, np.array(feats, dtype=np.float32))
    _, best_contiguous = K.kf_dag_plan(dag, [float(c) if ok else -1.0 for c, ok in zip(pred, groups)])
    cuts, xm, cost = K.kf_dag_plan_recompute(dag, W, H, T, model=ctx)
    assert cost <= best_contiguous * (1 + 1e-5)
    assert not (xm >> (n - 1))
    K.kf_dag_destroy(dag)


def test_bad_plans_are_rejected(ctx):
    rows = sd.to_array(sd.random_dag(4002))
    n = len(rows)
    dag = K.kf_dag_create(ctx, rows)
    for cuts, xm in [(0, 1 << (n - 1)), (0, 1 << n), (1 << (n - 1), 0)]:  # output inlined; past the DAG
        with pytest.raises(K.KfuseError):
            K.kf_dag_xplan_traffic(dag, cuts, xm, W, H, T)
    K.kf_dag_destroy(dag)
