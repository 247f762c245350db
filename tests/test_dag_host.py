"""Host-side planning over kernel DAGs (CPU only): the DP over per-group costs equals the
brute-force minimum over all 2^(n-1) partitions; features, on-chip bytes and traffic are
consistent with the group structure."""
import math

import numpy as np
import pytest

from oracle import partition as op
from paper_1509_04394_gb300 import build as kbuild
from paper_1509_04394_gb300 import kfuse as K
from synth import dags as sd


@pytest.fixture(scope="module", autouse=True)
def _built():
    kbuild.build()


@pytest.mark.parametrize("seed", range(8))
def test_dag_plan_is_the_brute_force_minimum(seed):
    rows = sd.to_array(sd.random_dag(seed, 3, 12))
    n = len(rows)
    ctx = K.kf_create(-1)
    dag = K.kf_dag_create(ctx, rows)
    rng = np.random.default_rng(seed)
    cost = [float(rng.uniform(0.1, 5.0)) if rng.random() > 0.1 else -1.0 for _ in range(n * (n + 1) // 2)]
    best = None
    for groups in op.all_partitions(n):
        cs = [cost[K.group_index(n, a, b)] for a, b in groups]
        if any(c < 0 for c in cs):
            continue
        tot = sum(cs)
        best = tot if best is None or tot < best else best
    if best is None:
        with pytest.raises(K.KfuseError):
            K.kf_dag_plan(dag, cost)
    else:
        cuts, c = K.kf_dag_plan(dag, cost)
        assert c == pytest.approx(best, rel=1e-12)
        assert sum(cost[K.group_index(n, a, b)] for a, b in op.groups_of(n, cuts)) == pytest.approx(best, rel=1e-12)
    K.kf_dag_destroy(dag)
    K.kf_destroy(ctx)


def test_group_info_is_consistent():
    rows = sd.to_array(sd.random_dag(11))
    n = len(rows)
    ctx = K.kf_create(-1)
    dag = K.kf_dag_create(ctx, rows)
    W, H, T = 1920, 1080, 240
    for a in range(n):
        f1, oc1, tr1 = K.kf_dag_group_info(dag, a, a, W, H, T)
        assert f1[0] <= 1 and f1[11] == pytest.approx(math.log(W * H * T), rel=1e-6)
        if f1[0] == 1:
            assert tr1 > 0 and oc1 > 0
        else:  # a dead node (read by nobody, not the output) is not computed
            assert tr1 == 0 and oc1 == 0
    # fusing everything stores only the output node
    f, oc, tr = K.kf_dag_group_info(dag, 0, n - 1, W, H, T)
    assert f[10] == 1 and f[9] == 1  # one external input (the frame), one stored output
    assert f[5] == 4.0
    with pytest.raises(K.KfuseError):
        K.kf_dag_group_info(dag, 3, 2, W, H, T)
    K.kf_dag_destroy(dag)
    K.kf_destroy(ctx)


def test_dag_validation():
    ctx = K.kf_create(-1)
    with pytest.raises(K.KfuseError):
        K.kf_dag_create(ctx, [(1, 1, -1, 0, 1.0, 0.0)])  # reads itself
    with pytest.raises(K.KfuseError):
        K.kf_dag_create(ctx, [(4, 0, -1, 4, 0.0, 0.0)])  # radius 4
    with pytest.raises(K.KfuseError):
        K.kf_dag_create(ctx, [(3, 0, -1, 0, 0.0, 0.0)])  # product without a second input
    K.kf_destroy(ctx)
