"""GPU parity of the fused DAG executor against the FP64 oracle.

Every node is computed by the same formula whatever the grouping, so every partition
(and every plan with recomputed nodes) must give the same bits; the results stay within
the per-pixel FP32 error bound of the stage definitions (running error analysis of the
oracle's FP64 values, `oracle.dag.fp32_error_bounds`) and within 1e-5 normwise of the
FP64 oracle, across chains of up to 24 FP32 stages."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dag as od  # noqa: E402
from paper_1509_04394_gb300 import build as kbuild  # noqa: E402
from paper_1509_04394_gb300 import kfuse as K  # noqa: E402
from synth import dags as sd  # noqa: E402
from synth import video as sv  # noqa: E402
from tests._parity import TOL_F32, normwise  # noqa: E402


def check_output(rows, frame_u8, got):
    """One frame of the DAG's output against the oracle: inside the per-pixel FP32 bound
    and within the FP32 tolerance normwise."""
    ref = od.run_frame(rows, frame_u8)[-1]
    bound = od.fp32_error_bounds(rows, frame_u8)[-1]
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= bound), float(np.max(err - bound))
    assert normwise(got, ref) <= TOL_F32


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("seed,shape", [(1, (2, 37, 53)), (2, (2, 64, 96)), (3, (3, 16, 32)), (4, (1, 5, 7)),
                                        (5, (2, 70, 130))])
def test_dag_partitions_match_the_oracle(dev, seed, shape):
    T, H, W = shape
    rows = sd.to_array(sd.random_dag(seed))
    n = len(rows)
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=seed, n_blobs=4, n_patches=2), pitch=sv.pitch_for(W))
    ctx = K.Context(0, harris=False)
    dag = K.kf_dag_create(ctx.h, rows)
    f = torch.from_numpy(fr).to(dev)
    ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(seed)
    parts = [(1 << (n - 1)) - 1, 0] + [int(rng.integers(0, 1 << (n - 1))) for _ in range(4)]
    outs = {}
    for cuts in parts:
        out = torch.full((T, H, sv.pitch_for(W)), float("nan"), dtype=torch.float32, device=dev)
        try:
            K.kf_dag_run(dag, cuts, f, W, out, ws)
        except K.KfuseError as e:
            assert e.status == K.KF_ESMEM  # a group too large for shared memory
            continue
        outs[cuts] = out[:, :, :W].cpu()
    ref = outs[(1 << (n - 1)) - 1]
    for cuts, o in outs.items():
        assert torch.equal(o, ref), cuts
    for t in range(T):
        check_output(rows, fr[t][:, :W], ref[t].numpy())
    K.kf_dag_destroy(dag)


def test_group_timing_covers_every_group(dev):
    rows = sd.to_array(sd.random_dag(9, 12, 14))
    n = len(rows)
    T, H, W = 2, 128, 256
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=9), pitch=sv.pitch_for(W))
    ctx = K.Context(0, harris=False)
    dag = K.kf_dag_create(ctx.h, rows)
    f = torch.from_numpy(fr).to(dev)
    ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=dev)
    out = torch.zeros((T, H, W), dtype=torch.float32, device=dev)
    ms = K.kf_dag_time_groups(dag, n, f, W, out, ws, reps=2)
    assert len(ms) == n * (n + 1) // 2
    for a in range(n):
        for b in range(a, n):
            _, onchip, _ = K.kf_dag_group_info(dag, a, b, W, H, T)
            t = ms[K.group_index(n, a, b)]
            assert (t > 0) == (onchip <= 200 * 1024), (a, b, t, onchip)
    K.kf_dag_destroy(dag)


@pytest.mark.parametrize("seed,shape,deep", [(11, (2, 40, 70), False), (12, (2, 64, 96), True), (13, (1, 9, 13), True),
                                             (14, (2, 50, 33), False), (15, (2, 45, 120), True)])
def test_plans_with_recomputed_nodes_give_the_same_bits(dev, seed, shape, deep):
    """Plans that recompute inlined nodes in their consumer groups compute every node by
    the same formula: bit-identical to the unfused run, including the planner's own plans
    (traffic and a tight on-chip limit), and so within the FP32 bound of the oracle, which
    checks the unfused run (random and deep DAGs) frame by frame."""
    T, H, W = shape
    rows = sd.to_array(sd.deep_dag(5000 + seed) if deep else sd.random_dag(seed))
    n = len(rows)
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=seed, n_blobs=4, n_patches=2), pitch=sv.pitch_for(W))
    ctx = K.Context(0, harris=False)
    dag = K.kf_dag_create(ctx.h, rows)
    f = torch.from_numpy(fr).to(dev)
    ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=dev)
    P = sv.pitch_for(W)
    ref = torch.full((T, H, P), float("nan"), dtype=torch.float32, device=dev)
    K.kf_dag_run(dag, (1 << (n - 1)) - 1, f, W, ref, ws)
    ref_h = ref[:, :, :W].cpu().numpy()
    for t in range(T):
        check_output(rows, fr[t][:, :W], ref_h[t])
    rng = np.random.default_rng(seed)
    plans = [(int(rng.integers(0, 1 << (n - 1))), int(rng.integers(0, 1 << (n - 1)))) for _ in range(6)]
    plans.append(K.kf_dag_plan_recompute(dag, W, H, T)[:2])
    plans.append(K.kf_dag_plan_recompute(dag, W, H, T, 30000)[:2])
    ran = 0
    for cuts, xm in plans:
        out = torch.full((T, H, P), float("nan"), dtype=torch.float32, device=dev)
        try:
            K.kf_dag_run_x(dag, cuts, xm, f, W, out, ws)
        except K.KfuseError as e:
            assert e.status == K.KF_ESMEM
            continue
        ran += 1
        assert torch.equal(out[:, :, :W], ref[:, :, :W]), (cuts, xm)
        if xm:  # a plan that recomputes nodes, against the oracle directly
            check_output(rows, fr[0][:, :W], out[0, :, :W].cpu().numpy())
    assert ran >= 2
    K.kf_dag_destroy(dag)


def test_timing_groups_with_inlined_nodes(dev):
    """kf_dag_time_xgroups: a time for every feasible group, and with no inlined node
    the features of the contiguous group."""
    from paper_1509_04394_gb300 import costmodel as cm
    rows = sd.to_array(sd.random_dag(21, 12, 14))
    n = len(rows)
    T, H, W = 2, 96, 160
    fr, _ = sv.generate(sv.VideoSpec(T=T, H=H, W=W, seed=21), pitch=sv.pitch_for(W))
    ctx = K.Context(0, harris=False)
    dag = K.kf_dag_create(ctx.h, rows)
    f = torch.from_numpy(fr).to(dev)
    ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=dev)
    out = torch.zeros((T, H, W), dtype=torch.float32, device=dev)
    groups = cm.inlined_samples(rows, 3, 12) + [(0, n - 1, 0), (2, 5, 0)]
    ms, feats = K.kf_dag_time_xgroups(dag, groups, f, W, out, ws, reps=2)
    for (a, b, xm), t, ft in zip(groups, ms, feats):
        assert t > 0 or t == -1
        if xm == 0:
            fi, oc, _ = K.kf_dag_group_info(dag, a, b, W, H, T)
            np.testing.assert_array_equal(ft, np.array(fi, dtype=np.float32))
            assert (t > 0) == (oc <= 200 * 1024)
    with pytest.raises(K.KfuseError):  # the output node may not be inlined
        K.kf_dag_time_xgroups(dag, [(0, 1, 1 << (n - 1))], f, W, out, ws)
    K.kf_dag_destroy(dag)
