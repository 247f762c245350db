"""The C ABI on the host (no GPU): symbols, argument checks, and the partitioner.

The library's dynamic program must find the same optimum as the oracle's brute-force
enumeration of all 2^(n-1) partitions (Sec. VI, Fig. 5) under the traffic model of
Sec. VI-D, on the Harris chain and on random chains of up to 12 kernels.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import partition as op
from paper_1509_04394_gb300 import build as kbuild
from paper_1509_04394_gb300 import kfuse as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    kbuild.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kfuse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    import ctypes
    lib = ctypes.CDLL(K.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(K.exported_symbols()) == names


def declared_arity():
    """Parameter count of every function kfuse.h declares."""
    src = open(os.path.join(ROOT, "include", "kfuse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(kf_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    arity = declared_arity()
    assert len(arity) == len(declared_functions())
    L = K._lib()
    for name, n in arity.items():
        f = getattr(L, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)


def test_version_and_status_strings():
    assert K.kf_version() == (1, 0)
    L = K._lib()
    for s in range(8):
        assert L.kf_status_str(s)


@pytest.fixture
def hctx():
    h = K.kf_create(-1)
    yield h
    K.kf_destroy(h)


def test_host_only_context_refuses_to_run(hctx):
    K.kf_add_harris_chain(hctx)
    with pytest.raises(K.KfuseError) as e:
        K._check("kf_run", K._lib().kf_run(hctx, 0, None, None, None, 0, None))
    assert e.value.status in (K.KF_ESTATE, K.KF_EINVAL)
    st = K._lib().kf_run_group(hctx, 0, 7, None, None, 8, 8, 1, None, None)
    assert st == K.KF_ESTATE


def test_argument_checks(hctx):
    L = K._lib()
    with pytest.raises(K.KfuseError):
        K.kf_add_stage(hctx, K.KF_STAGE_GAUSS_H if hasattr(K, "KF_STAGE_GAUSS_H") else 2, rx=3)  # builtin radii fixed
    with pytest.raises(K.KfuseError):
        K.kf_add_stage(hctx, 0, rx=-1, in_bytes=1, out_bytes=1)
    with pytest.raises(K.KfuseError):
        K.kf_add_stage(hctx, 0, rx=1)  # custom stage without byte counts
    with pytest.raises(K.KfuseError):
        K.kf_set_precision(hctx, 7)
    with pytest.raises(K.KfuseError):
        K.kf_set_chunk_rows(hctx, 0)
    K.kf_add_harris_chain(hctx)
    with pytest.raises(K.KfuseError):
        K.kf_add_harris_chain(hctx)
    with pytest.raises(K.KfuseError):
        K.kf_partition_traffic(hctx, 1 << 7, 600, 800, 10)
    with pytest.raises(K.KfuseError):
        K.kf_partition_traffic(hctx, 0, 0, 800, 10)
    with pytest.raises(K.KfuseError):
        K.kf_group_traffic(hctx, 3, 2, 600, 800, 10)
    with pytest.raises(K.KfuseError):
        K.kf_workspace_bytes(hctx, 1 << 7, 600, 800, 10)
    assert L.kf_plan(hctx, None, 1.0, None, None) == K.KF_EINVAL
    for _ in range(KF_MAX := 24 - 8):
        K.kf_add_stage(hctx, 0, in_bytes=1, out_bytes=1)
    with pytest.raises(K.KfuseError):
        K.kf_add_stage(hctx, 0, in_bytes=1, out_bytes=1)


def oracle_stages(elem):
    return op.harris_chain(elem)


@pytest.mark.parametrize("prec,elem", [(K.KF_PREC_F32, 4), (K.KF_PREC_F16, 2)])
@pytest.mark.parametrize("geom", [(600, 800, 1000, (116, 200, 1)), (432, 192, 600, (116, 64, 1)),
                                  (256, 256, 1000, (8, 8, 8)), (1920, 1080, 240, (32, 16, 1))])
def test_traffic_model_and_plan_match_the_oracle_on_the_harris_chain(hctx, prec, elem, geom):
    W, H, T, box = geom
    K.kf_set_precision(hctx, prec)
    K.kf_add_harris_chain(hctx)
    st = oracle_stages(elem)
    for cuts in range(128):
        got = K.kf_partition_traffic(hctx, cuts, W, H, T, box)
        exp = op.partition_cost(st, op.groups_of(8, cuts), W, H, T, box)
        assert got == pytest.approx(exp, rel=1e-12)
    for a, b in op.candidate_groups(8):
        assert K.kf_group_onchip(hctx, a, b, W, H, T, box) == pytest.approx(op.group_onchip(st, a, b, box), rel=1e-12)
    for limit in (math.inf, 20000.0, 8000.0, 600.0):
        best = op.brute_force_best(st, W, H, T, box, limit)
        if best is None:
            with pytest.raises(K.KfuseError) as e:
                K.kf_plan(hctx, W, H, T, box, limit)
            assert e.value.status == K.KF_ESMEM
            continue
        cuts, cost = K.kf_plan(hctx, W, H, T, box, limit)
        g, c = best
        assert cost == pytest.approx(c, rel=1e-12)
        assert op.feasible(st, op.groups_of(8, cuts), box, limit)
        assert K.kf_partition_traffic(hctx, cuts, W, H, T, box) == pytest.approx(cost, rel=1e-12)


@pytest.mark.parametrize("seed", range(12))
def test_plan_matches_brute_force_on_random_chains(hctx, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 13))
    st = []
    for i in range(n):
        s = op.Stage(f"s{i}", int(rng.integers(0, 4)), int(rng.integers(0, 4)), int(rng.integers(0, 2)),
                     float(rng.choice([1, 2, 4, 8, 12])), float(rng.choice([1, 2, 4, 8, 12])))
        st.append(s)
        K.kf_add_stage(hctx, 0, s.rx, s.ry, s.rt, s.in_bytes, s.out_bytes)
    assert K.kf_num_stages(hctx) == n
    assert K.kf_enumerate(hctx) == list(range(2 ** (n - 1)))
    box = (int(rng.choice([8, 16, 32, 64])), int(rng.choice([8, 16, 32])), int(rng.choice([1, 4, 8])))
    W, H, T = 512, 384, 100
    limit = float(rng.choice([math.inf, 30000.0, 120000.0]))
    best = op.brute_force_best(st, W, H, T, box, limit)
    if best is None:
        with pytest.raises(K.KfuseError) as e:
            K.kf_plan(hctx, W, H, T, box, limit)
        assert e.value.status == K.KF_ESMEM
        return
    cuts, cost = K.kf_plan(hctx, W, H, T, box, limit)
    assert cost == pytest.approx(best[1], rel=1e-12)
    assert op.feasible(st, op.groups_of(n, cuts), box, limit)


def test_workspace_accounts_for_the_cut_maps(hctx):
    K.kf_add_harris_chain(hctx)
    W, H, T = 600, 800, 10
    assert K.kf_workspace_bytes(hctx, 0, W, H, T) == 0
    pitch = 600  # W rounded up to 8 elements
    one = pitch * H * T * 4
    # unfused: the widest maps are 3 channels, alternating between two buffers
    assert K.kf_workspace_bytes(hctx, 127, W, H, T) == 2 * 3 * one
    assert K.kf_workspace_bytes(hctx, 1 << 6, W, H, T) == one  # cut before NMS: R only
    K.kf_set_precision(hctx, K.KF_PREC_F16)
    assert K.kf_workspace_bytes(hctx, 1 << 6, W, H, T) == one // 2


def test_map_scales(hctx):
    K.kf_add_harris_chain(hctx)
    assert K.kf_map_scale(hctx, 0) == pytest.approx(1 / 255)
    assert K.kf_map_scale(hctx, 2) == pytest.approx(1 / 65280)
    assert K.kf_map_scale(hctx, 6) == pytest.approx(65280.0 ** -4)
    K.kf_set_precision(hctx, K.KF_PREC_F16)
    assert K.kf_map_scale(hctx, 2) == pytest.approx(1 / 65280)  # exact uint16 map
    assert all(K.kf_map_scale(hctx, s) == 1.0 for s in range(3, 8))  # FP16, true units


def test_workspace_sizes_refuse_volumes_whose_byte_counts_could_overflow(hctx):
    # every side 1..2^30, at most 2^31 - 1 frames and 2^46 pixels: the byte counts at the
    # bound are exact (no 64-bit wrap), one step past it is refused
    from synth import dags as sd
    K.kf_add_harris_chain(hctx)
    side, lim = 1 << 30, 1 << 46
    ok = [(side, 1 << 16, 1), (1 << 13, 1 << 13, 1 << 20)]
    bad = [(side + 1, 4, 1), (4, side + 1, 1), (4, 4, 1 << 31), (side, 1 << 16, 2), (1 << 13, 1 << 13, (1 << 20) + 1),
           (1 << 40, 1 << 40, 1 << 40), (0, 4, 1), (4, 4, -1)]
    dag = K.kf_dag_create(hctx, sd.to_array(sd.random_dag(1)))
    for W, H, T in ok:
        assert W * H * T == lim
        assert K.kf_workspace_bytes(hctx, 127, W, H, T) >= 2 * 4 * W * H * T  # the cut maps, double buffered
        assert K.kf_pc_workspace_bytes(hctx, 15, W, H, T) >= 2 * 4 * W * H * T
        assert K.kf_pc_group_workspace_bytes(hctx, 0, 4, W, H, T) >= 4 * W * H
        assert K.kf_dag_workspace_bytes(dag, W, H, T) >= 4 * W * H * T
    for W, H, T in bad:
        for call in (lambda: K.kf_workspace_bytes(hctx, 127, W, H, T),
                     lambda: K.kf_pc_workspace_bytes(hctx, 15, W, H, T),
                     lambda: K.kf_pc_group_workspace_bytes(hctx, 0, 4, W, H, T),
                     lambda: K.kf_dag_workspace_bytes(dag, W, H, T),
                     lambda: K.kf_track_workspace_bytes(hctx, W, H, T)):
            with pytest.raises(K.KfuseError):
                call()
    # the tracking workspace also needs W * H below 2^31
    assert K.kf_track_workspace_bytes(hctx, 1 << 15, 1 << 15, 1 << 16) > 0
    with pytest.raises(K.KfuseError):
        K.kf_track_workspace_bytes(hctx, 1 << 16, 1 << 15, 1)
    # a batch within the bound as a whole
    L = K._lib()
    vids = (K.kf_video * 2)(K.kf_video(16, 1 << 13, 1 << 13, 1 << 19, 1 << 13), K.kf_video(16, 1 << 13, 1 << 13, 1 << 19, 1 << 13))
    b = ctypes.c_size_t()
    assert L.kf_batch_workspace_bytes(hctx, vids, 2, 0, ctypes.byref(b)) == K.KF_OK and b.value > 0
    vids[1].T += 1
    assert L.kf_batch_workspace_bytes(hctx, vids, 2, 0, ctypes.byref(b)) == K.KF_EINVAL
    K.kf_dag_destroy(dag)
