"""Learned cost model workflow: measure, train, plan, evaluate (argument marshalling and
bookkeeping only; every measurement, the training and the planning DP run in libkfuse).

1. measure(): for a random kernel DAG, the executor times every one of its n(n+1)/2
   candidate fused groups on a video (kf_dag_time_groups) and reports each group's
   features, on-chip bytes and Sec. VI-D traffic (kf_dag_group_info);
2. train(): the library fits its MLP to (features, measured ms) of the training DAGs'
   feasible groups (kf_costmodel_train, GPU kernels);
3. plan_costs(): per-group costs under three models -- measured ms (the exhaustive
   optimum: the DP over measured group times is the minimum over all 2^(n-1)
   partitions), the analytic traffic model, and the MLP's predictions -- each planned by
   the same exact DP (kf_dag_plan);
4. evaluate(): the measured cost of each model's chosen partition relative to the
   measured optimum (regret), per held-out DAG.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import kfuse as K


@dataclasses.dataclass
class Measured:
    seed: int
    n: int
    rows: list
    ms: np.ndarray        # [G] measured group time, -1 infeasible
    feats: np.ndarray     # [G, KF_NFEAT]
    traffic: np.ndarray   # [G] bytes
    onchip: np.ndarray    # [G] bytes


def measure(ctx, rows, frames, W: int, seed: int, reps: int = 2) -> Measured:
    import torch
    T, H, _ = frames.shape
    n = len(rows)
    dag = K.kf_dag_create(ctx, rows)
    try:
        ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=frames.device)
        out = torch.empty((T, H, W), dtype=torch.float32, device=frames.device)
        ms = np.array(K.kf_dag_time_groups(dag, n, frames, W, out, ws, reps=reps), dtype=np.float64)
        G = n * (n + 1) // 2
        feats = np.zeros((G, K.KF_NFEAT), dtype=np.float32)
        traffic, onchip = np.zeros(G), np.zeros(G)
        for a in range(n):
            for b in range(a, n):
                g = K.group_index(n, a, b)
                f, oc, tr = K.kf_dag_group_info(dag, a, b, W, H, T)
                feats[g], onchip[g], traffic[g] = f, oc, tr
        del ws, out
    finally:
        K.kf_dag_destroy(dag)
    return Measured(seed, n, rows, ms, feats, traffic, onchip)


def inlined_samples(rows, seed: int, count: int = 60) -> list[tuple[int, int, int]]:
    """(first, last, inline_mask) groups of plans that recompute nodes: a random range
    and a random non-empty set of the stored maps it reads (sometimes with one of their
    own stored inputs, or one of its own nodes), drawn from a seeded generator."""
    n = len(rows)
    rng = np.random.default_rng(seed)

    def inputs(j):
        kind, i1, i2 = rows[j - 1][0], rows[j - 1][1], rows[j - 1][2]
        return [i1, i2] if kind == 3 else [i1]
    out, tries = [], 0
    while len(out) < count and tries < 20 * count:
        tries += 1
        a = int(rng.integers(1, n + 1))
        b = int(rng.integers(a, n + 1))
        ext = sorted({i for j in range(a, b + 1) for i in inputs(j) if 0 < i < a})
        if not ext:
            continue
        pick = [e for e in ext if rng.random() < 0.5] or [ext[int(rng.integers(len(ext)))]]
        X = set(pick)
        if rng.random() < 0.3:
            deeper = sorted({i for e in pick for i in inputs(e) if i > 0})
            if deeper:
                X.add(deeper[int(rng.integers(len(deeper)))])
        if rng.random() < 0.2 and b > a:
            X.add(int(rng.integers(a, b)))  # a range node, never the output n
        X.discard(n)
        mask = sum(1 << (j - 1) for j in X)
        out.append((a - 1, b - 1, mask))
    return out


def measure_inlined(ctx, rows, frames, W: int, seed: int, count: int = 60, reps: int = 2):
    """(features, ms) of sampled groups with inlined nodes (feasible ones only)."""
    import torch
    T, H, _ = frames.shape
    dag = K.kf_dag_create(ctx, rows)
    try:
        ws = torch.empty(K.kf_dag_workspace_bytes(dag, W, H, T), dtype=torch.uint8, device=frames.device)
        out = torch.empty((T, H, W), dtype=torch.float32, device=frames.device)
        groups = inlined_samples(rows, seed, count)
        ms, feats = K.kf_dag_time_xgroups(dag, groups, frames, W, out, ws, reps=reps)
        del ws, out
    finally:
        K.kf_dag_destroy(dag)
    ok = ms > 0
    return feats[ok], ms[ok].astype(np.float64)


def dataset(ms_list: list[Measured]):
    X = np.concatenate([m.feats[m.ms > 0] for m in ms_list])
    y = np.concatenate([m.ms[m.ms > 0] for m in ms_list])
    return X, y


def partition_cost(m: Measured, cuts: int) -> float:
    """Measured cost of a partition: the sum of its groups' measured times."""
    a, tot = 0, 0.0
    for i in range(m.n):
        if i == m.n - 1 or (cuts >> i) & 1:
            t = m.ms[K.group_index(m.n, a, i)]
            if t <= 0:
                return math.inf
            tot += t
            a = i + 1
    return tot


def plan_costs(ctx, m: Measured) -> dict[str, int]:
    """Cut mask chosen under each cost model (infeasible groups excluded everywhere)."""
    dag = K.kf_dag_create(ctx, m.rows)
    try:
        feasible = m.ms > 0
        measured = np.where(feasible, m.ms, -1.0)
        traffic = np.where(feasible, m.traffic, -1.0)
        pred = K.kf_costmodel_predict(ctx, m.feats).astype(np.float64)
        mlp = np.where(feasible, pred, -1.0)
        return {"measured": K.kf_dag_plan(dag, measured)[0], "traffic": K.kf_dag_plan(dag, traffic)[0],
                "mlp": K.kf_dag_plan(dag, mlp)[0]}
    finally:
        K.kf_dag_destroy(dag)


def evaluate(ctx, held_out: list[Measured]) -> dict:
    rows = []
    for m in held_out:
        plans = plan_costs(ctx, m)
        opt = partition_cost(m, plans["measured"])
        rows.append({"seed": m.seed, "n": m.n, "opt_ms": opt,
                     "traffic_regret": partition_cost(m, plans["traffic"]) / opt - 1.0,
                     "mlp_regret": partition_cost(m, plans["mlp"]) / opt - 1.0,
                     "plans": plans})
    tr = np.array([r["traffic_regret"] for r in rows])
    ml = np.array([r["mlp_regret"] for r in rows])
    small = np.array([r["n"] <= 13 for r in rows])
    return {"dags": len(rows), "traffic_mean_regret": float(tr.mean()), "mlp_mean_regret": float(ml.mean()),
            "traffic_median_regret": float(np.median(tr)), "mlp_median_regret": float(np.median(ml)),
            "mlp_better_or_equal": int(np.sum(ml <= tr + 1e-12)),
            "enumerable_dags": int(small.sum()),
            "enumerable_traffic_mean_regret": float(tr[small].mean()) if small.any() else None,
            "enumerable_mlp_mean_regret": float(ml[small].mean()) if small.any() else None,
            "per_dag": rows}
